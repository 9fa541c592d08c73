"""The autotuner's pass variants (pair-local or block-cooperative row passes, L2 prefetch on or
off, fields per block of the field epilogue) give the same results bit for bit, and the tuner
records a valid choice for the geometry it measured."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu

CLASSIC = 0x1 | 0x2 | 0x4
NO_L2 = 0x8 | 0x10


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2411_18591_gb300 as T
    return T


def field(seed, shape):
    x = S.normal(seed, shape) + 1j * S.normal(S.sub_seed(seed, 1), shape)
    return torch.from_numpy(S.to_c64(x)).cuda()


def run_all(T, x, phase, lams, d):
    pupil = T.Modulation(phase=phase, radius=1.5e-3)
    lens = T.Modulation(focal_length=0.1, radius=2.2e-3)
    out = [T.top_propagate(x, d, d, lams, 0.02, 2.0, pre=lens)]
    gp = torch.empty_like(phase)
    out.append(T.top_propagate_backward(x, d, d, lams, 0.02, 2.0, pre=pupil, post=lens, saved_in=x, grad_phase=gp))
    out.append(gp)
    keep = torch.empty_like(x)
    stages = [T.Stage(0.01, pre=pupil), T.Stage(0.02, pre=lens, keep=keep), T.Stage(0.01, pre=lens)]
    y, inten = T.top_fused_chain(x, d, d, lams, stages, 2.0, intensity_group=3)
    out += [y, inten, keep]
    gi = inten * 0.5
    gp2 = torch.empty_like(phase)
    back = [T.Stage(s.z, pre=s.pre) for s in stages]
    out.append(T.top_fused_chain_backward(y, gi, d, d, lams, back, 2.0, intensity_group=3, saved_in=x,
                                          grad_phase=gp2))
    out.append(gp2)
    torch.cuda.synchronize()
    return [o.clone() for o in out]


def test_variants_give_the_same_results(T):
    n, d = 1024, 5e-6
    x = field(81, (6, n, n))
    phase = torch.from_numpy(S.uniform(82, (n, n), -np.pi, np.pi).astype(np.float32)).cuda()
    lams = [450e-9, 575e-9, 700e-9] * 2
    T.autotune_clear()
    try:
        ref = run_all(T, x, phase, lams, d)
        for flags in (CLASSIC, NO_L2, (1 << 8), (2 << 8), (4 << 8), CLASSIC | NO_L2):
            T.autotune_set(1024, flags)
            got = run_all(T, x, phase, lams, d)
            for a, b in zip(got, ref):
                assert torch.equal(a, b), hex(flags)
    finally:
        T.autotune_clear()


def test_autotune_records_a_valid_choice(T, tmp_path):
    T.autotune_clear()
    try:
        rows, cols = T.top_autotune(16, 1024, 1024, 5e-6, 5e-6, 2.0)
        assert rows == T.autotune_get(1024) and cols == T.autotune_get(1024)
        assert (rows & ~0x71f) == 0
        path = tmp_path / "tune.txt"
        T.autotune_save(str(path))
        T.autotune_clear()
        T.autotune_load(str(path))
        assert T.autotune_get(1024) == rows
    finally:
        T.autotune_clear()
