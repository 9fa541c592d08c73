"""Plain propagations of 64 x 64 fields at padding 2 (128-point transforms) run as one on-chip
kernel: the results match the float64 oracle (forward, adjoint, every method, per-field lambda
and z, in place, batches that span launch chunks) and agree with the three-pass path to rounding."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

THREE_PASS = 0x800
TOL = 1e-5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2411_18591_gb300 as T
    return T


def fields(seed, b, n=64):
    x = S.normal(seed, (b, n, n)) + 1j * S.normal(S.sub_seed(seed, 1), (b, n, n))
    return S.to_c64(x)


def onchip_launches(T, fn):
    """Runs fn with the library's timing on; returns (result, on-chip launches, three-pass launches)."""
    T.binding.profile_enable(True)
    try:
        out = fn()
        torch.cuda.synchronize()
        pr = T.binding.profile_read()
    finally:
        T.binding.profile_enable(False)
    return out, pr.get("onchip", (0.0, 0))[1], pr.get("cols", (0.0, 0))[1]


@pytest.mark.parametrize("method", ["as", "fresnel", "di"])
def test_forward_and_adjoint_match_oracle(T, rel, method):
    b, d = 5, 10e-6
    x0 = fields(301, b)
    lams = [450e-9, 532e-9, 633e-9, 700e-9, 532e-9]
    zs = [0.004, 0.02, 0.05, 0.1, 0.0125]
    x = torch.from_numpy(x0).cuda()
    m = {"as": O.AS, "fresnel": O.FRESNEL_TF, "di": O.DI}[method]
    y, n_on, n_cols = onchip_launches(T, lambda: T.top_propagate(x, d, d, lams, zs, 2.0, method))
    assert n_on >= 1 and n_cols == 0
    ref = O.propagate(x0, d, d, lams, zs, 2.0, m)
    assert rel(y.cpu().numpy(), ref) < TOL
    g, n_on, n_cols = onchip_launches(T, lambda: T.top_propagate_backward(x, d, d, lams, zs, 2.0, method))
    assert n_on >= 1 and n_cols == 0
    gref = O.propagate_adjoint(x0, d, d, lams, zs, 2.0, m)
    assert rel(g.cpu().numpy(), gref) < TOL


def test_agrees_with_three_passes(T, rel):
    b, d = 7, 8e-6
    x = torch.from_numpy(fields(302, b)).cuda()
    lams = [450e-9 + 40e-9 * i for i in range(b)]
    zs = [0.01 + 0.005 * i for i in range(b)]
    T.autotune_clear()
    try:
        on = T.top_propagate(x, d, d, lams, zs, 2.0)
        on_adj = T.top_propagate_backward(x, d, d, lams, zs, 2.0)
        T.autotune_set(64, THREE_PASS)
        (three, n_on, n_cols) = onchip_launches(T, lambda: T.top_propagate(x, d, d, lams, zs, 2.0))
        assert n_on == 0 and n_cols >= 1
        three_adj = T.top_propagate_backward(x, d, d, lams, zs, 2.0)
    finally:
        T.autotune_clear()
    assert rel(on.cpu().numpy(), three.cpu().numpy()) < 1e-6
    assert rel(on_adj.cpu().numpy(), three_adj.cpu().numpy()) < 1e-6


def test_in_place_equals_out_of_place(T):
    d = 10e-6
    x = torch.from_numpy(fields(303, 3)).cuda()
    y = T.top_propagate(x, d, d, 633e-9, 0.03, 2.0)
    x2 = x.clone()
    T.top_propagate(x2, d, d, 633e-9, 0.03, 2.0, out=x2)
    torch.cuda.synchronize()
    assert torch.equal(x2, y)


def test_batch_across_launch_chunks(T, rel):
    # more fields than one launch takes (2048), two (lambda, z) sets alternating
    b, d = 2101, 10e-6
    x0 = fields(304, b)
    lams = [532e-9 if i % 2 else 633e-9 for i in range(b)]
    zs = [0.02 if i % 2 else 0.05 for i in range(b)]
    x = torch.from_numpy(x0).cuda()
    y = T.top_propagate(x, d, d, lams, zs, 2.0).cpu().numpy()
    for i in (0, 1, 1023, 2046, 2047, 2048, 2100):
        ref = O.propagate(x0[i:i + 1], d, d, lams[i], zs[i], 2.0)
        assert rel(y[i:i + 1], ref) < TOL, i


def test_modulated_requests_keep_the_three_passes(T, rel):
    # a phase mask on the source is not taken by the on-chip kernel; results still match the oracle
    d = 10e-6
    x0 = fields(305, 2)
    phi = S.uniform(306, (64, 64), -np.pi, np.pi).astype(np.float32)
    x = torch.from_numpy(x0).cuda()
    ph = torch.from_numpy(phi).cuda()
    y, n_on, n_cols = onchip_launches(T, lambda: T.top_propagate(x, d, d, 633e-9, 0.02, 2.0,
                                                                  pre=T.Modulation(phase=ph)))
    assert n_on == 0 and n_cols >= 1
    ref = O.propagate(x0 * np.exp(1j * phi.astype(np.float64)), d, d, 633e-9, 0.02, 2.0)
    assert rel(y.cpu().numpy(), ref) < TOL


def test_noalloc_call_takes_the_same_kernel(T):
    # the handle-free call gives top_propagate's results bit for bit at this size too
    d = 10e-6
    x = torch.from_numpy(fields(307, 5)).cuda()
    lams = [450e-9, 532e-9, 633e-9, 700e-9, 532e-9]
    ref = T.top_propagate(x, d, d, lams, 0.02, 2.0)
    out = torch.empty_like(x)
    T.top_propagate_noalloc(x, d, d, lams, 0.02, 2.0, out=out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
