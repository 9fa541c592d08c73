"""top_fused_chain: a system of propagations and modulations with the row passes between
consecutive propagations fused (GPU, through the C ABI).

The chain must equal the same sequence of top_propagate calls bit for bit (the fused kernel
does the same arithmetic), and the FP64 oracle within the parity tolerance.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

from conftest import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2411_18591_gb300 as T
    return T


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def fields(seed, b, ny, nx):
    return S.to_c64(S.normal(seed, (b, ny, nx)) + 1j * S.normal(S.sub_seed(seed, 1), (b, ny, nx)))


def fourf_like(T, ny, nx, d, seed):
    phi = S.uniform(S.sub_seed(seed, 2), (ny, nx), -np.pi, np.pi).astype(np.float32)
    pupil = T.Modulation(phase=dev(phi), radius=0.3 * min(ny, nx) * d)
    lens = T.Modulation(focal_length=0.05, radius=0.45 * min(ny, nx) * d)
    return phi, pupil, lens


@pytest.mark.parametrize("ny,nx,pad", [(256, 256, 2.0), (96, 48, 2.667), (250, 250, 2.0)])
def test_chain_equals_the_same_calls(T, ny, nx, pad):
    """Four stages (none, lens + kept output, pupil phase + aperture, lens), intensity groups of 3.
    250 columns are not 16-byte rows for the phase plane: that boundary runs unfused."""
    d = 6e-6
    lams = [450e-9, 575e-9, 700e-9] * 2
    x = dev(fields(31, 6, ny, nx))
    _, pupil, lens = fourf_like(T, ny, nx, d, 31)
    keep = torch.empty_like(x)
    zs = [2e-3, 3e-3, 1e-3, 2e-3]
    stages = [T.Stage(zs[0]), T.Stage(zs[1], pre=lens, keep=keep), T.Stage(zs[2], pre=pupil), T.Stage(zs[3], pre=lens)]
    out, inten = T.top_fused_chain(x, d, d, lams, stages, pad, intensity_group=3)
    y = T.top_propagate(x, d, d, lams, zs[0], pad)
    y = T.top_propagate(y, d, d, lams, zs[1], pad, pre=lens)
    k = y.clone()
    y = T.top_propagate(y, d, d, lams, zs[2], pad, pre=pupil)
    i_ref, y_ref = T.top_propagate_intensity(y, d, d, lams, zs[3], pad, group=3, pre=lens, keep_field=True)
    torch.cuda.synchronize()
    assert torch.equal(keep, k)
    assert torch.equal(out, y_ref)
    assert torch.equal(inten, i_ref)


def test_chain_matches_the_oracle(T):
    ny, nx, d, pad = 128, 128, 8e-6, 2.0
    lams = [480e-9, 633e-9]
    xh = fields(32, 2, ny, nx)
    phi, pupil, lens = fourf_like(T, ny, nx, d, 32)
    zs = [0.01, 0.02, 0.015]
    out, _ = T.top_fused_chain(dev(xh), d, d, lams, [T.Stage(zs[0]), T.Stage(zs[1], pre=pupil), T.Stage(zs[2], pre=lens)],
                               pad)
    pm = O.circ(ny, nx, d, d, 0.3 * ny * d) * np.exp(1j * phi.astype(np.float64))
    lm = np.stack([O.circ(ny, nx, d, d, 0.45 * ny * d) * O.lens(ny, nx, d, d, l, 0.05) for l in lams])
    o = O.propagate(xh.astype(np.complex128), d, d, lams, zs[0], pad)
    o = O.propagate(o * pm, d, d, lams, zs[1], pad)
    o = O.propagate(o * lm, d, d, lams, zs[2], pad)
    assert rel_l2(host(out), o) < 1e-5


def test_chain_input_repeat_intensity_only(T):
    ny, nx, d = 64, 64, 5e-6
    xh = fields(33, 2, ny, nx)
    lams = [500e-9, 600e-9, 700e-9] * 2
    lens = T.Modulation(focal_length=0.03)
    out, inten = T.top_fused_chain(dev(xh), d, d, lams, [T.Stage(1e-3), T.Stage(2e-3, pre=lens)], 2.0,
                                   intensity_group=3, input_repeat=3, want_field=False)
    assert out is None
    xr = np.repeat(xh, 3, axis=0).astype(np.complex128)
    o = O.propagate(xr, d, d, lams, 1e-3, 2.0)
    o = O.propagate(o * np.stack([O.lens(ny, nx, d, d, l, 0.03) for l in lams]), d, d, lams, 2e-3, 2.0)
    assert rel_l2(host(inten), O.intensity_sum(o, 3)) < 1e-5


def test_chain_rejects_bad_stages(T):
    x = dev(fields(34, 1, 32, 32))
    with pytest.raises(T.TopError, match="keep must be NULL"):
        T.top_fused_chain(x, 5e-6, 5e-6, 5e-7, [T.Stage(1e-3), T.Stage(1e-3, keep=torch.empty_like(x))])
    with pytest.raises(T.TopError, match="at least one stage"):
        T.top_fused_chain(x, 5e-6, 5e-6, 5e-7, [])
