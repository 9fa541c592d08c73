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


@pytest.mark.parametrize("ny,nx,pad", [(256, 256, 2.0), (96, 48, 2.667), (250, 250, 2.0), (1024, 1024, 2.0)])
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


def backward_chain_case(T, ny, nx, d, seed, b=6):
    lams = [450e-9, 575e-9, 700e-9] * (b // 3)
    x0 = dev(fields(seed, b, ny, nx))
    phi, pupil, lens = fourf_like(T, ny, nx, d, seed)
    mask = T.Modulation(mask=dev(fields(S.sub_seed(seed, 5), 1, ny, nx)[0] * 0.5))
    zs = [2e-3, 1e-3, 3e-3]
    stages = [T.Stage(zs[0], pre=pupil), T.Stage(zs[1], pre=lens), T.Stage(zs[2], pre=mask)]
    xk, _ = T.top_fused_chain(x0, d, d, lams, stages, 2.0 if ny > 61 else 1.0)
    gi = dev(S.normal(S.sub_seed(seed, 7), (b // 3, ny, nx)).astype(np.float32))
    return lams, x0, phi, pupil, lens, mask, zs, stages, xk, gi


@pytest.mark.parametrize("ny,nx", [(256, 256), (1024, 1024), (61, 61)])
def test_backward_chain_equals_the_same_calls(T, ny, nx):
    """The backward of a three-stage chain (pupil, lens, complex mask) from its grouped intensity:
    the phase gradient of the first stage's pupil and the input gradient, against the intensity
    backward of the last stage and the propagation backwards of the others. 61^2 fields at
    padding 1 have no plan: the fallback runs the same calls."""
    d = 6e-6
    pad = 2.0 if ny > 61 else 1.0
    lams, x0, phi, pupil, lens, mask, zs, stages, xk, gi = backward_chain_case(T, ny, nx, d, 41)
    gp = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    gin = T.top_fused_chain_backward(xk, gi, d, d, lams, stages, pad, intensity_group=3, saved_in=x0, grad_phase=gp)
    g = T.top_propagate_intensity_backward(xk, gi, d, d, lams, zs[2], pad, group=3, pre=mask)
    g = T.top_propagate_backward(g, d, d, lams, zs[1], pad, pre=lens)
    gp_ref = torch.empty_like(gp)
    gin_ref = T.top_propagate_backward(g, d, d, lams, zs[0], pad, pre=pupil, saved_in=x0, grad_phase=gp_ref)
    torch.cuda.synchronize()
    assert torch.equal(gin, gin_ref)
    assert torch.equal(gp, gp_ref)


def test_backward_chain_matches_the_oracle(T):
    ny, nx, d = 128, 128, 8e-6
    lams, x0, phi, pupil, lens, mask, zs, stages, xk, gi = backward_chain_case(T, ny, nx, d, 42)
    gp = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    gin = T.top_fused_chain_backward(xk, gi, d, d, lams, stages, 2.0, intensity_group=3, saved_in=x0, grad_phase=gp)
    xh = host(x0).astype(np.complex128)
    pm = O.circ(ny, nx, d, d, 0.3 * ny * d) * np.exp(1j * phi.astype(np.float64))
    lm = np.stack([O.circ(ny, nx, d, d, 0.45 * ny * d) * O.lens(ny, nx, d, d, l, 0.05) for l in lams])
    mm = fields(S.sub_seed(42, 5), 1, ny, nx)[0].astype(np.complex128) * 0.5
    x1 = O.propagate(xh * pm, d, d, lams, zs[0], 2.0)
    x2 = O.propagate(x1 * lm, d, d, lams, zs[1], 2.0)
    x3 = O.propagate(x2 * mm, d, d, lams, zs[2], 2.0)
    g3 = 2.0 * np.repeat(host(gi).astype(np.float64), 3, axis=0) * x3
    h3 = O.propagate_adjoint(g3, d, d, lams, zs[2], 2.0)
    h2 = O.propagate_adjoint(np.conj(mm) * h3, d, d, lams, zs[1], 2.0)
    h1 = O.propagate_adjoint(np.conj(lm) * h2, d, d, lams, zs[0], 2.0)
    gp_ref = np.sum(np.imag(h1 * np.conj(pm * xh)), axis=0)
    assert rel_l2(host(gin), np.conj(pm) * h1) < 1e-5
    assert rel_l2(host(gp).astype(np.float64), gp_ref) < 1e-5


def test_fourf_step_fused_backward_equals_unfused(T):
    """The bench step's backward as one fused chain call against the intensity backward and the
    propagation backward as two calls: the same pupil gradient bit for bit."""
    from paper_2411_18591_gb300.fourf import FourF
    c = S.CFG4
    sysm = FourF(n=c["n"], d=c["d"], f=c["f"], lens_radius=c["lens_radius"], pupil_radius=c["pupil_radius"],
                 objects=1, comps=3, wavelengths=tuple(S.cfg4_wavelengths(2)), pad=c["pad"])
    obj = dev(S.cfg4_objects(1, 3, c["n"]).reshape(-1, c["n"], c["n"]).astype(np.complex64))
    phase = dev(S.cfg4_pupil_phase(c["n"]).astype(np.float32))
    target = dev(S.cfg4_target(1, c["n"]).astype(np.float32))
    g1, g2 = torch.empty_like(phase), torch.empty_like(phase)
    l1, i1 = sysm.step(obj, phase, target, g1)
    l2, i2 = sysm.step_unfused_backward(obj, phase, target, g2)
    torch.cuda.synchronize()
    assert torch.equal(i1, i2) and float(l1) == float(l2)
    assert torch.equal(g1, g2)
