"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Every comparison is element-wise over the whole output, reported as
rel-L2 = ||gpu - oracle|| / ||oracle|| with the tolerance of the propagation
target: 1e-5 up to 1024^2 (complex64 data, FP32 arithmetic, FP64 phases).
Sizes cover every FFT engine (power-of-two and mixed radix), padding factors
below, at and above 2 (folded halves), ragged row tiles, non-square grids with
unequal spacings, per-field wavelengths, chunked batches and the evanescent
cutoff.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from synthetic import gaussian_beam, gaussian_schell, normal, to_c64, uniform

from conftest import rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5


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


def cfield(seed, shape):
    return to_c64(normal(seed, shape) + 1j * normal(seed + 1, shape))


ENGINE_CASES = [
    # ny, nx, pad: padded sizes hit every engine; ragged tiles; folds with pad < 2 and > 2
    (16, 16, 2.0), (16, 32, 2.0), (32, 64, 2.0), (64, 128, 2.0), (128, 256, 2.0), (256, 512, 2.0),
    (24, 48, 1.34), (12, 24, 2.667), (300, 600, 1.7067), (16, 1024, 2.0), (1024, 16, 2.0),
    (16, 2048, 2.0), (2048, 16, 2.0), (16, 4096, 2.0), (4096, 16, 2.0),
    (250, 16, 2.0), (16, 500, 2.0), (768, 16, 2.0), (16, 1000, 2.0), (256, 250, 2.0), (200, 200, 2.5),
    # the 2048- and 4096-point plans with a padding other than 2 (transfer function not staged)
    (2000, 125, 2.048), (125, 2000, 2.048), (4000, 125, 2.048), (8192, 32, 1.0),
]


@pytest.mark.parametrize("ny,nx,pad", ENGINE_CASES)
@pytest.mark.parametrize("method", ["as", "fresnel"])
def test_propagate_matches_oracle(T, ny, nx, pad, method):
    x = cfield(1, (2, ny, nx))
    dy, dx, lam, z = 3e-6, 4e-6, 600e-9, 2e-4
    out = host(T.top_propagate(dev(x), dy, dx, lam, z, pad, method))
    ref = O.propagate(x.astype(np.complex128), dy, dx, lam, z, pad, O.AS if method == "as" else O.FRESNEL_TF)
    assert rel_l2(out, ref) < TOL


def test_config1_gaussian_beam(T):
    """64 x 64 Gaussian (waist 50 um), 10 um, 700 nm, z = 0.1 m, AS, 2x padding, forward."""
    import synthetic
    c = synthetic.cfg1_gaussian()
    out = host(T.top_propagate(dev(c["field"]), c["dy"], c["dx"], c["lam"], c["z"], c["pad"]))
    ref = O.propagate(c["field"].astype(np.complex128), c["dy"], c["dx"], c["lam"], c["z"], c["pad"])
    assert rel_l2(out, ref) < TOL


def test_fresnel_matches_exact_gaussian_beam(T):
    """Through the GPU path: the Fresnel TF reproduces the exact paraxial Gaussian beam."""
    from test_oracle_pins import paraxial_gaussian
    ny, nx, dy, dx, wx, wy, x0, y0, ax, ay = (128, 256, 9e-6, 6e-6, 80e-6, 120e-6, 150e-6, -100e-6, 2e3, -1.5e3)
    f0 = to_c64(gaussian_beam(ny, nx, dy, dx, wx, wy, x0, y0, ax, ay)[None])
    out = host(T.top_propagate(dev(f0), dy, dx, 700e-9, 0.03, 2.0, "fresnel"))[0]
    ref = paraxial_gaussian(ny, nx, dy, dx, 700e-9, 0.03, wx, wy, x0, y0, ax, ay)
    assert rel_l2(out, ref) < TOL


def test_plane_wave_eigenvector_on_gpu(T):
    py, px, dy, dx, lam, z = 32, 64, 2e-6, 1.5e-6, 0.8e-6, 3.7e-4
    a, b = -5, 3
    m = np.arange(px)[None, :]
    l = np.arange(py)[:, None]
    f = to_c64(np.exp(2j * math.pi * (a * m / px + b * l / py))[None])
    k = 2 * math.pi / lam
    kx, ky = 2 * math.pi * a / (px * dx), 2 * math.pi * b / (py * dy)
    h = np.exp(1j * z * math.sqrt(k * k - kx * kx - ky * ky))
    out = host(T.top_propagate(dev(f), dy, dx, lam, z, 1.0))
    assert rel_l2(out, h * f.astype(np.complex128)) < TOL


def test_evanescent_cutoff_on_gpu(T):
    x = cfield(3, (2, 64, 64))
    d, lam, z = 0.2e-6, 0.5e-6, 1e-6
    out = host(T.top_propagate(dev(x), d, d, lam, z, 2.0))
    assert rel_l2(out, O.propagate(x.astype(np.complex128), d, d, lam, z, 2.0)) < TOL


def test_per_field_wavelengths_and_distances_chunked(T):
    """40 fields with 40 (lambda, z) pairs: more than one launch's parameter sets, so chunked."""
    B, n, d = 40, 64, 5e-6
    x = cfield(5, (B, n, n))
    lams = np.linspace(450e-9, 700e-9, B)
    zs = np.linspace(1e-3, 5e-3, B)
    out = host(T.top_propagate(dev(x), d, d, lams, zs, 2.0))
    ref = np.concatenate([O.propagate(x[i:i + 1].astype(np.complex128), d, d, lams[i], zs[i], 2.0) for i in range(B)])
    assert rel_l2(out, ref) < TOL


def test_in_place_and_input_repeat(T):
    n, d = 64, 5e-6
    x = cfield(7, (3, n, n))
    ref = O.propagate(x.astype(np.complex128), d, d, 500e-9, 2e-3, 2.0)
    t = dev(x)
    T.top_propagate(t, d, d, 500e-9, 2e-3, 2.0, out=t)
    assert rel_l2(host(t), ref) < TOL
    lams = [450e-9, 600e-9]
    out = host(T.top_propagate(dev(x), d, d, lams * 3, 2e-3, 2.0, input_repeat=2))
    ref2 = np.stack([O.propagate(x[i // 2].astype(np.complex128), d, d, lams[i % 2], 2e-3, 2.0)[0] for i in range(6)])
    assert rel_l2(out, ref2) < TOL


@pytest.mark.parametrize("ny,nx,pad", [(64, 64, 2.0), (48, 96, 2.667), (250, 250, 2.0)])
def test_shared_source_equals_repeated_inputs(T, ny, nx, pad):
    """With input_repeat the forward transform of each source runs once and the fields start from
    its spectrum; that must equal repeating the inputs bit for bit (plain, with a shared phase and
    aperture, and with a lens, which depends on the wavelength and so is not shared)."""
    d, rep = 5e-6, 3
    x = cfield(8, (2, ny, nx))
    lams = [450e-9, 560e-9, 690e-9] * 2
    xr = dev(np.repeat(x, rep, axis=0))
    phi = uniform(9, (ny, nx), -math.pi, math.pi).astype(np.float32)
    for pre in (None, T.Modulation(phase=dev(phi), radius=0.4 * nx * d), T.Modulation(focal_length=0.05)):
        a = T.top_propagate(dev(x), d, d, lams, 2e-3, pad, pre=pre, input_repeat=rep)
        b = T.top_propagate(xr, d, d, lams, 2e-3, pad, pre=pre)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


# ----------------------------------------------------------------------------- modulation

def _mods(T, ny, nx, per_field=False, B=3):
    shape = (B, ny, nx) if per_field else (ny, nx)
    phi = uniform(11, shape, -math.pi, math.pi).astype(np.float32)
    amp = uniform(12, shape, 0.2, 1.0).astype(np.float32)
    cm = to_c64(np.exp(1j * uniform(13, shape, 0, 6.28)) * 0.8)
    return phi, amp, cm


@pytest.mark.parametrize("per_field", [False, True])
def test_fused_modulations(T, per_field):
    B, ny, nx, d = 3, 64, 32, 5e-6
    x = cfield(15, (B, ny, nx))
    lams = np.array([450e-9, 520e-9, 700e-9])
    z = 3e-3
    phi, amp, cm = _mods(T, ny, nx, per_field, B)
    pre = T.Modulation(phase=dev(phi), amplitude=dev(amp), radius=100e-6)
    post = T.Modulation(mask=dev(cm), focal_length=0.05, radius=110e-6)
    out = host(T.top_propagate(dev(x), d, d, lams, z, 2.0, pre=pre, post=post))
    pm = O.circ(ny, nx, d, d, 100e-6) * amp * np.exp(1j * phi.astype(np.float64))
    ref = np.stack([O.propagate(x[i] * (pm[i] if per_field else pm), d, d, lams[i], z, 2.0)[0] *
                    (cm[i] if per_field else cm) * O.lens(ny, nx, d, d, lams[i], 0.05) * O.circ(ny, nx, d, d, 110e-6)
                    for i in range(B)])
    assert rel_l2(out, ref) < TOL


def test_standalone_modulate_and_backward(T):
    B, ny, nx, d = 5, 40, 56, 5e-6  # standalone modulation has no FFT: any size
    x = cfield(17, (B, ny, nx))
    lams = np.linspace(450e-9, 700e-9, B)
    phi, amp, cm = _mods(T, ny, nx)
    m = T.Modulation(phase=dev(phi), amplitude=dev(amp), mask=dev(cm), focal_length=0.1, radius=90e-6)
    y = host(T.top_modulate(dev(x), m, d, d, lams))
    M = np.stack([cm * amp * np.exp(1j * phi.astype(np.float64)) * O.lens(ny, nx, d, d, l, 0.1) *
                  O.circ(ny, nx, d, d, 90e-6) for l in lams])
    X = x.astype(np.complex128)
    assert rel_l2(y, M * X) < TOL
    g = cfield(19, (B, ny, nx))
    gp = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    ga = torch.zeros_like(gp)
    gm = torch.zeros((ny, nx), dtype=torch.complex64, device="cuda")
    gi = host(T.top_modulate_backward(dev(g), m, d, d, lams, saved_in=dev(x), grad_phase=gp, grad_amplitude=ga,
                                      grad_mask=gm))
    G = g.astype(np.complex128)
    assert rel_l2(gi, np.conj(M) * G) < TOL
    assert rel_l2(host(gp), np.imag(G * np.conj(M * X)).sum(0)) < TOL
    assert rel_l2(host(ga), np.real(np.conj(G) * (M / amp) * X).sum(0)) < TOL
    assert rel_l2(host(gm), (G * np.conj((M / cm) * X)).sum(0)) < TOL


# ----------------------------------------------------------------------------- backward

@pytest.mark.parametrize("method", ["as", "fresnel"])
def test_adjoint_identity_on_gpu(T, method):
    ny, nx, d = 128, 64, 4e-6
    x, y = cfield(21, (2, ny, nx)), cfield(23, (2, ny, nx))
    px = host(T.top_propagate(dev(x), d, d, [450e-9, 650e-9], 5e-3, 2.0, method)).astype(np.complex128)
    phy = host(T.top_propagate_backward(dev(y), d, d, [450e-9, 650e-9], 5e-3, 2.0, method)).astype(np.complex128)
    lhs, rhs = np.vdot(y, px), np.vdot(phy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-6


@pytest.mark.parametrize("per_field", [False, True])
def test_backward_with_modulation_gradients(T, per_field):
    B, ny, nx, d = 3, 64, 32, 5e-6
    x = cfield(25, (B, ny, nx))
    lams = np.array([450e-9, 520e-9, 700e-9])
    z = 3e-3
    phi, amp, cm = _mods(T, ny, nx, per_field, B)
    pre = T.Modulation(phase=dev(phi), amplitude=dev(amp), mask=dev(cm), radius=100e-6)
    post = T.Modulation(focal_length=0.05, radius=110e-6)
    g = cfield(27, (B, ny, nx))
    shape = (B, ny, nx) if per_field else (ny, nx)
    gp = torch.zeros(shape, dtype=torch.float32, device="cuda")
    ga = torch.zeros_like(gp)
    gm = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    gi = host(T.top_propagate_backward(dev(g), d, d, lams, z, 2.0, pre=pre, post=post, saved_in=dev(x),
                                       grad_phase=gp, grad_amplitude=ga, grad_mask=gm))
    postm = np.stack([O.lens(ny, nx, d, d, l, 0.05) * O.circ(ny, nx, d, d, 110e-6) for l in lams])
    gy = np.stack([O.propagate_adjoint(g[i] * np.conj(postm[i]), d, d, lams[i], z, 2.0)[0] for i in range(B)])
    M = O.circ(ny, nx, d, d, 100e-6) * cm * amp * np.exp(1j * phi.astype(np.float64))
    X = x.astype(np.complex128)
    assert rel_l2(gi, np.conj(M) * gy) < TOL
    red = (lambda a: a) if per_field else (lambda a: a.sum(0))
    assert rel_l2(host(gp), red(np.imag(gy * np.conj(M * X)))) < TOL
    assert rel_l2(host(ga), red(np.real(np.conj(gy) * (M / amp) * X))) < TOL
    assert rel_l2(host(gm), red(gy * np.conj((M / cm) * X))) < TOL


def test_intensity_groups_and_backward(T):
    B, group, ny, nx, d = 12, 4, 64, 64, 5e-6
    x = cfield(29, (B, ny, nx))
    lams = np.tile([450e-9, 500e-9, 600e-9, 700e-9], 3)
    z = 4e-3
    w = uniform(30, B, 0.5, 1.5).astype(np.float32)
    post = T.Modulation(focal_length=0.08, radius=120e-6)
    inten, psi = T.top_propagate_intensity(dev(x), d, d, lams, z, 2.0, group=group, weights=dev(w), post=post,
                                           keep_field=True)
    pm = np.stack([O.lens(ny, nx, d, d, l, 0.08) * O.circ(ny, nx, d, d, 120e-6) for l in lams])
    ref_psi = np.stack([O.propagate(x[i], d, d, lams[i], z, 2.0)[0] * pm[i] for i in range(B)])
    assert rel_l2(host(psi), ref_psi) < TOL
    assert rel_l2(host(inten), O.intensity_sum(ref_psi, group, w.astype(np.float64))) < TOL
    gI = uniform(31, (B // group, ny, nx)).astype(np.float32)
    gi = host(T.top_propagate_intensity_backward(psi, dev(gI), d, d, lams, z, 2.0, group=group, weights=dev(w),
                                                 post=post))
    gpsi = 2.0 * np.repeat(gI, group, axis=0) * w[:, None, None] * host(psi).astype(np.complex128)
    ref = np.stack([O.propagate_adjoint(gpsi[i] * np.conj(pm[i]), d, d, lams[i], z, 2.0)[0] for i in range(B)])
    assert rel_l2(gi, ref) < TOL


def test_mse_loss(T):
    I = uniform(33, (4, 100, 90)).astype(np.float32)
    Tg = uniform(34, (4, 100, 90)).astype(np.float32)
    loss, grad = T.top_mse_loss(dev(I), dev(Tg))
    lr, gr = O.mse_loss(I, Tg)
    # residuals are formed in float32 (2^-24 relative each), the sum in float64
    assert abs(float(loss) - lr) / lr < 1e-6
    assert rel_l2(host(grad), gr) < 1e-6


def test_gradient_vs_finite_differences(T):
    """GPU analytic gradient of a 2-mask diffractive chain vs FP64 central differences of the oracle loss."""
    n, d, lam = 32, 8e-6, 532e-9
    x = to_c64(uniform(40, (2, n, n)) < 0.5)
    target = uniform(41, (2, n, n)).astype(np.float32)
    p1 = uniform(42, (n, n), 0, 2 * math.pi).astype(np.float32)
    p2 = uniform(43, (n, n), 0, 2 * math.pi).astype(np.float32)
    z1, z2 = 0.01, 0.015

    def loss64(a, b):
        y = O.propagate(x.astype(np.complex128) * np.exp(1j * a), d, d, lam, z1, 2.0)
        out = O.propagate(y * np.exp(1j * b), d, d, lam, z2, 2.0)
        return O.mse_loss(O.intensity(out), target)[0]

    xd = dev(x)
    y = T.top_propagate(xd, d, d, lam, z1, 2.0, pre=T.Modulation(phase=dev(p1)))
    inten, psi = T.top_propagate_intensity(y, d, d, lam, z2, 2.0, pre=T.Modulation(phase=dev(p2)), keep_field=True)
    _, gI = T.top_mse_loss(inten, dev(target))
    g2 = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    gy = T.top_propagate_intensity_backward(psi, gI, d, d, lam, z2, 2.0, pre=T.Modulation(phase=dev(p2)),
                                            saved_in=y, grad_phase=g2)
    g1 = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    T.top_propagate_backward(gy, d, d, lam, z1, 2.0, pre=T.Modulation(phase=dev(p1)), saved_in=xd,
                             want_grad_in=False, grad_phase=g1)
    idx = np.array(sorted(set(int(v) for v in uniform(44, 40) * n * n)))[:32]
    fd1 = O.finite_difference(lambda a: loss64(a, p2.astype(np.float64)), p1.astype(np.float64), idx)
    fd2 = O.finite_difference(lambda b: loss64(p1.astype(np.float64), b), p2.astype(np.float64), idx)
    for fd, g in ((fd1, host(g1).reshape(-1)[idx]), (fd2, host(g2).reshape(-1)[idx])):
        assert np.max(np.abs(fd - g)) <= 1e-3 * np.max(np.abs(fd))


# ----------------------------------------------------------------------------- coherence

def test_coherence_forward_backward(T):
    n, d, lam, z = 16, 10e-6, 633e-9, 0.004
    g0 = to_c64(gaussian_schell(n, d, 60e-6, 25e-6))
    phi = uniform(50, (n, n), -math.pi, math.pi).astype(np.float32)
    mask = T.Modulation(phase=dev(phi), radius=70e-6)
    gz = T.top_propagate_coherence(dev(g0), d, d, lam, z, 2.0, mask=mask)
    M = O.circ(n, n, d, d, 70e-6) * np.exp(1j * phi.astype(np.float64))
    ref = O.propagate_coherence(O.modulate_coherence(g0.astype(np.complex128), M), d, d, lam, z, 2.0)
    assert rel_l2(host(gz), ref) < TOL
    inten = T.top_coherence_intensity(gz)
    assert rel_l2(host(inten), O.coherence_diag(ref)) < TOL
    tgt = uniform(51, (n, n)).astype(np.float32)
    _, gI = O.mse_loss(O.coherence_diag(ref), tgt)
    G = T.top_coherence_intensity_backward(dev(gI.astype(np.float32)), gz)
    gp = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    gin = T.top_propagate_coherence_backward(G, d, d, lam, z, 2.0, mask=mask, saved_in=dev(g0), grad_phase=gp)
    gd = np.diag(gI.reshape(-1).astype(np.complex128)).reshape(n, n, n, n)
    gm_gamma = O.propagate_coherence(gd, d, d, lam, z, 2.0, adjoint=True)
    gM = O.grad_modulate_coherence(g0.astype(np.complex128), M, gm_gamma)
    assert rel_l2(host(gp), np.imag(np.conj(M) * gM)) < TOL
    D = M[:, :, None, None] * np.conj(M)[None, None, :, :]
    assert rel_l2(host(gin), np.conj(D) * gm_gamma) < TOL


# ----------------------------------------------------------------------------- errors

def test_errors_are_reported_not_launched(T):
    from paper_2411_18591_gb300._lib import TopError
    x = dev(cfield(60, (1, 61, 61)))
    with pytest.raises(TopError, match="UNSUPPORTED"):
        T.top_propagate_noalloc(x, 1e-6, 1e-6, 5e-7, 1e-3, 1.0, out=x)  # no-alloc call at an unplanned (odd) size
    with pytest.raises(TopError, match="INVALID_ARG"):
        T.top_propagate(dev(cfield(61, (1, 64, 64))), 1e-6, 1e-6, -5e-7, 1e-3, 2.0)   # negative wavelength
    big = dev(cfield(62, (1, 64, 65)))
    with pytest.raises(ValueError, match="contiguous"):
        T.top_propagate(big[:, :, 1:], 1e-6, 1e-6, 5e-7, 1e-3, 2.0)
    # misaligned pointer: a view one element into a buffer
    buf = torch.zeros(1 * 64 * 64 + 1, dtype=torch.complex64, device="cuda")
    mis = buf[1:].view(1, 64, 64)
    from paper_2411_18591_gb300 import _lib
    import ctypes as C
    g = _lib.TopGrid(1, 64, 64, 1e-6, 1e-6, 2.0, 0, 0)
    lam = _lib.doubles([5e-7])
    from paper_2411_18591_gb300.binding import handle
    st = _lib.load().top_propagate(handle(), C.byref(g), mis.data_ptr(), mis.data_ptr(), lam, lam, 1, None, None,
                                   None)
    assert st == 1 and b"aligned" in _lib.load().top_last_error()
    torch.cuda.synchronize()
