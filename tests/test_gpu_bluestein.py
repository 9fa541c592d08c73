"""Padded sizes without an FFT plan of their own (odd, prime, or with prime factors above 5):
Bluestein line transforms on the power-of-two engines, against the FP64 oracle.

Every comparison is element-wise rel-L2 over the whole output with the propagation
tolerance (1e-5): prime sizes (61, 127, 257), products with 7, 11, 13, a padded size
of 2042 (4096-point transforms), sizes below the smallest plan (16), one axis planned
and the other not, per-field wavelengths and distances, the Fresnel form, repeated
inputs, modulations before and after, the adjoint (backward) and its identity, modulation
gradients and the autograd wrapper, grouped intensities and their backward, fused chains and
ragged batches mixing planned and unplanned sizes, overlaps and powers, Direct Integration.
"""
import numpy as np
import pytest
import torch

import oracle as O
from synthetic import normal, to_c64, uniform

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


CASES = [
    # ny, nx, pad -> padded sizes (Py, Px)
    (61, 61, 1.0),     # 61 x 61, prime
    (127, 64, 1.0),    # 127 (prime) x 64 (planned axis)
    (257, 31, 1.0),    # 257 x 31, primes; 257 needs 1024-point transforms
    (100, 90, 2.31),   # 231 = 3 7 11, 208 = 16 13
    (8, 16, 2.0),      # 16 x 32: 16 is below the smallest plan
    (45, 37, 2.0),     # 90, 74 = 2 37
    (1021, 24, 2.0),   # 2042 = 2 1021: two 2048-point halves per transform; 48 planned
    (3001, 16, 1.0),   # 3001 (prime): two 4096-point halves per transform
]


@pytest.mark.parametrize("ny,nx,pad", CASES)
@pytest.mark.parametrize("method", ["as", "fresnel"])
def test_bluestein_propagate_matches_oracle(T, ny, nx, pad, method):
    x = cfield(31, (2, ny, nx))
    dy, dx, lam, z = 3e-6, 4e-6, 600e-9, 2e-4
    out = host(T.top_propagate(dev(x), dy, dx, lam, z, pad, method))
    ref = O.propagate(x.astype(np.complex128), dy, dx, lam, z, pad, O.AS if method == "as" else O.FRESNEL_TF)
    assert rel_l2(out, ref) < TOL


@pytest.mark.parametrize("ny,nx,pad", [(61, 61, 1.0), (100, 90, 2.31), (1021, 24, 2.0)])
def test_bluestein_backward_is_the_adjoint_propagation(T, ny, nx, pad):
    g = cfield(33, (2, ny, nx))
    dy, dx, lam, z = 3e-6, 3e-6, 520e-9, 1e-3
    out = host(T.top_propagate_backward(dev(g), dy, dx, lam, z, pad))
    ref = O.propagate_adjoint(g.astype(np.complex128), dy, dx, lam, z, pad)
    assert rel_l2(out, ref) < TOL
    x = cfield(35, (2, ny, nx))
    px = host(T.top_propagate(dev(x), dy, dx, lam, z, pad)).astype(np.complex128)
    lhs, rhs = np.vdot(g, px), np.vdot(out.astype(np.complex128), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-6


def test_bluestein_per_field_parameters_repeat_and_modulations(T):
    """Six fields from three inputs (input_repeat 2), each with its own wavelength and distance,
    a phase mask and aperture before and a lens after the propagation."""
    ny, nx, pad, d = 70, 50, 1.94, 5e-6  # 136 = 8 17, 97 (prime)
    x = cfield(37, (3, ny, nx))
    lams = np.linspace(450e-9, 700e-9, 6)
    zs = np.linspace(1e-3, 4e-3, 6)
    phi = uniform(39, (ny, nx), -np.pi, np.pi).astype(np.float32)
    pre = T.Modulation(phase=dev(phi), radius=110e-6)
    post = T.Modulation(focal_length=0.05)
    out = host(T.top_propagate(dev(x), d, d, lams, zs, pad, pre=pre, post=post, input_repeat=2))
    pm = O.circ(ny, nx, d, d, 110e-6) * np.exp(1j * phi.astype(np.float64))
    ref = np.stack([O.propagate(x[i // 2].astype(np.complex128) * pm, d, d, lams[i], zs[i], pad)[0] *
                    O.lens(ny, nx, d, d, lams[i], 0.05) for i in range(6)])
    assert rel_l2(out, ref) < TOL
    # the backward applies the conjugate modulations in the reverse order
    g = cfield(41, (6, ny, nx))
    gi = host(T.top_propagate_backward(dev(g), d, d, lams, zs, pad, pre=pre, post=post))
    refb = np.stack([np.conj(pm) * O.propagate_adjoint(g[i].astype(np.complex128) *
                                                       np.conj(O.lens(ny, nx, d, d, lams[i], 0.05)),
                                                       d, d, lams[i], zs[i], pad)[0] for i in range(6)])
    assert rel_l2(gi, refb) < TOL


def test_bluestein_backward_with_modulation_gradients(T):
    """The phase, amplitude and complex-mask gradients of the modulation before the propagation,
    shared by the batch, at a prime padded size (adjoint propagation, then the modulation's
    backward)."""
    B, ny, nx, pad, d = 3, 61, 45, 1.0, 5e-6  # 61 x 45 = 3^2 5
    x = cfield(51, (B, ny, nx))
    lams = np.array([450e-9, 520e-9, 700e-9])
    z = 3e-3
    phi = uniform(53, (ny, nx), -np.pi, np.pi).astype(np.float32)
    amp = uniform(54, (ny, nx), 0.2, 1.0).astype(np.float32)
    cm = to_c64(np.exp(1j * uniform(55, (ny, nx), 0, 6.28)) * 0.8)
    pre = T.Modulation(phase=dev(phi), amplitude=dev(amp), mask=dev(cm), radius=100e-6)
    post = T.Modulation(focal_length=0.05)
    g = cfield(57, (B, ny, nx))
    gp = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    ga = torch.zeros_like(gp)
    gm = torch.zeros((ny, nx), dtype=torch.complex64, device="cuda")
    gi = host(T.top_propagate_backward(dev(g), d, d, lams, z, pad, pre=pre, post=post, saved_in=dev(x),
                                       grad_phase=gp, grad_amplitude=ga, grad_mask=gm))
    gy = np.stack([O.propagate_adjoint(g[i] * np.conj(O.lens(ny, nx, d, d, lams[i], 0.05)), d, d, lams[i], z,
                                       pad)[0] for i in range(B)])
    M = O.circ(ny, nx, d, d, 100e-6) * cm * amp * np.exp(1j * phi.astype(np.float64))
    X = x.astype(np.complex128)
    assert rel_l2(gi, np.conj(M) * gy) < TOL
    assert rel_l2(host(gp), np.imag(gy * np.conj(M * X)).sum(0)) < TOL
    assert rel_l2(host(ga), np.real(np.conj(gy) * (M / amp) * X).sum(0)) < TOL
    assert rel_l2(host(gm), (gy * np.conj((M / cm) * X)).sum(0)) < TOL


def test_bluestein_autograd_phase_mask(T):
    """autograd.propagate with a trainable phase mask at a Bluestein size: the mask gradient of
    L = sum w |y|^2 (a fixed detector weight w; at padding 1 the unweighted sum would not depend
    on the mask) against the oracle (g = 2 w y)."""
    ny, nx, pad, d, lam, z = 37, 37, 1.0, 4e-6, 600e-9, 2e-3
    x = cfield(59, (2, ny, nx))
    phi = uniform(61, (ny, nx), -np.pi, np.pi).astype(np.float32)
    w = uniform(63, (ny, nx), 0.0, 1.0)
    from paper_2411_18591_gb300 import autograd as A
    xt = dev(x)
    pt = dev(phi).requires_grad_(True)
    y = A.propagate(xt, d, d, lam, z, pad, phase=pt)
    (dev(w.astype(np.float32)) * y.abs() ** 2).sum().backward()
    M = np.exp(1j * phi.astype(np.float64))
    X = x.astype(np.complex128)
    yo = O.propagate(X * M, d, d, lam, z, pad)
    gy = O.propagate_adjoint(2 * w * yo, d, d, lam, z, pad)
    assert rel_l2(host(y.detach()), yo) < TOL
    assert rel_l2(host(pt.grad), np.imag(gy * np.conj(M * X)).sum(0)) < TOL


def test_bluestein_intensity_forward_and_backward(T):
    """Grouped, weighted detector intensity (Eq. 14) and its backward with phase gradients at a
    prime padded size: the intensity sums and the backward source as separate passes."""
    B, group, ny, nx, pad, d = 4, 2, 53, 40, 1.0, 5e-6  # 53 (prime) x 40 = 8 5
    x = cfield(71, (B, ny, nx))
    lams = np.array([450e-9, 520e-9, 600e-9, 700e-9])
    z = 2e-3
    w = uniform(73, (B,), 0.5, 1.5).astype(np.float32)
    phi = uniform(75, (ny, nx), -np.pi, np.pi).astype(np.float32)
    pre = T.Modulation(phase=dev(phi))
    inten, psi = T.top_propagate_intensity(dev(x), d, d, lams, z, pad, group=group, weights=dev(w), pre=pre,
                                           keep_field=True)
    M = np.exp(1j * phi.astype(np.float64))
    X = x.astype(np.complex128)
    po = np.stack([O.propagate(X[i] * M, d, d, lams[i], z, pad)[0] for i in range(B)])
    iref = O.intensity_sum(po, group, w.astype(np.float64))
    assert rel_l2(host(psi), po) < TOL
    assert rel_l2(host(inten), iref) < TOL
    gI = uniform(77, (B // group, ny, nx), -1.0, 1.0).astype(np.float32)
    gp = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    gi = host(T.top_propagate_intensity_backward(psi, dev(gI), d, d, lams, z, pad, group=group, weights=dev(w),
                                                 pre=pre, saved_in=dev(x), grad_phase=gp))
    src = 2 * w[:, None, None].astype(np.float64) * np.repeat(gI.astype(np.float64), group, axis=0) * po
    gy = np.stack([O.propagate_adjoint(src[i], d, d, lams[i], z, pad)[0] for i in range(B)])
    assert rel_l2(gi, np.conj(M) * gy) < TOL
    assert rel_l2(host(gp), np.imag(gy * np.conj(M * X)).sum(0)) < TOL


def test_bluestein_fused_chain_equals_the_same_calls(T):
    """A three-stage chain with a kept field and the grouped intensity at a padded size without a
    plan equals the same sequence of calls, bit for bit."""
    ny, nx, pad, d = 45, 45, 1.0, 6e-6  # 45 = 3^2 5
    lams = [450e-9, 600e-9, 700e-9, 520e-9]
    x = dev(cfield(79, (4, ny, nx)))
    phi = uniform(81, (ny, nx), -np.pi, np.pi).astype(np.float32)
    pupil = T.Modulation(phase=dev(phi), radius=0.3 * ny * d)
    lens = T.Modulation(focal_length=0.05)
    keep = torch.empty_like(x)
    zs = [1e-3, 2e-3, 1.5e-3]
    out, inten = T.top_fused_chain(x, d, d, lams, [T.Stage(zs[0], keep=keep), T.Stage(zs[1], pre=lens),
                                                   T.Stage(zs[2], pre=pupil)], pad, intensity_group=2)
    y = T.top_propagate(x, d, d, lams, zs[0], pad)
    k = y.clone()
    y = T.top_propagate(y, d, d, lams, zs[1], pad, pre=lens)
    i_ref, y_ref = T.top_propagate_intensity(y, d, d, lams, zs[2], pad, group=2, pre=pupil, keep_field=True)
    torch.cuda.synchronize()
    assert torch.equal(keep, k)
    assert torch.equal(out, y_ref)
    assert torch.equal(inten, i_ref)
    ref = O.propagate(host(x).astype(np.complex128), d, d, lams, zs[0], pad)
    assert rel_l2(host(keep), ref) < TOL


def test_bluestein_chain_with_repeated_inputs(T):
    """Two inputs each feeding three wavelengths (input_repeat 3) through a two-stage chain at a
    padded size without a plan: equal to the same calls on the repeated inputs."""
    ny, nx, pad, d = 37, 41, 1.0, 5e-6
    lams = [450e-9, 550e-9, 650e-9] * 2
    x = dev(cfield(97, (2, ny, nx)))
    lens = T.Modulation(focal_length=0.04, radius=0.4 * ny * d)
    out, inten = T.top_fused_chain(x, d, d, lams, [T.Stage(1e-3), T.Stage(2e-3, pre=lens)], pad,
                                   intensity_group=3, input_repeat=3)
    xr = x.repeat_interleave(3, dim=0)
    y = T.top_propagate(xr, d, d, lams, 1e-3, pad)
    i_ref, y_ref = T.top_propagate_intensity(y, d, d, lams, 2e-3, pad, group=3, pre=lens, keep_field=True)
    torch.cuda.synchronize()
    assert torch.equal(out, y_ref)
    assert torch.equal(inten, i_ref)


def test_bluestein_ragged_batch_with_planned_and_unplanned_sizes(T):
    descs = [(61, 61, 1.0), (64, 64, 2.0), (45, 37, 2.0), (48, 96, 2.667)]
    xs = [dev(cfield(83 + i, (ny, nx))) for i, (ny, nx, _) in enumerate(descs)]
    lams = [450e-9, 500e-9, 550e-9, 600e-9]
    zs = [1e-3, 2e-3, 3e-3, 4e-3]
    for pad in sorted({p for *_, p in descs}):
        idx = [i for i, desc in enumerate(descs) if desc[2] == pad]
        ys = T.top_propagate_ragged([xs[i] for i in idx], [4e-6] * len(idx), [lams[i] for i in idx],
                                    [zs[i] for i in idx], pad)
        gs = T.top_propagate_ragged(ys, [4e-6] * len(idx), [lams[i] for i in idx], [zs[i] for i in idx], pad,
                                    backward=True)
        for j, i in enumerate(idx):
            xh = host(xs[i]).astype(np.complex128)
            ref = O.propagate(xh, 4e-6, 4e-6, lams[i], zs[i], pad)[0]
            assert rel_l2(host(ys[j]), ref) < TOL
            back = O.propagate_adjoint(host(ys[j]).astype(np.complex128), 4e-6, 4e-6, lams[i], zs[i], pad)[0]
            assert rel_l2(host(gs[j]), back) < TOL


@pytest.mark.parametrize("per_field", [False, True])
def test_bluestein_overlap_and_power(T, per_field):
    """The overlaps and powers of Eq. 7 at a prime padded size, with a lens after the propagation,
    against a shared or a per-field target."""
    B, ny, nx, pad, d = 3, 61, 50, 1.0, 5e-6
    x = cfield(91, (B, ny, nx))
    tgt = cfield(93, (B, ny, nx) if per_field else (ny, nx))
    lams = np.array([450e-9, 550e-9, 650e-9])
    z = 2e-3
    post = T.Modulation(focal_length=0.05)
    ov, pw, psi = T.top_propagate_overlap(dev(x), dev(tgt), d, d, lams, z, pad, post=post, keep_field=True)
    po = np.stack([O.propagate(x[i].astype(np.complex128), d, d, lams[i], z, pad)[0] *
                   O.lens(ny, nx, d, d, lams[i], 0.05) for i in range(B)])
    assert rel_l2(host(psi), po) < TOL
    o_ref = O.overlap(po, tgt.astype(np.complex128), d, d)
    assert rel_l2(ov.cpu().numpy(), o_ref) < TOL
    assert rel_l2(pw.cpu().numpy(), O.power(po, d, d)) < TOL


@pytest.mark.parametrize("n", [45, 61])
def test_bluestein_direct_integration(T, n):
    """DI (Eq. 2-3) at padded sizes without a plan of their own (90 = 2 3^2 5, 122 = 2 61): the
    kernel's samples transformed by Bluestein rows and columns; and TOP_AUTO beyond z_critical."""
    d, lam = 4e-6, 633e-9
    x = cfield(95, (2, n, n))
    z = 0.05  # beyond z_critical = n d^2 / lambda (1.1 mm and 1.5 mm)
    for method in ("di", "auto"):
        out = host(T.top_propagate(dev(x), d, d, lam, z, 2.0, method))
        ref = O.propagate(x.astype(np.complex128), d, d, lam, z, 2.0, O.DI)
        assert rel_l2(out, ref) < TOL
    back = host(T.top_propagate_backward(dev(x), d, d, lam, z, 2.0, "di"))
    assert rel_l2(back, O.propagate_adjoint(x.astype(np.complex128), d, d, lam, z, 2.0, O.DI)) < TOL


def test_bluestein_limits_are_reported(T):
    x = dev(cfield(43, (1, 61, 61)))
    with pytest.raises(T.TopError, match="2 n - 1"):
        T.top_propagate(x, 2e-6, 2e-6, 600e-9, 1e-2, 1.0, "di")  # DI needs a padded size >= 2 n - 1
    with pytest.raises(T.TopError, match="UNSUPPORTED"):
        T.top_propagate_noalloc(x, 2e-6, 2e-6, 600e-9, 1e-3, 1.0, out=x)  # the no-alloc call needs a plan
    with pytest.raises(T.TopError, match="4096"):
        T.top_propagate(dev(cfield(45, (1, 16, 2500))), 2e-6, 2e-6, 600e-9, 1e-3, 2.0)  # 5000 = 8 5^4
