"""Pins of the FP64 oracle to closed forms, invariants and independent brute force.

None of these re-types the oracle's own formula as its only check: each compares
the oracle with something the paper or the mathematics fixes (the paraxial
Gaussian beam, the Airy pattern, the Rayleigh-Sommerfeld sum of Eq. 2-3, the
Mandel-Wolf spreading of a Gaussian Schell-model source, Parseval, group and
adjoint identities, finite differences). ``test_planted_mistakes`` checks that a
plausible slip in the oracle makes at least one of these pins fail.
"""
import math

import numpy as np
import pytest
from scipy.special import j1

import oracle as O
from synthetic import gaussian_beam, gaussian_schell, normal, uniform, to_c64

from conftest import rel_l2


def paraxial_gaussian(ny, nx, dy, dx, lam, z, wx, wy, x0=0.0, y0=0.0, ax=0.0, ay=0.0):
    """Exact solution of the paraxial wave equation for a (tilted, offset) Gaussian.

    Per axis: q = z - i zR, u = sqrt(q0/q) exp(i k s^2 / (2 q)) with s the offset
    coordinate moved by lambda z a, times the tilt phase exp(2 pi i a x - i pi lambda z a^2);
    overall exp(i k z). zR = pi w^2 / lambda (Gouy phase and waist follow from q).
    """
    k = 2.0 * math.pi / lam
    x = O.coords(nx, dx)[None, :]
    y = O.coords(ny, dy)[:, None]

    def axis(c, w, a, c0):
        q0 = -1j * math.pi * w * w / lam
        q = q0 + z
        s = c - c0 - lam * z * a
        return np.sqrt(q0 / q) * np.exp(1j * k * s * s / (2.0 * q)) * \
            np.exp(2j * math.pi * a * c - 1j * math.pi * lam * z * a * a)

    return np.exp(1j * k * z) * axis(x, wx, ax, x0) * axis(y, wy, ay, y0)


GAUSS_CASES = [
    # ny, nx, dy, dx, wx, wy, x0, y0, ax, ay
    (256, 256, 10e-6, 10e-6, 100e-6, 100e-6, 0.0, 0.0, 0.0, 0.0),
    (96, 128, 12e-6, 9e-6, 80e-6, 120e-6, 150e-6, -100e-6, 2e3, -1.5e3),
]


# ----------------------------------------------------------------------------- DFT

@pytest.mark.parametrize("p", [1, 2, 3, 5, 7, 8, 12, 61, 64])
def test_dft_naive_matches_library(p):
    x = normal(11 + p, (3, p)) + 1j * normal(12 + p, (3, p))
    x2 = x[:, :, None] * np.ones((1, 1, 3))
    a = O.dft2(np.moveaxis(x2, 1, -2), naive=True)
    b = O.dft2(np.moveaxis(x2, 1, -2), naive=False)
    assert rel_l2(a, b) < 1e-13
    assert rel_l2(O.idft2(a, naive=True), np.moveaxis(x2, 1, -2)) < 1e-13


def _naive_line_dft(x, sign):
    """X[k] = sum_n x[n] exp(sign 2 pi i (k n mod P) / P) for one line, in blocks of k."""
    p = x.shape[0]
    n = np.arange(p, dtype=np.int64)
    out = np.empty(p, dtype=np.complex128)
    for k0 in range(0, p, 256):
        k = np.arange(k0, min(p, k0 + 256), dtype=np.int64)
        kn = np.outer(k, n) % p
        out[k0:k0 + k.size] = np.exp(sign * 2j * math.pi * kn.astype(np.float64) / p) @ x
    return out


@pytest.mark.parametrize("p", [2039, 2048, 4096, 8192])
def test_library_fft_matches_definition_at_kernel_lengths(p):
    """The oracle's library FFT on single lines of the padded lengths the kernels transform (2048,
    4096 and 8192 points, and the prime 2039 that the Bluestein path covers), along either axis,
    against the DFT written out from its definition."""
    x = normal(31 + p, (p,)) + 1j * normal(32 + p, (p,))
    ref = _naive_line_dft(x, -1)
    assert rel_l2(O.dft2(x[:, None])[:, 0], ref) < 1e-12
    assert rel_l2(O.dft2(x[None, :])[0], ref) < 1e-12
    inv = _naive_line_dft(x, +1) / p
    assert rel_l2(O.idft2(x[:, None])[:, 0], inv) < 1e-12
    assert rel_l2(O.idft2(x[None, :])[0], inv) < 1e-12


def test_dft_of_delta_and_exponential():
    p = 12
    for n0 in range(p):
        x = np.zeros((p, 1))
        x[n0, 0] = 1.0
        X = O.dft2(x, naive=True)[:, 0]
        k = np.arange(p)
        assert np.allclose(X, np.exp(-2j * math.pi * k * n0 / p), atol=1e-14)
    a = 5
    x = np.exp(2j * math.pi * a * np.arange(p) / p)[:, None]
    X = O.dft2(x)[:, 0]
    expect = np.zeros(p)
    expect[a] = p
    assert np.allclose(X, expect, atol=1e-12)


def test_padded_size_and_offset():
    assert O.padded_size(250, 2.0) == 500
    assert O.padded_size(5, 1.5) == 8           # floor(7.5 + 0.5)
    assert O.padded_size(61, 1.0) == 61
    assert O.pad_offset(64, 128) == 32
    assert O.pad_offset(5, 8) == 1
    with pytest.raises(ValueError):
        O.padded_size(10, 0.5)
    assert list(O.signed_index(5)) == [0, 1, 2, -2, -1]
    assert list(O.signed_index(4)) == [0, 1, -2, -1]


def test_zcritical():
    # Eq. 6 for a 256-sample, 10 um grid at 700 nm: L = 2.56 mm
    assert O.z_critical(256 * 10e-6, 10e-6, 700e-9) == pytest.approx(0.0365714285714, rel=1e-12)


# ----------------------------------------------------------------------------- operator identities

@pytest.mark.parametrize("method", [O.AS, O.FRESNEL_TF])
@pytest.mark.parametrize("pad", [1.0, 2.0, 1.5])
def test_identity_at_z0(method, pad):
    f = normal(1, (2, 12, 10)) + 1j * normal(2, (2, 12, 10))
    out = O.propagate(f, 3e-6, 4e-6, 600e-9, 0.0, pad, method)
    assert rel_l2(out, f) < 1e-14


@pytest.mark.parametrize("a,b", [(0, 0), (3, 1), (-4, 2), (5, -3), (-8, -5)])
def test_plane_wave_is_eigenvector(a, b):
    """With pad 1 a sampled plane wave exp(2 pi i (a m/Px + b l/Py)) is an eigenvector.

    The eigenvalue is Eq. 5 at kx = 2 pi a/(Px dx), ky = 2 pi b/(Py dy) with k = 2 pi/lambda.
    """
    py, px, dy, dx, lam, z = 12, 16, 2e-6, 1.5e-6, 0.8e-6, 3.7e-4
    m = np.arange(px)[None, :]
    l = np.arange(py)[:, None]
    f = np.exp(2j * math.pi * (a * m / px + b * l / py))
    k = 2 * math.pi / lam
    kx = 2 * math.pi * a / (px * dx)
    ky = 2 * math.pi * b / (py * dy)
    h = np.exp(1j * z * math.sqrt(k * k - kx * kx - ky * ky))
    out = O.propagate(f, dy, dx, lam, z, 1.0)[0]
    assert rel_l2(out, h * f) < 1e-12


@pytest.mark.parametrize("a,b", [(0, 0), (4, -6), (-8, 5), (8, 6)])
def test_plane_wave_is_eigenvector_at_prime_sizes(a, b):
    """The same eigenvalue at prime padded sizes (13 x 17), where the frequency index a of an odd
    size runs over -(P - 1)/2 .. (P - 1)/2: the padded sizes that take Bluestein transforms."""
    py, px, dy, dx, lam, z = 13, 17, 2e-6, 1.5e-6, 0.8e-6, 3.7e-4
    m = np.arange(px)[None, :]
    l = np.arange(py)[:, None]
    f = np.exp(2j * math.pi * (a * m / px + b * l / py))
    k = 2 * math.pi / lam
    kx = 2 * math.pi * a / (px * dx)
    ky = 2 * math.pi * b / (py * dy)
    h = np.exp(1j * z * math.sqrt(k * k - kx * kx - ky * ky))
    out = O.propagate(f, dy, dx, lam, z, 1.0)[0]
    assert rel_l2(out, h * f) < 1e-12


def test_parseval_pad1():
    f = normal(3, (3, 20, 24)) + 1j * normal(4, (3, 20, 24))
    out = O.propagate(f, 5e-6, 5e-6, 633e-9, 0.07, 1.0)
    assert np.allclose(np.linalg.norm(out, axis=(1, 2)), np.linalg.norm(f, axis=(1, 2)), rtol=1e-13)


@pytest.mark.parametrize("method", [O.AS, O.FRESNEL_TF])
def test_additivity_and_time_reversal(method):
    f = normal(5, (2, 16, 16)) + 1j * normal(6, (2, 16, 16))
    args = (4e-6, 4e-6, 500e-9)
    p12 = O.propagate(O.propagate(f, *args, 0.013, 1.0, method), *args, 0.021, 1.0, method)
    p = O.propagate(f, *args, 0.034, 1.0, method)
    # phases reach 2 pi z / lambda ~ 4e5 rad, so FP64 rounding of H is ~1e-11
    assert rel_l2(p12, p) < 1e-10
    back = O.propagate(O.propagate(f, *args, 0.05, 1.0, method), *args, -0.05, 1.0, method)
    assert rel_l2(back, f) < 1e-10


def test_offset_invariance():
    """The result does not depend on where the field sits in the padded grid."""
    f = normal(7, (1, 10, 14)) + 1j * normal(8, (1, 10, 14))
    ref = O.propagate(f, 3e-6, 3e-6, 500e-9, 2e-3, 2.0)
    for off in [(0, 0), (10, 14), (3, 9)]:
        out = O.propagate(f, 3e-6, 3e-6, 500e-9, 2e-3, 2.0, offset=off)
        assert rel_l2(out, ref) < 1e-13


@pytest.mark.parametrize("method", [O.AS, O.FRESNEL_TF])
def test_adjoint_identity(method):
    """<P x, y> = <x, P^H y> with the adjoint built from conj(H) (backward pass, §4)."""
    x = normal(9, (3, 18, 14)) + 1j * normal(10, (3, 18, 14))
    y = normal(11, (3, 18, 14)) + 1j * normal(12, (3, 18, 14))
    lams = [450e-9, 520e-9, 700e-9]
    px = O.propagate(x, 6e-6, 5e-6, lams, 0.02, 2.0, method)
    phy = O.propagate_adjoint(y, 6e-6, 5e-6, lams, 0.02, 2.0, method)
    lhs = np.vdot(y, px)
    rhs = np.vdot(phy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_evanescent_cutoff():
    """Sub-wavelength sampling: H vanishes where 1/lambda^2 < fx^2 + fy^2, |H| = 1 elsewhere."""
    p, d, lam = 32, 0.2e-6, 0.5e-6
    h = O.transfer_function(p, p, d, d, lam, 1e-6)
    fx = O.freqs(p, d)
    r2 = fx[None, :] ** 2 + fx[:, None] ** 2
    ev = r2 > 1.0 / lam ** 2
    assert ev.sum() > 0 and (~ev).sum() > 0
    assert np.all(h[ev] == 0)
    assert np.allclose(np.abs(h[~ev]), 1.0, atol=1e-14)
    # energy is lost exactly by the evanescent part of the spectrum (pad 1, Parseval)
    f = normal(13, (1, p, p)) + 1j * normal(14, (1, p, p))
    out = O.propagate(f, d, d, lam, 1e-6, 1.0)
    spec = np.fft.fft2(f[0])
    assert np.linalg.norm(out) ** 2 == pytest.approx(np.sum(np.abs(spec[~ev]) ** 2) / p ** 2, rel=1e-12)


# ----------------------------------------------------------------------------- physics closed forms

@pytest.mark.parametrize("case", GAUSS_CASES)
def test_fresnel_tf_equals_paraxial_gaussian(case):
    """The Fresnel transfer function propagates a Gaussian beam exactly (waist, Gouy phase)."""
    ny, nx, dy, dx, wx, wy, x0, y0, ax, ay = case
    lam, z = 700e-9, 0.03
    f0 = gaussian_beam(ny, nx, dy, dx, wx, wy, x0, y0, ax, ay)
    out = O.propagate(f0, dy, dx, lam, z, 2.0, O.FRESNEL_TF)[0]
    ref = paraxial_gaussian(ny, nx, dy, dx, lam, z, wx, wy, x0, y0, ax, ay)
    assert rel_l2(out, ref) < 1e-7


@pytest.mark.parametrize("case", GAUSS_CASES)
def test_as_matches_paraxial_gaussian(case):
    """AS agrees with the paraxial beam up to non-paraxial terms ~ 1/(k w0)^2 (here < 1e-5)."""
    ny, nx, dy, dx, wx, wy, x0, y0, ax, ay = case
    lam, z = 700e-9, 0.03
    f0 = gaussian_beam(ny, nx, dy, dx, wx, wy, x0, y0, ax, ay)
    out = O.propagate(f0, dy, dx, lam, z, 2.0, O.AS)[0]
    ref = paraxial_gaussian(ny, nx, dy, dx, lam, z, wx, wy, x0, y0, ax, ay)
    assert rel_l2(out, ref) < 2e-5
    # on-axis amplitude w0/w(z) and Gouy phase for the centred round beam
    if x0 == 0 and wx == wy and ny % 2 == 0:
        zr = math.pi * wx * wx / lam
        w = wx * math.sqrt(1 + (z / zr) ** 2)
        c = ny // 2
        centre = out[c - 1:c + 1, c - 1:c + 1].mean()
        r2 = 2 * (dx / 2) ** 2
        expect = (wx / w) * np.exp(1j * (2 * math.pi / lam * z - math.atan(z / zr))) * \
            np.exp(-r2 / w ** 2) * np.exp(1j * math.pi * r2 / (lam * z * (1 + (zr / z) ** 2)))
        assert abs(centre - expect) < 1e-5


def test_lens_focus_is_airy():
    """Plane wave through circ(a) and a thin lens of focal length f, propagated f (AS).

    I(r) = I0 (2 J1(v)/v)^2 with v = k a r / f and I0 = (pi a^2 / (lambda f))^2.
    """
    n, d, lam, f, a = 512, 10e-6, 0.5e-6, 0.2, 1e-3
    e = O.circ(n, n, d, d, a) * O.lens(n, n, d, d, lam, f)
    out = O.intensity(O.propagate(e, d, d, lam, f, 2.0)[0])
    x = O.coords(n, d)
    r = np.sqrt(x[None, :] ** 2 + x[:, None] ** 2)
    v = 2 * math.pi / lam * a * r / f
    airy = (2 * j1(v) / v) ** 2
    i0 = (math.pi * a * a / (lam * f)) ** 2
    m = r < 5 * 0.61 * lam * f / a
    err = np.linalg.norm((out - i0 * airy)[m]) / np.linalg.norm((i0 * airy)[m])
    assert err < 3e-3


def test_rayleigh_sommerfeld_bruteforce_matches_as():
    """Brute-force Eq. 2-3 on a 32^2 grid at z = z_critical agrees with AS (Eq. 4-5)."""
    n, d, lam, w0 = 32, 2e-6, 0.5e-6, 8e-6
    z = 250e-6
    f0 = gaussian_beam(n, n, d, d, w0)
    rs = O.rs_bruteforce(f0, d, d, lam, z)
    asr = O.propagate(f0, d, d, lam, z, 3.0)[0]
    assert rel_l2(asr, rs) < 2e-5
    c = n // 4
    assert rel_l2(asr[c:-c, c:-c], rs[c:-c, c:-c]) < 1e-7


def test_direct_integration_is_the_rayleigh_sommerfeld_sum():
    """DI (Eq. 2-3 by FFT with P >= 2n - 1) equals the brute-force sum of Eq. 2 to rounding, on a
    non-square grid with dx != dy, at a short and a long distance."""
    ny, nx, dy, dx, lam = 24, 32, 3e-6, 2e-6, 0.6e-6
    f0 = to_c64(normal(41, (ny, nx)) + 1j * normal(42, (ny, nx))).astype(np.complex128)
    for z, pad in ((40e-6, 2.0), (2e-3, 2.5)):
        rs = O.rs_bruteforce(f0, dy, dx, lam, z)
        di = O.propagate(f0, dy, dx, lam, z, pad, O.DI)[0]
        assert rel_l2(di, rs) < 1e-12
    with pytest.raises(ValueError):
        O.propagate(f0, dy, dx, lam, 2e-3, 1.5, O.DI)


def test_direct_integration_beyond_z_critical_follows_the_beam():
    """Far beyond z_critical (Eq. 6) the AS transfer function is undersampled while DI keeps
    following the Gaussian beam (exact paraxial solution; the beam is wide against lambda, so
    its non-paraxial correction is far below the tolerance)."""
    n, d, lam, w0 = 64, 5e-6, 0.5e-6, 10e-6
    zc = O.z_critical(n * d, d, lam)
    z = 4 * zc  # the beam has spread to w(z) = 204 um on a 320 um grid
    f0 = gaussian_beam(n, n, d, d, w0)
    ref = paraxial_gaussian(n, n, d, d, lam, z, w0, w0)
    err_di = rel_l2(O.propagate(f0, d, d, lam, z, 2.0, O.DI)[0], ref)
    err_as = rel_l2(O.propagate(f0, d, d, lam, z, 2.0, O.AS)[0], ref)
    assert err_di < 5e-4  # the paraxial model's own error, (lambda / (pi w0))^2 = 2.5e-4
    assert err_as > 5 * err_di


def test_automatic_method_follows_eq6():
    ny, nx, dy, dx, lam = 16, 24, 4e-6, 5e-6, 0.5e-6
    f0 = to_c64(normal(43, (ny, nx)) + 1j * normal(44, (ny, nx))).astype(np.complex128)
    zc = min(O.z_critical(nx * dx, dx, lam), O.z_critical(ny * dy, dy, lam))
    assert zc == pytest.approx(ny * dy * dy / lam)
    below = O.propagate(f0, dy, dx, lam, 0.5 * zc, 2.0, O.AUTO)
    above = O.propagate(f0, dy, dx, lam, 2.0 * zc, 2.0, O.AUTO)
    assert np.array_equal(below, O.propagate(f0, dy, dx, lam, 0.5 * zc, 2.0, O.AS))
    assert np.array_equal(above, O.propagate(f0, dy, dx, lam, 2.0 * zc, 2.0, O.DI))


def test_direct_integration_adjoint_identity():
    ny, nx, d, lam, z = 16, 16, 4e-6, 0.5e-6, 3e-3
    x = to_c64(normal(45, (ny, nx)) + 1j * normal(46, (ny, nx))).astype(np.complex128)
    y = to_c64(normal(47, (ny, nx)) + 1j * normal(48, (ny, nx))).astype(np.complex128)
    px = O.propagate(x, d, d, lam, z, 2.0, O.DI)[0]
    phy = O.propagate_adjoint(y, d, d, lam, z, 2.0, O.DI)[0]
    assert abs(np.vdot(y, px) - np.vdot(phy, x)) < 1e-12 * abs(np.vdot(y, px))


def test_overlap_of_two_gaussians_closed_form():
    """Eq. 7's integral of exp(-|r - a|^2 / w1^2) exp(-|r - b|^2 / w2^2) is
    pi / (1/w1^2 + 1/w2^2) exp(-|a - b|^2 / (w1^2 + w2^2)); well-sampled Gaussians inside the
    grid reproduce it to rounding. The power of a Gaussian is the same integral with itself."""
    ny, nx, dy, dx = 96, 128, 2e-6, 1.5e-6
    w1, w2 = 20e-6, 14e-6
    a, b = (6e-6, -4e-6), (-3e-6, 5e-6)
    x = O.coords(nx, dx)[None, :]
    y = O.coords(ny, dy)[:, None]
    g1 = np.exp(-((x - a[0]) ** 2 + (y - a[1]) ** 2) / w1 ** 2)
    g2 = np.exp(-((x - b[0]) ** 2 + (y - b[1]) ** 2) / w2 ** 2) * np.exp(0.7j)
    ref = math.pi / (1 / w1 ** 2 + 1 / w2 ** 2) * math.exp(-((a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2) / (w1 ** 2 + w2 ** 2))
    o = O.overlap(g1, g2, dy, dx)[0]
    assert abs(o - ref * np.exp(-0.7j)) < 1e-10 * ref
    assert O.power(g1, dy, dx)[0] == pytest.approx(math.pi * w1 * w1 / 2, rel=1e-10)


def test_overlap_loss_gradient_by_finite_differences():
    """dL/dphi of Eq. 7 (batch mean) through a phase mask and an AS propagation: the analytic chain
    (overlap-loss gradient, adjoint propagation, phase gradient) against central differences."""
    n, d, lam, z = 16, 8e-6, 0.6e-6, 2e-3
    s = 0.4 / (n * d)  # unit-order powers
    x = to_c64(normal(51, (2, n, n)) + 1j * normal(52, (2, n, n))).astype(np.complex128) * s
    phi = uniform(55, (n, n), -math.pi, math.pi)
    # a target close to the first output, so |O| is of order 1 and the differences resolve
    tgt = 1.5 * O.propagate(x[:1] * np.exp(1j * uniform(56, (n, n), -0.3, 0.3) + 1j * phi), d, d, lam, z, 2.0)[0]

    def loss(p):
        out = O.propagate(x * np.exp(1j * p), d, d, lam, z, 2.0)
        return O.overlap_loss(out, tgt, d, d)[0]

    m = np.exp(1j * phi)
    out = O.propagate(x * m, d, d, lam, z, 2.0)
    _, g = O.overlap_loss(out, tgt, d, d)
    gy = O.propagate_adjoint(g, d, d, lam, z, 2.0)
    g_phi = O.grad_modulation(x, m, gy)[2]
    idx = np.arange(0, n * n, 7)
    fd = O.finite_difference(loss, phi, idx)
    assert np.max(np.abs(fd - g_phi.reshape(-1)[idx])) < 1e-6 * np.max(np.abs(fd))


def _golden(name):
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_polarizer_powers_printed_in_the_paper():
    """Listing 6: a normalised x-polarised field through linear polarisers at 45 and 90 degrees."""
    n, d = 64, 10e-6
    f = np.zeros((3, n, n), dtype=np.complex128)
    f[0] = 1.0
    f /= math.sqrt(O.power(f, d, d).sum())
    elems = {"polarizer_45": O.linear_polarizer(math.pi / 4), "polarizer_90": O.linear_polarizer(math.pi / 2)}
    for seq, val in _golden("polarizer_powers.txt"):
        g = f
        if seq != "none":
            for e in seq.split(","):
                g = O.jones_modulate(g, elems[e])
        assert O.power(g, d, d).sum() == pytest.approx(float(val), abs=1e-12)


def test_malus_law_and_waveplates():
    """Malus's law cos^2; a quarter-wave plate at 45 degrees turns x into circular light (equal
    powers, phase +-pi/2 between y and x); a half-wave plate at theta rotates x to 2 theta; a
    circular polariser passes half of linear light."""
    f = np.zeros((3, 1, 1), dtype=np.complex128)
    f[0] = 1.0
    for th in (0.1, 0.7, 1.3):
        assert np.sum(np.abs(O.jones_modulate(f, O.linear_polarizer(th))) ** 2) == pytest.approx(math.cos(th) ** 2, abs=1e-14)
    q = O.jones_modulate(f, O.waveplate(math.pi / 2, math.pi / 4))[:, 0, 0]
    assert abs(abs(q[0]) - abs(q[1])) < 1e-14 and abs(abs(np.angle(q[1] / q[0])) - math.pi / 2) < 1e-14
    th = 0.3
    h = O.jones_modulate(f, O.waveplate(math.pi, th))[:, 0, 0]
    assert abs(abs(h[0]) - abs(math.cos(2 * th))) < 1e-14 and abs(abs(h[1]) - abs(math.sin(2 * th))) < 1e-14
    for hand in (1, -1):
        assert np.sum(np.abs(O.jones_modulate(f, O.circular_polarizer(hand))) ** 2) == pytest.approx(0.5, abs=1e-14)
        v = O.jones_modulate(O.jones_modulate(f, O.circular_polarizer(hand)), O.circular_polarizer(-hand))
        assert np.sum(np.abs(v) ** 2) < 1e-28


def test_jones_backward_by_finite_differences():
    rng_f = to_c64(normal(61, (2, 3, 4, 5)) + 1j * normal(62, (2, 3, 4, 5))).astype(np.complex128)
    jm = to_c64(normal(63, (3, 3, 4, 5)) + 1j * normal(64, (3, 3, 4, 5))).astype(np.complex128)
    w = to_c64(normal(65, (2, 3, 4, 5)) + 1j * normal(66, (2, 3, 4, 5))).astype(np.complex128)

    def loss(jr, ji, fr, fi):
        out = O.jones_modulate(fr + 1j * fi, jr + 1j * ji)
        return float(np.real(np.sum(np.conj(w) * out)))  # L = Re <w, out>, so dL/dout = w

    g_in, g_j = O.grad_jones(rng_f, jm, w)
    h = 1e-6
    for idx in [(0, 1, 2, 3), (2, 2, 0, 0), (1, 0, 3, 4)]:
        for part, g in ((0, g_j.real), (1, g_j.imag)):
            a = [jm.real.copy(), jm.imag.copy()]
            a[part][idx] += h
            lp = loss(a[0], a[1], rng_f.real, rng_f.imag)
            a[part][idx] -= 2 * h
            lm = loss(a[0], a[1], rng_f.real, rng_f.imag)
            assert (lp - lm) / (2 * h) == pytest.approx(g[idx], rel=1e-6, abs=1e-9)
    for idx in [(0, 1, 2, 3), (1, 2, 0, 4)]:
        for part, g in ((0, g_in.real), (1, g_in.imag)):
            a = [rng_f.real.copy(), rng_f.imag.copy()]
            a[part][idx] += h
            lp = loss(jm.real, jm.imag, a[0], a[1])
            a[part][idx] -= 2 * h
            lm = loss(jm.real, jm.imag, a[0], a[1])
            assert (lp - lm) / (2 * h) == pytest.approx(g[idx], rel=1e-6, abs=1e-9)


def test_bilinear_resampling_reproduces_bilinear_functions():
    """Bilinear interpolation is exact for a + b x + c y + e x y inside the input grid; nearest
    picks the closest sample; equal grids give the identity; the adjoint identity holds."""
    ny, nx, dy, dx = 20, 30, 3e-6, 2e-6
    ny2, nx2, dy2, dx2 = 17, 23, 2.5e-6, 1.7e-6
    x = O.coords(nx, dx)[None, :]
    y = O.coords(ny, dy)[:, None]
    fn = lambda xx, yy: (0.3 + 2e5 * xx - 1e5 * yy + 4e9 * xx * yy) * (1 + 0.5j)
    out = O.resample(fn(x, y), dy, dx, ny2, nx2, dy2, dx2, O.BILINEAR)[0]
    x2 = O.coords(nx2, dx2)[None, :]
    y2 = O.coords(ny2, dy2)[:, None]
    assert np.max(np.abs(out - fn(x2, y2))) < 1e-12
    near = O.resample(fn(x, y), dy, dx, ny2, nx2, dy2, dx2, O.NEAREST)[0]
    jx = np.floor(x2[0] / dx + (nx - 1) / 2 + 0.5).astype(int)
    jy = np.floor(y2[:, 0] / dy + (ny - 1) / 2 + 0.5).astype(int)
    assert np.array_equal(near, fn(x, y)[np.ix_(jy, jx)])
    f = to_c64(normal(71, (2, ny, nx)) + 1j * normal(72, (2, ny, nx))).astype(np.complex128)
    assert np.array_equal(O.resample(f, dy, dx, ny, nx, dy, dx), f)
    g = to_c64(normal(73, (2, ny2, nx2)) + 1j * normal(74, (2, ny2, nx2))).astype(np.complex128)
    for mode in (O.NEAREST, O.BILINEAR):
        a = np.vdot(g, O.resample(f, dy, dx, ny2, nx2, dy2, dx2, mode))
        b = np.vdot(O.resample_adjoint(g, ny, nx, dy, dx, dy2, dx2, mode), f)
        assert abs(a - b) < 1e-12 * abs(a)


# ----------------------------------------------------------------------------- coherence

def test_gsm_spreading_mandel_wolf():
    """GSM source: I(r, z) = exp(-r^2 / (2 s^2 D^2)) / D^2, D^2 = 1 + (z/(k s delta))^2.

    s = w/2 is the rms intensity width, 1/delta^2 = 1/(4 s^2) + 1/l^2 (Eq. 11-13).
    """
    n, d, lam, w0, lc = 32, 10e-6, 633e-9, 60e-6, 20e-6
    g = gaussian_schell(n, d, w0, lc)
    for z in (0.002, 0.005):
        gz = O.propagate_coherence(g, d, d, lam, z, 2.0, O.FRESNEL_TF)
        s = w0 / 2
        k = 2 * math.pi / lam
        delta = 1 / math.sqrt(1 / (4 * s * s) + 1 / (lc * lc))
        d2 = 1 + (z / (k * s * delta)) ** 2
        x = O.coords(n, d)
        r2 = x[None, :] ** 2 + x[:, None] ** 2
        assert rel_l2(O.coherence_diag(gz), np.exp(-r2 / (2 * s * s * d2)) / d2) < 5e-6
        m = gz.reshape(n * n, n * n)
        assert np.abs(m - m.conj().T).max() < 1e-14 * np.abs(m).max()


def test_coherence_rank_one_equals_coherent():
    """Gamma = psi psi^H gives Gamma_z = (P psi)(P psi)^H; sums of rank-one terms likewise."""
    n, d, lam, z = 10, 8e-6, 600e-9, 0.01
    psis = [normal(20 + i, (n, n)) + 1j * normal(30 + i, (n, n)) for i in range(2)]
    g = sum(np.einsum("ab,cd->abcd", p, np.conj(p)) for p in psis)
    mask = np.exp(1j * uniform(40, (n, n), -math.pi, math.pi))
    gz = O.propagate_coherence(O.modulate_coherence(g, mask), d, d, lam, z, 2.0)
    expect = 0
    for p in psis:
        q = O.propagate(p * mask, d, d, lam, z, 2.0)[0]
        expect = expect + np.einsum("ab,cd->abcd", q, np.conj(q))
    assert rel_l2(gz, expect) < 1e-13


# ----------------------------------------------------------------------------- gradients

def _chain_loss(phi, x, target, d, lam):
    y = O.modulate(O.propagate(x, d, d, lam, 0.01, 2.0), O.phase_mask(phi))
    i = O.intensity(O.propagate(y, d, d, lam, 0.015, 2.0))
    return O.mse_loss(i, target)[0]


def test_phase_mask_gradient_vs_finite_differences():
    n, d, lam = 12, 8e-6, 532e-9
    x = normal(50, (2, n, n)) + 1j * normal(51, (2, n, n))
    target = uniform(52, (2, n, n))
    phi = uniform(53, (n, n), 0, 2 * math.pi)
    # analytic backward: MSE -> |.|^2 -> adjoint propagation -> phase mask
    p1 = O.propagate(x, d, d, lam, 0.01, 2.0)
    y = p1 * O.phase_mask(phi)
    p2 = O.propagate(y, d, d, lam, 0.015, 2.0)
    _, g_i = O.mse_loss(O.intensity(p2), target)
    g_y = O.propagate_adjoint(O.grad_intensity(p2, g_i), d, d, lam, 0.015, 2.0)
    _, _, g_phi = O.grad_modulation(p1, O.phase_mask(phi), g_y)
    idx = np.arange(n * n)
    fd = O.finite_difference(lambda p: _chain_loss(p, x, target, d, lam), phi, idx)
    assert np.max(np.abs(fd - g_phi.reshape(-1))) < 1e-6 * np.max(np.abs(fd)) + 1e-12


def test_complex_input_gradient_vs_finite_differences():
    """Backward of propagate is the adjoint: check dL/dRe, dL/dIm of the input."""
    n, d, lam = 8, 5e-6, 600e-9
    x = normal(60, (1, n, n)) + 1j * normal(61, (1, n, n))
    w = normal(62, (1, n, n)) + 1j * normal(63, (1, n, n))

    def loss(xr, xi):
        out = O.propagate(xr + 1j * xi, d, d, lam, 0.004, 2.0)
        return float(np.real(np.vdot(w, out)))  # L = Re <w, P x>

    g = O.propagate_adjoint(w, d, d, lam, 0.004, 2.0)  # dL/dRe + i dL/dIm = P^H w
    idx = np.arange(n * n)
    fr = O.finite_difference(lambda a: loss(a, x.imag), x.real, idx)
    fi = O.finite_difference(lambda b: loss(x.real, b), x.imag, idx)
    assert np.allclose(fr + 1j * fi, g.reshape(-1), atol=1e-8)


def test_coherence_mask_gradient_vs_finite_differences():
    n, d, lam, z = 6, 10e-6, 633e-9, 0.002
    g0 = gaussian_schell(n, d, 30e-6, 15e-6)
    target = uniform(70, (n, n))
    phi = uniform(71, (n, n), -math.pi, math.pi)

    def loss(p):
        gz = O.propagate_coherence(O.modulate_coherence(g0, np.exp(1j * p)), d, d, lam, z, 2.0)
        return O.mse_loss(O.coherence_diag(gz), target)[0]

    m = np.exp(1j * phi)
    gz = O.propagate_coherence(O.modulate_coherence(g0, m), d, d, lam, z, 2.0)
    _, g_i = O.mse_loss(O.coherence_diag(gz), target)
    gd = np.diag(g_i.reshape(-1).astype(np.complex128)).reshape(n, n, n, n)
    g_m_gamma = O.propagate_coherence(gd, d, d, lam, z, 2.0, adjoint=True)
    g_m = O.grad_modulate_coherence(g0, m, g_m_gamma)
    g_phi = np.imag(np.conj(m) * g_m)  # dM/dphi = i M, so dL/dphi = Re(conj(g_M) i M)
    fd = O.finite_difference(loss, phi, np.arange(n * n))
    assert np.max(np.abs(fd - g_phi.reshape(-1))) < 1e-6 * np.max(np.abs(fd))


def test_intensity_sum_closed_form():
    """Eq. 14 on constant fields c_b: each group's plane is sum_b w_b |c_b|^2 (here 30 and 5.25
    unweighted, 21.5 and 13.25 with the weights)."""
    c = np.array([1, 2j, 3 + 4j, 0.5, -1, 2])
    fields = c[:, None, None] * np.ones((6, 3, 4))
    i = O.intensity_sum(fields, 3)
    np.testing.assert_allclose(i[:, 0, 0], [30.0, 5.25], rtol=1e-15)
    assert np.all(i == i[:, :1, :1])
    iw = O.intensity_sum(fields, 3, [1.0, 2.0, 0.5, 1.0, 1.0, 3.0])
    np.testing.assert_allclose(iw[:, 0, 0], [21.5, 13.25], rtol=1e-15)


def test_fourf_images_the_inverted_object():
    """The 4f system with an open pupil is an imaging system: the intensity at the output plane
    is the object's, inverted through the axis (a Gaussian 150 um right and 100 um down of the
    axis arrives 150 um left and 100 um up). A diverging lens, a swapped order or a missing
    inversion fails it."""
    n, d, f, lam = 128, 10e-6, 0.05, 500e-9
    x = (np.arange(n) - (n - 1) / 2) * d
    X, Y = np.meshgrid(x, x)
    obj = np.exp(-((X - 150e-6) ** 2 + (Y + 100e-6) ** 2) / (80e-6) ** 2).astype(np.complex128)[None]
    p4, _ = O.fourf_forward(obj, [lam], d, f, 0.64e-3, 0.64e-3, np.zeros((n, n)), 2.0)
    image = np.abs(p4[0]) ** 2
    assert rel_l2(image, np.abs(obj[0][::-1, ::-1]) ** 2) < 1e-5


def test_fourf_pupil_gradient_vs_finite_differences():
    n, d, f = 16, 20e-6, 0.05
    lams = np.array([500e-9, 650e-9, 500e-9, 650e-9])
    obj = np.repeat(uniform(80, (2, 1, n, n)), 2, axis=1).reshape(4, n, n)
    target = uniform(81, (2, n, n))
    phi = uniform(82, (n, n), -math.pi, math.pi)
    loss, g_phi, _ = O.fourf_loss_and_grad(obj, lams, d, f, 0.16e-3, 0.1e-3, phi, 2, target)
    idx = np.flatnonzero(O.circ(n, n, d, d, 0.1e-3).reshape(-1))[::3]

    def fl(p):
        return O.fourf_loss_and_grad(obj, lams, d, f, 0.16e-3, 0.1e-3, p, 2, target)[0]

    fd = O.finite_difference(fl, phi, idx)
    assert np.max(np.abs(fd - g_phi.reshape(-1)[idx])) < 1e-5 * np.max(np.abs(fd))


# ----------------------------------------------------------------------------- planted mistakes

def _pins_pass():
    """Run a cheap subset of the pins; False if any fails."""
    try:
        for case in GAUSS_CASES:
            test_fresnel_tf_equals_paraxial_gaussian(case)
            test_as_matches_paraxial_gaussian(case)
        test_rayleigh_sommerfeld_bruteforce_matches_as()
        test_adjoint_identity(O.AS)
        test_identity_at_z0(O.AS, 2.0)
        for ab in [(3, 1), (-4, 2)]:
            test_plane_wave_is_eigenvector(*ab)
        test_direct_integration_is_the_rayleigh_sommerfeld_sum()
        test_automatic_method_follows_eq6()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mistake", ["h_sign", "h_conj_adjoint", "swap_axes", "no_norm", "crop_shift",
                                     "freq_order", "fresnel_sign", "drop_global_phase", "di_no_area",
                                     "di_unsigned_lags", "di_conj_kernel", "auto_inverted"])
def test_planted_mistakes(monkeypatch, mistake):
    """A plausible slip planted in the oracle must make at least one pin fail."""
    assert _pins_pass()
    tf = O.optics.transfer_function
    prop = O.optics.propagate
    if mistake == "h_sign":
        monkeypatch.setattr(O.optics, "transfer_function", lambda *a, **k: np.conj(tf(*a, **k)))
    elif mistake == "h_conj_adjoint":
        monkeypatch.setattr(O, "propagate_adjoint",
                            lambda f, dy, dx, lam, z, pad=2.0, method=O.AS, **kw:
                            prop(f, dy, dx, lam, z, pad, method, adjoint=False, **kw))
    elif mistake == "swap_axes":
        monkeypatch.setattr(O.optics, "transfer_function",
                            lambda py, px, dy, dx, lam, z, m=O.AS: tf(py, px, dx, dy, lam, z, m))
    elif mistake == "no_norm":
        monkeypatch.setattr(O.optics, "idft2", lambda x, naive=False: np.fft.ifft2(x) * x.shape[-1])
    elif mistake == "crop_shift":
        # crop one sample away from the window that was padded
        monkeypatch.setattr(O, "propagate", lambda *a, **k: np.roll(prop(*a, **k), 1, axis=-1))
    elif mistake == "freq_order":
        monkeypatch.setattr(O.optics, "freqs", lambda p, d: np.fft.fftshift(O.signed_index(p)) / (p * d))
    elif mistake == "fresnel_sign":
        monkeypatch.setattr(O.optics, "transfer_function",
                            lambda py, px, dy, dx, lam, z, m=O.AS:
                            tf(py, px, dy, dx, lam, z, m) if m == O.AS else
                            np.exp(2j * math.pi * z / lam) * np.conj(tf(py, px, dy, dx, lam, z, m) *
                                                                     np.exp(-2j * math.pi * z / lam)))
    elif mistake == "drop_global_phase":
        monkeypatch.setattr(O.optics, "transfer_function",
                            lambda py, px, dy, dx, lam, z, m=O.AS:
                            tf(py, px, dy, dx, lam, z, m) * np.exp(-2j * math.pi * z / lam))
    elif mistake == "di_no_area":
        di = O.optics.di_transfer_function
        monkeypatch.setattr(O.optics, "di_transfer_function", lambda py, px, dy, dx, lam, z:
                            di(py, px, dy, dx, lam, z) / (dx * dy))
    elif mistake == "di_unsigned_lags":
        monkeypatch.setattr(O.optics, "signed_index", lambda p: np.arange(p))
    elif mistake == "di_conj_kernel":
        h = O.optics.impulse_response
        monkeypatch.setattr(O.optics, "impulse_response", lambda x, y, lam, z: np.conj(h(x, y, lam, z)))
    elif mistake == "auto_inverted":
        ch = O.optics.choose_method
        monkeypatch.setattr(O.optics, "choose_method",
                            lambda *a: O.DI if ch(*a) == O.AS else O.AS)
    assert not _pins_pass()
