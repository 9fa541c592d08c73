"""FP64 CPU oracle for scalar free-space propagation of sampled fields.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The CUDA library never
calls it, and this module never imports the CUDA library.

Everything here is the plain definition written out in float64, following the
paper (TorchOptics, arXiv 2411.18591):

* modulation is a point-wise product (Eq. 1);
* the Rayleigh-Sommerfeld integral (Eq. 2) with impulse response h_z (Eq. 3) is
  evaluated by brute-force summation on tiny grids;
* angular-spectrum (AS) propagation (Eq. 4) multiplies the 2-D Fourier transform
  of the zero-padded field by the transfer function H_z (Eq. 5), then inverts,
  with "configurable zero-padding" (§3);
* the Fresnel variant (§3) uses the Fresnel transfer function;
* Direct Integration (DI, §3) evaluates Eq. 2 as a convolution with h_z of Eq. 3
  sampled at the grid's lags: the DFT of those samples (times dx dy) multiplies the
  spectrum of the zero-padded field; with P >= 2n - 1 the cropped result is exactly the
  direct sum of Eq. 2;
* the critical distance is Eq. 6, and the automatic choice takes AS below it and DI
  above it (§3);
* mutual coherence is modulated by M(r1) M*(r2) (Eq. 12) and propagated with
  h_z on r1 and h_z* on r2 (Eq. 13);
* polychromatic intensity is the incoherent sum over wavelengths (Eq. 14);
* the overlap loss is Eq. 7 with the integral as a sum times dx dy, averaged over a batch;
* polarisation elements act as Jones matrices on (psi_x, psi_y) per pixel (§5.1), the z
  component of a three-component field passing unchanged;
* a field moves between grids of different spacing by nearest or bilinear interpolation of
  the centred sample positions (§3), samples outside the input grid counting as zero.

Readings of points the paper leaves open:

* padded size P = floor(pad * n + 0.5) per axis; the field sits at offset
  floor((P - n)/2) of the padded grid and is cropped from the same window;
* frequencies f_k = k / (P d), k in FFT order (0 .. ceil(P/2)-1, -floor(P/2) .. -1);
* the forward DFT is unnormalised, the inverse carries 1/(Py Px);
* AS evanescent samples (1/lambda^2 - fx^2 - fy^2 < 0) are set to zero;
* Fresnel transfer function H = exp(2 pi i z / lambda) exp(-i pi lambda z (fx^2 + fy^2));
* grid samples at (i - (n-1)/2) d; apertures pass r <= R (pixel centres);
* thin lens M = exp(-i pi (x^2 + y^2) / (lambda f)), converging for z > 0;
* gradients follow the real-loss convention g = dL/dRe + i dL/dIm, so the
  backward of a complex-linear map A is A^H.

The library FFT (numpy's pocketfft) serves as a step; ``dft_naive`` is the
definition written out and is used to cross-check it on small sizes.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

AS = 0
FRESNEL_TF = 1
DI = 2
AUTO = 3


# ----------------------------------------------------------------------------- grid

def padded_size(n: int, pad: float) -> int:
    """P = floor(pad * n + 0.5); P >= n is required (§3 zero-padding)."""
    p = int(math.floor(pad * n + 0.5))
    if p < n:
        raise ValueError("padded size smaller than the field")
    return p


def pad_offset(n: int, p: int) -> int:
    return (p - n) // 2


def coords(n: int, d: float) -> np.ndarray:
    """x_i = (i - (n-1)/2) d: grid centred on the optical axis (§3)."""
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * d


def signed_index(p: int) -> np.ndarray:
    """FFT-order frequency index: 0 .. ceil(P/2)-1, then -floor(P/2) .. -1."""
    k = np.arange(p, dtype=np.int64)
    return np.where(k < (p + 1) // 2, k, k - p)


def freqs(p: int, d: float) -> np.ndarray:
    """Spatial frequencies f_k = k / (P d) in cycles per metre."""
    return signed_index(p).astype(np.float64) / (p * d)


def z_critical(L: float, dx: float, lam: float) -> float:
    """Eq. 6: z_critical = L dx / lambda; AS is preferred below it."""
    return L * dx / lam


# ----------------------------------------------------------------------------- DFT

def dft_matrix(p: int, sign: int) -> np.ndarray:
    """W[k, n] = exp(sign * 2 pi i (k n mod P) / P), the DFT written out.

    The product k n is reduced modulo P in integers before the phase is formed,
    so the phase argument stays in [0, 2 pi).
    """
    k = np.arange(p, dtype=np.int64)
    kn = np.outer(k, k) % p
    return np.exp(sign * 2j * math.pi * kn.astype(np.float64) / p)


def dft2(x: np.ndarray, naive: bool = False) -> np.ndarray:
    """Unnormalised forward 2-D DFT over the last two axes."""
    if not naive:
        return np.fft.fft2(x, axes=(-2, -1))
    wy = dft_matrix(x.shape[-2], -1)
    wx = dft_matrix(x.shape[-1], -1)
    return np.einsum("ky,...yx,jx->...kj", wy, x, wx)


def idft2(x: np.ndarray, naive: bool = False) -> np.ndarray:
    """Inverse 2-D DFT over the last two axes, with 1/(Py Px)."""
    if not naive:
        return np.fft.ifft2(x, axes=(-2, -1))
    py, px = x.shape[-2], x.shape[-1]
    wy = dft_matrix(py, +1)
    wx = dft_matrix(px, +1)
    return np.einsum("ky,...yx,jx->...kj", wy, x, wx) / (py * px)


# ----------------------------------------------------------------------------- transfer function

def impulse_response(x, y, lam: float, z: float):
    """h_z of Eq. 3 at lateral offsets (x, y): z / (i lambda d) (1 + i / (k d)) exp(i k d) / d,
    d = sqrt(x^2 + y^2 + z^2), k = 2 pi / lambda."""
    k = 2.0 * math.pi / lam
    d = np.sqrt(x * x + y * y + z * z)
    return z / (1j * lam * d) * (1.0 + 1j / (k * d)) * np.exp(1j * k * d) / d


def di_transfer_function(py: int, px: int, dy: float, dx: float, lam: float, z: float) -> np.ndarray:
    """DI (§3): the forward DFT of h_z (Eq. 3) sampled at the signed lags of the padded grid
    (lag m of an axis is its signed FFT index), times dx dy, shape [Py, Px]. Multiplying the
    spectrum of a zero-padded field by it is the circular convolution with those samples; for
    an n-sample field and P >= 2n - 1 the cropped window is the direct sum of Eq. 2."""
    x = signed_index(px).astype(np.float64) * dx
    y = signed_index(py).astype(np.float64) * dy
    h = impulse_response(x[None, :], y[:, None], lam, z) * (dx * dy)
    return np.fft.fft2(h)


def choose_method(ny: int, nx: int, dy: float, dx: float, lam: float, z: float) -> int:
    """Eq. 6 per axis, z_crit = L dx / lambda with L = n d the grid length: AS when z is below
    the smaller of the two critical distances, else DI."""
    zc = min(z_critical(nx * dx, dx, lam), z_critical(ny * dy, dy, lam))
    return AS if z < zc else DI


def transfer_function(py: int, px: int, dy: float, dx: float, lam: float, z: float,
                      method: int = AS) -> np.ndarray:
    """H_z on the padded frequency grid, shape [Py, Px] (Eq. 5, §3).

    AS: H = exp(2 pi i z sqrt(1/lambda^2 - fx^2 - fy^2)), which is Eq. 5 with
    k = 2 pi / lambda and (kx, ky) = 2 pi (fx, fy); samples with a negative
    radicand are evanescent and set to zero. The radicand is evaluated as
    ((1/(lambda*lambda)) - fx*fx) - fy*fy.
    Fresnel: H = exp(2 pi i z / lambda) exp(-i pi lambda z (fx^2 + fy^2)).
    """
    fx = freqs(px, dx)
    fy = freqs(py, dy)
    fx2 = (fx * fx)[None, :]
    fy2 = (fy * fy)[:, None]
    if method == AS:
        inv_l2 = 1.0 / (lam * lam)
        rad = (inv_l2 - fx2) - fy2
        prop = rad >= 0.0
        kz = np.sqrt(np.where(prop, rad, 0.0))
        return np.where(prop, np.exp(2j * math.pi * z * kz), 0.0)
    if method == FRESNEL_TF:
        return np.exp(2j * math.pi * z / lam) * np.exp(-1j * math.pi * lam * z * (fx2 + fy2))
    if method == DI:
        return di_transfer_function(py, px, dy, dx, lam, z)
    raise ValueError("unknown method")


# ----------------------------------------------------------------------------- propagation

def _as_batch(field: np.ndarray) -> np.ndarray:
    f = np.asarray(field, dtype=np.complex128)
    return f[None] if f.ndim == 2 else f


def propagate(field: np.ndarray, dy: float, dx: float, lam: float, z: float, pad: float = 2.0,
              method: int = AS, adjoint: bool = False, naive: bool = False,
              offset: Optional[tuple] = None, pad_y: Optional[float] = None) -> np.ndarray:
    """Free-space propagation of a batch of fields [B, ny, nx] by distance z (Eq. 4).

    Steps: zero-pad each field to [Py, Px] at the offset, forward 2-D DFT,
    multiply by H_z (or conj(H_z) for the adjoint), inverse 2-D DFT, crop the
    same window. ``lam`` and ``z`` may be scalars or length-B sequences.
    """
    f = _as_batch(field)
    b, ny, nx = f.shape
    py = padded_size(ny, pad if pad_y is None else pad_y)
    px = padded_size(nx, pad)
    oy, ox = (pad_offset(ny, py), pad_offset(nx, px)) if offset is None else offset
    lams = np.broadcast_to(np.asarray(lam, dtype=np.float64), (b,))
    zs = np.broadcast_to(np.asarray(z, dtype=np.float64), (b,))
    out = np.empty_like(f)
    for i in range(b):
        buf = np.zeros((py, px), dtype=np.complex128)
        buf[oy:oy + ny, ox:ox + nx] = f[i]
        m = choose_method(ny, nx, dy, dx, float(lams[i]), float(zs[i])) if method == AUTO else method
        if m == DI and (py < 2 * ny - 1 or px < 2 * nx - 1):
            raise ValueError("DI needs a padded size of at least 2 n - 1 per axis")
        h = transfer_function(py, px, dy, dx, float(lams[i]), float(zs[i]), m)
        if adjoint:
            h = np.conj(h)
        res = idft2(dft2(buf, naive) * h, naive)
        out[i] = res[oy:oy + ny, ox:ox + nx]
    return out


def propagate_adjoint(field, dy, dx, lam, z, pad=2.0, method=AS, **kw):
    """Backward of ``propagate`` (the adjoint operator: conj(H_z) in place of H_z)."""
    return propagate(field, dy, dx, lam, z, pad, method, adjoint=True, **kw)


def rs_bruteforce(field: np.ndarray, dy: float, dx: float, lam: float, z: float) -> np.ndarray:
    """Rayleigh-Sommerfeld integral (Eq. 2) as a direct sum with h_z of Eq. 3.

    psi_z(x, y) = sum_{x', y'} h_z(x - x', y - y') psi_0(x', y') dx dy, with
    h_z = z / (i lambda d) (1 + i / (k d)) exp(i k d) / d and
    d = sqrt((x - x')^2 + (y - y')^2 + z^2). Output on the input grid. O(n^4).
    """
    f = np.asarray(field, dtype=np.complex128)
    ny, nx = f.shape
    k = 2.0 * math.pi / lam
    x = coords(nx, dx)
    y = coords(ny, dy)
    ddx = x[:, None] - x[None, :]  # [x_out, x_in]
    ddy = y[:, None] - y[None, :]
    d = np.sqrt(ddy[:, None, :, None] ** 2 + ddx[None, :, None, :] ** 2 + z * z)
    h = z / (1j * lam * d) * (1.0 + 1j / (k * d)) * np.exp(1j * k * d) / d
    return np.einsum("abcd,cd->ab", h, f) * dx * dy


# ----------------------------------------------------------------------------- elements

def circ(ny: int, nx: int, dy: float, dx: float, radius: float) -> np.ndarray:
    """Circular aperture: 1 where x^2 + y^2 <= R^2 at pixel centres, else 0 (§5.4)."""
    x = coords(nx, dx)[None, :]
    y = coords(ny, dy)[:, None]
    return ((x * x + y * y) <= radius * radius).astype(np.float64)


def lens(ny: int, nx: int, dy: float, dx: float, lam: float, focal: float) -> np.ndarray:
    """Thin-lens quadratic phase exp(-i pi (x^2 + y^2) / (lambda f)) (§2, §5.4)."""
    x = coords(nx, dx)[None, :]
    y = coords(ny, dy)[:, None]
    return np.exp(-1j * math.pi * (x * x + y * y) / (lam * focal))


def modulate(field: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Eq. 1: psi_out = M psi_in (point-wise; M broadcasts over the batch)."""
    return np.asarray(field, dtype=np.complex128) * np.asarray(mask)


def phase_mask(phase: np.ndarray, amplitude=None) -> np.ndarray:
    """M = A exp(i phi) for a phase (and optional amplitude) profile."""
    m = np.exp(1j * np.asarray(phase, dtype=np.float64))
    return m if amplitude is None else np.asarray(amplitude, dtype=np.float64) * m


def intensity(field: np.ndarray) -> np.ndarray:
    """|psi|^2."""
    f = np.asarray(field, dtype=np.complex128)
    return f.real * f.real + f.imag * f.imag


def intensity_sum(field: np.ndarray, group: int, weights=None) -> np.ndarray:
    """Incoherent sum of intensities over consecutive groups of fields (Eq. 14).

    Fields [B, ny, nx] are split into B/group consecutive groups; each output
    plane is sum_b w_b |psi_b|^2 over its group (weights default to 1).
    """
    i = intensity(field)
    b = i.shape[0]
    w = np.ones(b) if weights is None else np.broadcast_to(np.asarray(weights, np.float64), (b,))
    return (i * w[:, None, None]).reshape(b // group, group, *i.shape[1:]).sum(axis=1)


def power(field: np.ndarray, dy: float, dx: float) -> np.ndarray:
    """Total power sum |psi|^2 dx dy per field."""
    return intensity(_as_batch(field)).sum(axis=(-2, -1)) * dx * dy


def overlap(field: np.ndarray, target: np.ndarray, dy: float, dx: float) -> np.ndarray:
    """The integral of Eq. 7 per field: O_b = sum_{x,y} psi_b conj(phi) dx dy (phi [ny, nx] shared
    or [B, ny, nx] per field)."""
    f = _as_batch(field)
    t = np.asarray(target, dtype=np.complex128)
    return (f * np.conj(t)).sum(axis=(-2, -1)) * dx * dy


def overlap_loss(field: np.ndarray, target: np.ndarray, dy: float, dx: float):
    """Eq. 7 averaged over the batch, L = mean_b (1 - |O_b|^2), and dL/dpsi in the real-loss
    convention: d|O|^2 = 2 Re(conj(O) dO) with dO = conj(phi) dpsi dx dy gives
    g_b = -(2 / B) O_b phi dx dy."""
    f = _as_batch(field)
    o = overlap(f, target, dy, dx)
    b = f.shape[0]
    t = np.broadcast_to(np.asarray(target, dtype=np.complex128), f.shape)
    loss = float(np.mean(1.0 - np.abs(o) ** 2))
    grad = -(2.0 / b) * o[:, None, None] * t * (dx * dy)
    return loss, grad


# ----------------------------------------------------------------------------- unequal spacings (§3)

NEAREST = 0
BILINEAR = 1


def resample_weights(n_in: int, d_in: float, n_out: int, d_out: float, mode: int) -> np.ndarray:
    """Interpolation matrix [n_out, n_in] along one axis between centred grids (sample i at
    (i - (n-1)/2) d): output sample j sits at fractional input index
    u = (j - (n_out-1)/2) d_out / d_in + (n_in-1)/2. NEAREST takes sample floor(u + 1/2); BILINEAR
    weighs floor(u) by 1 - (u - floor(u)) and floor(u) + 1 by u - floor(u). Samples outside the
    input grid count as zero."""
    w = np.zeros((n_out, n_in))
    for j in range(n_out):
        u = (j - (n_out - 1) / 2.0) * d_out / d_in + (n_in - 1) / 2.0
        if mode == NEAREST:
            i = math.floor(u + 0.5)
            if 0 <= i < n_in:
                w[j, i] = 1.0
        else:
            i0 = math.floor(u)
            t = u - i0
            for i, c in ((i0, 1.0 - t), (i0 + 1, t)):
                if 0 <= i < n_in and c != 0.0:
                    w[j, i] += c
    return w


def resample(field: np.ndarray, dy: float, dx: float, ny_out: int, nx_out: int, dy_out: float, dx_out: float,
             mode: int = BILINEAR) -> np.ndarray:
    """A field on one centred grid interpolated onto another (§3: propagation keeps the input
    spacing, then the result is interpolated onto the output grid), separably along y and x."""
    f = _as_batch(field)
    wy = resample_weights(f.shape[-2], dy, ny_out, dy_out, mode)
    wx = resample_weights(f.shape[-1], dx, nx_out, dx_out, mode)
    return wy @ f @ wx.T


def resample_adjoint(g: np.ndarray, ny_in: int, nx_in: int, dy: float, dx: float, dy_out: float, dx_out: float,
                     mode: int = BILINEAR) -> np.ndarray:
    """Backward of ``resample``: the transposed interpolation."""
    gb = _as_batch(g)
    wy = resample_weights(ny_in, dy, gb.shape[-2], dy_out, mode)
    wx = resample_weights(nx_in, dx, gb.shape[-1], dx_out, mode)
    return wy.T @ gb @ wx


# ----------------------------------------------------------------------------- polarisation (§5.1)

def jones_matrix_3x3(j2) -> np.ndarray:
    """A 2 x 2 Jones matrix acting on (psi_x, psi_y), extended to the three field components
    (x, y, z) with the z component passed unchanged."""
    m = np.zeros((3, 3), dtype=np.complex128)
    m[:2, :2] = np.asarray(j2, dtype=np.complex128)
    m[2, 2] = 1.0
    return m


def linear_polarizer(theta: float) -> np.ndarray:
    """Transmission axis at angle theta to x: J = u u^T with u = (cos theta, sin theta)."""
    c, s = math.cos(theta), math.sin(theta)
    return jones_matrix_3x3([[c * c, c * s], [c * s, s * s]])


def circular_polarizer(handedness: int) -> np.ndarray:
    """Projector on (1, i handedness) / sqrt 2: J = v v^H (handedness +1 or -1)."""
    v = np.array([1.0, 1j * handedness]) / math.sqrt(2.0)
    return jones_matrix_3x3(np.outer(v, np.conj(v)))


def waveplate(retardance: float, theta: float) -> np.ndarray:
    """Retarder with its fast axis at theta: J = R(-theta) diag(1, exp(i retardance)) R(theta),
    R the rotation of the coordinates by theta."""
    c, s = math.cos(theta), math.sin(theta)
    r = np.array([[c, s], [-s, c]])
    return jones_matrix_3x3(r.T @ np.diag([1.0, np.exp(1j * retardance)]) @ r)


def jones_modulate(field: np.ndarray, jones: np.ndarray) -> np.ndarray:
    """|psi_out(r)> = J(r) |psi_in(r)> (§5.1) on fields [..., 3, ny, nx]; J is [3, 3] (uniform) or
    [3, 3, ny, nx] (spatially varying)."""
    f = np.asarray(field, dtype=np.complex128)
    j = np.asarray(jones, dtype=np.complex128)
    if j.ndim == 2:
        return np.einsum("ij,...jyx->...iyx", j, f)
    return np.einsum("ijyx,...jyx->...iyx", j, f)


def grad_jones(field: np.ndarray, jones: np.ndarray, g_out: np.ndarray):
    """Backward of jones_modulate: g_in = J^H g_out per pixel, and g_J = sum over the leading
    axes of g_out conj(psi_in)^T (per pixel), in the real-loss convention."""
    f = np.asarray(field, dtype=np.complex128)
    g = np.asarray(g_out, dtype=np.complex128)
    j = np.asarray(jones, dtype=np.complex128)
    if j.ndim == 2:
        g_in = np.einsum("ji,...jyx->...iyx", np.conj(j), g)
    else:
        g_in = np.einsum("jiyx,...jyx->...iyx", np.conj(j), g)
    gb = g.reshape((-1,) + g.shape[-3:])
    fb = f.reshape((-1,) + f.shape[-3:])
    g_j = np.einsum("biyx,bjyx->ijyx", gb, np.conj(fb))
    return g_in, g_j


# ----------------------------------------------------------------------------- coherence

def modulate_coherence(gamma: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Eq. 12: Gamma_out(r1, r2) = M(r1) M*(r2) Gamma_in(r1, r2); gamma [..., ny, nx, ny, nx]."""
    m = np.asarray(mask, dtype=np.complex128)
    return np.asarray(gamma, dtype=np.complex128) * m[:, :, None, None] * np.conj(m)[None, None, :, :]


def propagate_coherence(gamma: np.ndarray, dy: float, dx: float, lam: float, z: float,
                        pad: float = 2.0, method: int = AS, adjoint: bool = False) -> np.ndarray:
    """Eq. 13: h_z on (y1, x1) and h_z* on (y2, x2), i.e. Gamma_z = P Gamma P^H.

    The propagator P of ``propagate`` acts on r1 for every fixed r2, and its
    element-wise conjugate (equal to conj(H_z) in the frequency domain) acts on
    r2 for every fixed r1. ``adjoint`` swaps H and conj(H) (the backward map).
    """
    g = np.asarray(gamma, dtype=np.complex128)
    ny, nx = g.shape[0], g.shape[1]
    # r2 pass: each r1 slice [ny, nx] over (y2, x2) with conj(H) (H for the adjoint)
    a = g.reshape(ny * nx, ny, nx)
    a = propagate(a, dy, dx, lam, z, pad, method, adjoint=not adjoint)
    a = a.reshape(ny, nx, ny, nx)
    # r1 pass: each r2 slice over (y1, x1) with H (conj(H) for the adjoint)
    t = np.ascontiguousarray(a.transpose(2, 3, 0, 1)).reshape(ny * nx, ny, nx)
    t = propagate(t, dy, dx, lam, z, pad, method, adjoint=adjoint)
    return np.ascontiguousarray(t.reshape(ny, nx, ny, nx).transpose(2, 3, 0, 1))


def coherence_diag(gamma: np.ndarray) -> np.ndarray:
    """Intensity Gamma(r, r) (real part), shape [ny, nx]."""
    ny, nx = gamma.shape[0], gamma.shape[1]
    return np.real(np.asarray(gamma).reshape(ny * nx, ny * nx).diagonal()).reshape(ny, nx)


# ----------------------------------------------------------------------------- gradients

def mse_loss(i: np.ndarray, target: np.ndarray):
    """L = mean((I - T)^2) and dL/dI = 2 (I - T) / n."""
    r = np.asarray(i, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(r * r)), 2.0 * r / r.size


def grad_intensity(field: np.ndarray, grad_i: np.ndarray) -> np.ndarray:
    """Backward of I = |psi|^2: g_psi = 2 g_I psi."""
    return 2.0 * np.asarray(grad_i) * np.asarray(field, dtype=np.complex128)


def grad_modulation(x: np.ndarray, mask: np.ndarray, g_y: np.ndarray):
    """Backward of y = M x (Eq. 1).

    Returns (g_x, g_M, g_phi): g_x = conj(M) g_y, g_M = sum_b g_y conj(x), and for
    M = A exp(i phi) the phase gradient g_phi = sum_b Im(g_y conj(y)).
    """
    x = _as_batch(x)
    g = _as_batch(g_y)
    m = np.asarray(mask, dtype=np.complex128)
    y = m * x
    return np.conj(m) * g, (g * np.conj(x)).sum(axis=0), np.imag(g * np.conj(y)).sum(axis=0)


def grad_modulate_coherence(gamma_in: np.ndarray, mask: np.ndarray, g_out: np.ndarray) -> np.ndarray:
    """Backward of Eq. 12 w.r.t. a complex mask M (real-loss convention).

    With Gamma_out(r, s) = M(r) conj(M(s)) Gamma_in(r, s):
    g_M(r) = sum_s G(r, s) conj(Gamma_in(r, s)) M(s)
           + sum_s conj(G(s, r)) Gamma_in(s, r) M(s).
    """
    ny, nx = mask.shape
    n = ny * nx
    m = np.asarray(mask, np.complex128).reshape(n)
    gi = np.asarray(gamma_in, np.complex128).reshape(n, n)
    g = np.asarray(g_out, np.complex128).reshape(n, n)
    t1 = (g * np.conj(gi)) @ m
    t2 = (np.conj(g) * gi).T @ m
    return (t1 + t2).reshape(ny, nx)


def finite_difference(fn, x: np.ndarray, idx, h: float = 1e-6) -> np.ndarray:
    """Central differences (fn(x + h e_i) - fn(x - h e_i)) / 2h for flat indices ``idx``."""
    x = np.array(x, dtype=np.float64, copy=True)
    flat = x.reshape(-1)
    out = np.empty(len(idx))
    for j, i in enumerate(idx):
        v = flat[i]
        flat[i] = v + h
        fp = fn(x)
        flat[i] = v - h
        fm = fn(x)
        flat[i] = v
        out[j] = (fp - fm) / (2.0 * h)
    return out


# ----------------------------------------------------------------------------- systems

def fourf_forward(obj: np.ndarray, lams, d: float, f: float, lens_r: float, pupil_r: float,
                  pupil_phase: np.ndarray, pad: float = 2.0):
    """Polarised, polychromatic 4f system of Fig. 1 / Listing 5 on a batch of fields.

    ``obj`` is [B, ny, nx] (fields ordered object, component, wavelength) and
    ``lams`` the per-field wavelength. Sequence: propagate f, lens (inside a
    circ of radius ``lens_r``), propagate f, pupil circ(R) exp(i phi),
    propagate f, lens, propagate f. Returns (psi at the output plane, saved
    fields needed by the backward pass).
    """
    b, ny, nx = obj.shape
    lams = np.broadcast_to(np.asarray(lams, np.float64), (b,))
    lm = circ(ny, nx, d, d, lens_r)
    pm = circ(ny, nx, d, d, pupil_r) * np.exp(1j * pupil_phase)
    lens_b = np.stack([lm * lens(ny, nx, d, d, l, f) for l in lams])
    p1 = propagate(obj, d, d, lams, f, pad) * lens_b
    p2 = propagate(p1, d, d, lams, f, pad) * pm
    p3 = propagate(p2, d, d, lams, f, pad) * lens_b
    p4 = propagate(p3, d, d, lams, f, pad)
    return p4, dict(p2=p2, p4=p4, lens_b=lens_b, pm=pm)


def fourf_loss_and_grad(obj, lams, d, f, lens_r, pupil_r, pupil_phase, group, target, pad=2.0):
    """MSE on the grouped intensity (Eq. 14) of the 4f system and dL/d(pupil phase).

    Intensities of each consecutive group of ``group`` fields (one object's
    components and wavelengths) are summed before the loss.
    """
    b = obj.shape[0]
    lams = np.broadcast_to(np.asarray(lams, np.float64), (b,))
    p4, s = fourf_forward(obj, lams, d, f, lens_r, pupil_r, pupil_phase, pad)
    inten = intensity_sum(p4, group)
    loss, g_i = mse_loss(inten, target)
    g4 = grad_intensity(p4, np.repeat(g_i, group, axis=0))
    g3 = propagate_adjoint(g4, d, d, lams, f, pad) * np.conj(s["lens_b"])
    g2 = propagate_adjoint(g3, d, d, lams, f, pad)
    g_phi = np.imag(g2 * np.conj(s["p2"])).sum(axis=0)
    return loss, g_phi, inten
