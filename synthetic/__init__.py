"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds only random-number generation and input profiles. It contains
none of the propagation arithmetic (no transfer function, no FFT, no modulation
rule), so the CPU oracle and the CUDA path can both draw from it without sharing
any of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a 64-bit counter advanced by the
golden-ratio increment and passed through the published finaliser. Uniform
doubles take the top 53 bits. Normal deviates use the Box-Muller transform.

The workloads mimic the shapes of the paper's examples (the 4f system of Fig. 1,
the trainable phase masks of Listing 2, the Gaussian Schell-model field of
Listing 4, the polychromatic sum of Listing 5). The paper's own data files are
not available, so seeded stand-ins of the same shape are used.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2411185910

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start`` .. ``start + count - 1`` of the SplitMix64 stream of ``seed`` as uint64
    (the generator is a counter, so any stretch can be drawn directly)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape, low: float = 0.0, high: float = 1.0, start: int = 0) -> np.ndarray:
    """Uniform doubles in [low, high) from the top 53 bits of SplitMix64 (stream offset ``start``)."""
    shape = (shape,) if isinstance(shape, int) else tuple(shape)
    n = int(np.prod(shape)) if shape else 1
    u = (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (low + (high - low) * u).reshape(shape)


def normal(seed: int, shape) -> np.ndarray:
    """Standard normal doubles by Box-Muller on two uniform streams."""
    shape = (shape,) if isinstance(shape, int) else tuple(shape)
    n = int(np.prod(shape)) if shape else 1
    u = uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).reshape(shape)


def sub_seed(seed: int, index: int) -> int:
    """Per-item seed: seed * 1000003 + index (mod 2**64)."""
    return (seed * 1000003 + index) & 0xFFFFFFFFFFFFFFFF


def to_c64(a: np.ndarray) -> np.ndarray:
    """Round to complex64; both sides are fed the rounded values."""
    return np.ascontiguousarray(a, dtype=np.complex64)


def centred_coords(n: int, d: float) -> np.ndarray:
    """Sample positions (i - (n-1)/2) * d of a grid centred on the optical axis."""
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * d


# ----------------------------------------------------------------------------- profiles

def gaussian_beam(ny: int, nx: int, dy: float, dx: float, waist: float,
                  waist_y: float | None = None, x0: float = 0.0, y0: float = 0.0,
                  tilt_x: float = 0.0, tilt_y: float = 0.0) -> np.ndarray:
    """Waist-plane Gaussian exp(-(x-x0)^2/wx^2 - (y-y0)^2/wy^2) * exp(2 pi i (ax x + ay y)).

    ``tilt_x``/``tilt_y`` are spatial frequencies (1/m) of a linear phase. The
    profile family of the paper's profiles subpackage (§5.4); complex128.
    """
    wy = waist if waist_y is None else waist_y
    x = centred_coords(nx, dx)[None, :]
    y = centred_coords(ny, dy)[:, None]
    amp = np.exp(-((x - x0) ** 2) / waist ** 2 - ((y - y0) ** 2) / wy ** 2)
    ph = np.exp(2j * math.pi * (tilt_x * x + tilt_y * y))
    return amp * ph


def gaussian_schell(n: int, d: float, waist: float, coherence: float) -> np.ndarray:
    """Gaussian Schell-model mutual coherence on an n x n grid, shape [n, n, n, n].

    G(r1, r2) = exp(-(|r1|^2 + |r2|^2)/w^2) * exp(-|r1 - r2|^2 / (2 l^2)),
    with w the beam width and l the coherence length (§5.2, Listing 4).
    """
    c = centred_coords(n, d)
    y1 = c[:, None, None, None]
    x1 = c[None, :, None, None]
    y2 = c[None, None, :, None]
    x2 = c[None, None, None, :]
    inten = np.exp(-(x1 ** 2 + y1 ** 2 + x2 ** 2 + y2 ** 2) / waist ** 2)
    corr = np.exp(-((x1 - x2) ** 2 + (y1 - y2) ** 2) / (2.0 * coherence ** 2))
    return inten * corr


def binary_pattern(seed: int, batch: int, n: int, p: float = 0.5) -> np.ndarray:
    """Bernoulli(p) amplitude patterns with zero phase, [batch, n, n] float64."""
    return (uniform(seed, (batch, n, n)) < p).astype(np.float64)


def smooth_noise(seed: int, shape, sigma_px: float, std: float = 1.0) -> np.ndarray:
    """White N(0,1) noise filtered by a Gaussian of ``sigma_px`` pixels, rescaled to ``std``.

    The filter is a direct separable convolution with a truncated (4 sigma)
    normalised Gaussian kernel and periodic boundaries; no FFT is involved.
    """
    shape = tuple(shape)
    w = normal(seed, shape)
    r = int(math.ceil(4.0 * sigma_px))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma_px) ** 2)
    k /= k.sum()
    out = np.zeros_like(w)
    for i, kv in enumerate(k):
        out += kv * np.roll(w, i - r, axis=-1)
    out2 = np.zeros_like(out)
    for i, kv in enumerate(k):
        out2 += kv * np.roll(out, i - r, axis=-2)
    s = out2.std(axis=(-2, -1), keepdims=True)
    return out2 * (std / s)


def phase_screen_field(seed: int, n: int, sigma_px: float = 4.0, std: float = 1.0) -> np.ndarray:
    """exp(i phi) with phi a smooth Gaussian-filtered noise screen of the given std (rad)."""
    return np.exp(1j * smooth_noise(seed, (n, n), sigma_px, std))


# ----------------------------------------------------------------------------- workloads

def cfg1_gaussian():
    """Single scalar Gaussian beam: waist 50 um, 64 x 64, 10 um, 700 nm, z = 0.1 m, pad 2."""
    n, d = 64, 10e-6
    f = gaussian_beam(n, n, d, d, 50e-6)
    return dict(field=to_c64(f[None]), dy=d, dx=d, lam=700e-9, z=0.1, pad=2.0)


def cfg2_diffractive(batch: int = 64, n: int = 512, layers: int = 5):
    """Diffractive network: binary inputs, 5 phase masks 5 cm apart, MSE target."""
    seed = BASE_SEED + 1
    inp = binary_pattern(sub_seed(seed, 0), batch, n)
    masks = uniform(sub_seed(seed, 1), (layers, n, n), 0.0, 2.0 * math.pi)
    target = 0.5 * uniform(sub_seed(seed, 2), (batch, n, n))
    return dict(field=to_c64(inp), phases=masks.astype(np.float32), target=target.astype(np.float32),
                d=8e-6, lam=532e-9, gap=0.05, detector=0.05, pad=2.0)


CFG3_SIZES = (250, 256, 500, 512, 768, 1000)


def cfg3_ragged(count: int = 200):
    """Uneven-size batch: sizes, spacings, wavelengths and distances drawn per field."""
    seed = BASE_SEED + 2
    u = uniform(sub_seed(seed, 0), (count, 4))
    fields = []
    for i in range(count):
        n = CFG3_SIZES[min(int(u[i, 0] * len(CFG3_SIZES)), len(CFG3_SIZES) - 1)]
        fields.append(dict(n=n, d=4e-6 + 8e-6 * u[i, 1], lam=450e-9 + 250e-9 * u[i, 2],
                           z=0.01 + 0.49 * u[i, 3], seed=sub_seed(seed, 1000 + i)))
    return fields


def cfg3_field(desc) -> np.ndarray:
    return to_c64(phase_screen_field(desc["seed"], desc["n"]))


def cfg4_objects(objects: int = 16, comps: int = 3, n: int = 1024, first: int = 0):
    """Polarised 4f workload inputs: amplitude objects per (object, component); objects
    ``first`` .. ``first + objects - 1`` of one seeded stream (a data-parallel shard)."""
    seed = BASE_SEED + 3
    amp = uniform(sub_seed(seed, 0), (objects, comps, n, n), start=first * comps * n * n)
    return amp


CFG4 = dict(objects=16, comps=3, wavelengths=8, n=1024, d=5e-6, f=0.2, lens_radius=2.56e-3,
            pupil_radius=1.0e-3, lam_lo=450e-9, lam_hi=700e-9, pad=2.0)


def cfg4_wavelengths(count: int = 8) -> np.ndarray:
    return np.linspace(CFG4["lam_lo"], CFG4["lam_hi"], count)


def cfg4_pupil_phase(n: int = 1024) -> np.ndarray:
    return uniform(sub_seed(BASE_SEED + 3, 1), (n, n), -math.pi, math.pi)


def cfg4_target(objects: int = 16, n: int = 1024, first: int = 0) -> np.ndarray:
    return 0.5 * uniform(sub_seed(BASE_SEED + 3, 2), (objects, n, n), start=first * n * n)


def cfg5a_coherence(n: int = 64):
    """Gaussian Schell-model coherence 64^4 with a trainable aperture mask phase."""
    seed = BASE_SEED + 4
    g = gaussian_schell(n, 10e-6, 200e-6, 50e-6)
    phase = uniform(sub_seed(seed, 0), (n, n), -math.pi, math.pi)
    target = uniform(sub_seed(seed, 1), (n, n))
    return dict(gamma=to_c64(g), phase=phase.astype(np.float32), target=target.astype(np.float32),
                d=10e-6, lam=633e-9, z=0.2, pad=2.0)


def cfg5b_field(n: int = 4096):
    """Single large coherent field: smooth phase screen, 5 um, 633 nm, z = 0.2 m, pad 2."""
    seed = BASE_SEED + 5
    return dict(field=to_c64(phase_screen_field(sub_seed(seed, 0), n)[None]), d=5e-6,
                lam=633e-9, z=0.2, pad=2.0)
