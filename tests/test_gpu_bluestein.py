"""Padded sizes without an FFT plan of their own (odd, prime, or with prime factors above 5):
Bluestein line transforms on the power-of-two engines, against the FP64 oracle.

Every comparison is element-wise rel-L2 over the whole output with the propagation
tolerance (1e-5): prime sizes (61, 127, 257), products with 7, 11, 13, a padded size
of 2042 (4096-point transforms), sizes below the smallest plan (16), one axis planned
and the other not, per-field wavelengths and distances, the Fresnel form, repeated
inputs, modulations before and after, the adjoint (backward) and its identity.
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
    (1021, 24, 2.0),   # 2042 = 2 1021: 4096-point transforms; 48 planned
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


def test_bluestein_limits_are_reported(T):
    x = dev(cfield(43, (1, 61, 61)))
    with pytest.raises(T.TopError, match="Direct Integration"):
        T.top_propagate(x, 2e-6, 2e-6, 600e-9, 1e-2, 2.0, "di")  # 122 = 2 61
    with pytest.raises(T.TopError, match="Bluestein"):
        T.top_propagate_intensity(x, 2e-6, 2e-6, 600e-9, 1e-3, 1.0)
    with pytest.raises(T.TopError, match="2048"):
        T.top_propagate(dev(cfield(45, (1, 16, 1500))), 2e-6, 2e-6, 600e-9, 1e-3, 2.0)  # 3000 = 8 3 125
