"""Direct Integration (Eq. 2-3 by FFT) and the Eq. 6 automatic method on the GPU, through the
C ABI, against the FP64 oracle (whose DI equals the brute-force Rayleigh-Sommerfeld sum)."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

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


def fields(seed, b, ny, nx):
    return S.to_c64(S.normal(seed, (b, ny, nx)) + 1j * S.normal(S.sub_seed(seed, 1), (b, ny, nx)))


@pytest.mark.parametrize("ny,nx,dy,dx,lam,z,pad", [
    (16, 32, 3e-6, 2e-6, 0.6e-6, 40e-6, 2.0),
    (64, 64, 5e-6, 5e-6, 0.5e-6, 0.02, 2.0),
    (128, 64, 4e-6, 6e-6, 0.633e-6, 0.05, 2.0),
    (96, 48, 5e-6, 5e-6, 0.5e-6, 0.01, 2.667),
    (250, 250, 8e-6, 8e-6, 0.7e-6, 0.3, 2.0),
])
def test_di_forward_and_adjoint(T, ny, nx, dy, dx, lam, z, pad):
    x = fields(101, 2, ny, nx)
    y = T.top_propagate(dev(x), dy, dx, lam, z, pad, "di")
    ref = O.propagate(x.astype(np.complex128), dy, dx, lam, z, pad, O.DI)
    assert rel_l2(host(y), ref) < TOL
    if ny * nx <= 1024:
        assert rel_l2(host(y)[0], O.rs_bruteforce(x[0].astype(np.complex128), dy, dx, lam, z)) < TOL
    g = T.top_propagate_backward(dev(x), dy, dx, lam, z, pad, "di")
    assert rel_l2(host(g), O.propagate_adjoint(x.astype(np.complex128), dy, dx, lam, z, pad, O.DI)) < TOL


def test_di_full_size_field(T):
    """A 1024^2 field at 2x padding (the DI table is a 2048^2 transform of the sampled kernel)."""
    n, d, lam, z = 1024, 5e-6, 0.532e-6, 0.2
    x = S.to_c64(S.phase_screen_field(S.sub_seed(S.BASE_SEED, 102), n))[None]
    y = T.top_propagate(dev(x), d, d, lam, z, 2.0, "di")
    ref = O.propagate(x.astype(np.complex128), d, d, lam, z, 2.0, O.DI)
    assert rel_l2(host(y), ref) < TOL


def test_auto_mixes_as_and_di_in_one_batch(T):
    ny, nx, dy, dx, lam = 64, 64, 5e-6, 5e-6, 0.5e-6
    zc = min(nx * dx * dx / lam, ny * dy * dy / lam)
    zs = [0.3 * zc, 0.9 * zc, 1.5 * zc, 6.0 * zc]
    x = fields(103, 4, ny, nx)
    y = T.top_propagate(dev(x), dy, dx, [lam] * 4, zs, 2.0, "auto")
    ref = np.concatenate([O.propagate(x[i:i + 1].astype(np.complex128), dy, dx, lam, zs[i], 2.0, O.AUTO) for i in range(4)])
    assert rel_l2(host(y), ref) < TOL
    # the fields beyond z_critical differ from AS, the ones below equal it
    a = O.propagate(x.astype(np.complex128), dy, dx, lam, zs, 2.0, O.AS)
    assert rel_l2(ref[:2], a[:2]) == 0.0 and rel_l2(ref[2:], a[2:]) > 1e-6


def test_di_refuses_short_padding(T):
    x = dev(fields(104, 1, 32, 32))
    with pytest.raises(T.TopError, match="DI needs padded sizes"):
        T.top_propagate(x, 5e-6, 5e-6, 5e-7, 1e-3, 1.0, "di")
