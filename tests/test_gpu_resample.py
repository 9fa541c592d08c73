"""Resampling between grids of different spacing (§3) on the GPU, through the C ABI."""
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


@pytest.mark.parametrize("ny,nx,dy,dx,ny2,nx2,dy2,dx2", [
    (200, 300, 3e-6, 2e-6, 170, 230, 2.5e-6, 1.7e-6),
    (64, 64, 4e-6, 4e-6, 256, 256, 1e-6, 1e-6),
    (333, 210, 1e-6, 1.5e-6, 120, 90, 3e-6, 4.1e-6),
])
@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
def test_resample_and_transpose(T, ny, nx, dy, dx, ny2, nx2, dy2, dx2, mode):
    m = O.NEAREST if mode == "nearest" else O.BILINEAR
    x = S.to_c64(S.normal(141, (2, ny, nx)) + 1j * S.normal(142, (2, ny, nx)))
    g = S.to_c64(S.normal(143, (2, ny2, nx2)) + 1j * S.normal(144, (2, ny2, nx2)))
    out = T.top_resample(dev(x), dy, dx, ny2, nx2, dy2, dx2, mode)
    assert rel_l2(host(out), O.resample(x, dy, dx, ny2, nx2, dy2, dx2, m)) < 1e-6
    gi = T.top_resample_backward(dev(g), ny, nx, dy, dx, dy2, dx2, mode)
    assert rel_l2(host(gi), O.resample_adjoint(g, ny, nx, dy, dx, dy2, dx2, m)) < 1e-6


def test_propagation_onto_a_grid_of_another_spacing(T):
    """Propagate on the input spacing, then interpolate onto a coarser output grid (§3)."""
    n, d, lam, z = 256, 4e-6, 633e-9, 4e-3
    x = S.to_c64(S.phase_screen_field(S.sub_seed(S.BASE_SEED, 145), n))[None]
    y = T.top_resample(T.top_propagate(dev(x), d, d, lam, z, 2.0), d, d, 150, 150, 6e-6, 6e-6, "bilinear")
    ref = O.resample(O.propagate(x.astype(np.complex128), d, d, lam, z, 2.0), d, d, 150, 150, 6e-6, 6e-6, O.BILINEAR)
    assert rel_l2(host(y), ref) < 1e-5
