"""Jones-matrix modulation (§5.1) and field power on the GPU, through the C ABI."""
import math
import os

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


def golden(name):
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_polarizer_listing_powers(T):
    """The paper's polariser listing on its 1000^2 grid at 10 um: powers 1, 0.5, 0, 0.25."""
    n, d = 1000, 10e-6
    f = torch.zeros((3, n, n), dtype=torch.complex64, device="cuda")
    f[0] = 1.0
    f /= math.sqrt(float(T.top_field_power(f, d, d).sum()))
    elems = {"polarizer_45": T.linear_polarizer(math.pi / 4), "polarizer_90": T.linear_polarizer(math.pi / 2)}
    for seq, val in golden("polarizer_powers.txt"):
        g = f
        if seq != "none":
            for e in seq.split(","):
                g = T.top_jones(g, elems[e])
        assert float(T.top_field_power(g, d, d).sum()) == pytest.approx(float(val), abs=1e-6)


@pytest.mark.parametrize("inner", [1, 8])
def test_spatially_varying_jones_forward_and_backward(T, inner):
    ny, nx, k = 64, 48, 2
    b = 3 * inner * k
    x = S.to_c64(S.normal(131, (b, ny, nx)) + 1j * S.normal(132, (b, ny, nx)))
    J = S.to_c64(S.normal(133, (3, 3, ny, nx)) + 1j * S.normal(134, (3, 3, ny, nx)))
    g = S.to_c64(S.normal(135, (b, ny, nx)) + 1j * S.normal(136, (b, ny, nx)))
    out = T.top_jones(dev(x), dev(J), inner)
    gin, gj = T.top_jones_backward(dev(x), dev(g), dev(J), inner, want_grad_jones=True)

    def to_oracle(a):
        return a.reshape(k, 3, inner, ny, nx).transpose(0, 2, 1, 3, 4).astype(np.complex128)

    def from_oracle(a):
        return a.transpose(0, 2, 1, 3, 4).reshape(b, ny, nx)

    assert rel_l2(host(out), from_oracle(O.jones_modulate(to_oracle(x), J))) < 1e-6
    gi_ref, gj_ref = O.grad_jones(to_oracle(x), J, to_oracle(g))
    assert rel_l2(host(gin), from_oracle(gi_ref)) < 1e-6
    assert rel_l2(host(gj), gj_ref) < 1e-6


def test_polarised_field_through_a_waveplate_and_propagation(T):
    """x-polarised Gaussian, quarter-wave plate at 45 degrees, then each component propagated (AS)."""
    n, d, lam, z = 128, 5e-6, 633e-9, 5e-3
    x = O.coords(n, d)
    g0 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / (100e-6) ** 2)
    f = np.zeros((3, n, n), dtype=np.complex64)
    f[0] = g0
    qwp = T.waveplate(math.pi / 2, math.pi / 4)
    y = T.top_propagate(T.top_jones(dev(f), qwp), d, d, lam, z, 2.0)
    ref = O.propagate(O.jones_modulate(f.astype(np.complex128), O.waveplate(math.pi / 2, math.pi / 4)), d, d, lam, z, 2.0)
    assert rel_l2(host(y), ref) < 1e-5
