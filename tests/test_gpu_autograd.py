"""The torch.autograd wrapper: gradients through two masked propagations against the oracle."""
import math

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


def test_autograd_through_two_phase_masks(T):
    from paper_2411_18591_gb300 import autograd as A
    n, d, lams, z = 128, 6e-6, [500e-9, 640e-9], 3e-3
    x = S.to_c64(S.normal(151, (2, n, n)) + 1j * S.normal(152, (2, n, n)))
    p1 = S.uniform(153, (n, n), -math.pi, math.pi).astype(np.float32)
    p2 = S.uniform(154, (n, n), -math.pi, math.pi).astype(np.float32)
    w = S.uniform(155, (2, n, n)).astype(np.float32)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    t1 = torch.from_numpy(p1).cuda().requires_grad_(True)
    t2 = torch.from_numpy(p2).cuda().requires_grad_(True)
    y = A.propagate(A.propagate(xt, d, d, lams, z, 2.0, phase=t1), d, d, lams, 2 * z, 2.0, phase=t2)
    loss = (torch.from_numpy(w).cuda() * (y.real ** 2 + y.imag ** 2)).sum()
    gx, g1, g2 = torch.autograd.grad(loss, (xt, t1, t2))
    # oracle: L = sum w |y|^2, g_y = 2 w y, back through each mask and propagation
    m1, m2 = np.exp(1j * p1.astype(np.float64)), np.exp(1j * p2.astype(np.float64))
    x1 = O.propagate(x.astype(np.complex128) * m1, d, d, lams, z, 2.0)
    y2 = O.propagate(x1 * m2, d, d, lams, 2 * z, 2.0)
    gy = 2.0 * w * y2
    gb2 = O.propagate_adjoint(gy, d, d, lams, 2 * z, 2.0)
    g2_ref = O.grad_modulation(x1, m2, gb2)[2]
    g_x1 = gb2 * np.conj(m2)
    gb1 = O.propagate_adjoint(g_x1, d, d, lams, z, 2.0)
    g1_ref = O.grad_modulation(x.astype(np.complex128), m1, gb1)[2]
    gx_ref = gb1 * np.conj(m1)
    torch.cuda.synchronize()
    assert rel_l2(gx.cpu().numpy(), gx_ref) < 1e-5
    assert rel_l2(g1.cpu().numpy(), g1_ref) < 1e-5
    assert rel_l2(g2.cpu().numpy(), g2_ref) < 1e-5
