"""Degenerate cases of the propagation through the C ABI -- z = 0 is the identity, a propagation
by -z is the adjoint at z when no sample is evanescent, zero fields stay zero, empty requests are
refused (a batch of fields) or do nothing (a ragged list), on the on-chip path (64^2 at padding 2)
and on the three passes alike -- and the standalone detector intensity (Eq. 14) with its backward."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2411_18591_gb300 as T
    return T


def fields(seed, b, n):
    x = S.normal(seed, (b, n, n)) + 1j * S.normal(S.sub_seed(seed, 1), (b, n, n))
    return S.to_c64(x)


@pytest.mark.parametrize("n", [64, 256])
@pytest.mark.parametrize("method", ["as", "fresnel"])
def test_zero_distance_is_the_identity(T, rel, n, method):
    x0 = fields(401, 3, n)
    x = torch.from_numpy(x0).cuda()
    y = T.top_propagate(x, 5e-6, 5e-6, 633e-9, 0.0, 2.0, method)
    # the transforms round at float32; H(z = 0) = 1 / (Py Px) exactly
    assert rel(y.cpu().numpy(), x0) < 1e-6
    ref = O.propagate(x0, 5e-6, 5e-6, 633e-9, 0.0, 2.0, O.AS if method == "as" else O.FRESNEL_TF)
    assert np.allclose(ref, x0, atol=1e-12 * np.abs(x0).max())  # the oracle agrees exactly


@pytest.mark.parametrize("n", [64, 256])
def test_negative_distance_is_the_adjoint(T, rel, n):
    # 5 um spacing at 633 nm: no evanescent sample, so H(-z) = conj(H(z))
    x0 = fields(402, 2, n)
    x = torch.from_numpy(x0).cuda()
    back = T.top_propagate(x, 5e-6, 5e-6, 633e-9, -0.03, 2.0)
    adj = T.top_propagate_backward(x, 5e-6, 5e-6, 633e-9, 0.03, 2.0)
    assert rel(back.cpu().numpy(), adj.cpu().numpy()) < 1e-6
    ref = O.propagate(x0, 5e-6, 5e-6, 633e-9, -0.03, 2.0)
    assert rel(back.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("n", [64, 256])
def test_zero_field_stays_zero(T, n):
    x = torch.zeros((2, n, n), dtype=torch.complex64, device="cuda")
    y = T.top_propagate(x, 5e-6, 5e-6, 633e-9, 0.05, 2.0)
    g = T.top_propagate_backward(x, 5e-6, 5e-6, 633e-9, 0.05, 2.0)
    torch.cuda.synchronize()
    assert torch.count_nonzero(y).item() == 0 and torch.count_nonzero(g).item() == 0


def test_empty_requests(T):
    x = torch.zeros((0, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TopError, match="INVALID_ARG"):
        T.top_propagate(x, 5e-6, 5e-6, 633e-9, 0.05, 2.0)
    # a ragged call with no fields is a valid no-op at the C ABI
    from paper_2411_18591_gb300 import _lib
    from paper_2411_18591_gb300.binding import handle
    st = _lib.load().top_propagate_ragged(handle(), 0, None, None, None, None, None, 0, None)
    assert st == 0
    assert _lib.load().top_propagate_ragged(handle(), -1, None, None, None, None, None, 0, None) == 1


@pytest.mark.parametrize("group,weighted", [(1, False), (3, True), (6, False)])
def test_standalone_intensity_and_backward(T, rel, group, weighted):
    # Eq. 14 on fields already at the detector, and its backward, against the oracle
    b, n = 6, 96
    x0 = fields(403, b, n)
    w = np.linspace(0.5, 1.5, b).astype(np.float32) if weighted else None
    x = torch.from_numpy(x0).cuda()
    wt = torch.from_numpy(w).cuda() if weighted else None
    inten = T.top_intensity(x, group, wt)
    ref = O.intensity_sum(x0, group, None if w is None else w.astype(np.float64))
    assert rel(inten.cpu().numpy(), ref) < 1e-6
    gi0 = S.normal(404, (b // group, n, n)).astype(np.float32)
    g = T.top_intensity_backward(x, torch.from_numpy(gi0).cuda(), group, wt)
    wb = np.ones(b) if w is None else w.astype(np.float64)
    gref = np.stack([wb[i] * O.grad_intensity(x0[i], gi0[i // group].astype(np.float64)) for i in range(b)])
    assert rel(g.cpu().numpy(), gref) < 1e-6
    with pytest.raises(T.TopError, match="INVALID_ARG"):
        T.top_intensity(x, 4)  # 4 does not divide 6
