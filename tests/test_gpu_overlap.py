"""Overlap integral and loss of Eq. 7 fused into the last propagation pass (GPU, C ABI), and a
beam-splitter training step in the shape of the paper's phase-modulator example."""
import math

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


def fields(seed, shape):
    return S.to_c64(S.normal(seed, shape) + 1j * S.normal(S.sub_seed(seed, 1), shape))


@pytest.mark.parametrize("ny,nx,pad,shared", [(256, 256, 2.0, True), (96, 48, 2.667, False)])
def test_overlap_and_power(T, ny, nx, pad, shared):
    d, z = 6e-6, 3e-3
    lams = [480e-9, 560e-9, 640e-9]
    s = 1.0 / (math.sqrt(ny * nx) * d)
    x = fields(121, (3, ny, nx)) * s
    tgt = fields(122, (ny, nx) if shared else (3, ny, nx)) * s
    phi = S.uniform(123, (ny, nx), -np.pi, np.pi).astype(np.float32)
    pre = T.Modulation(phase=dev(phi))
    post = T.Modulation(focal_length=0.05, radius=0.4 * nx * d)
    ov, pw, psi = T.top_propagate_overlap(dev(x), dev(tgt), d, d, lams, z, pad, pre=pre, post=post, keep_field=True)
    lm = np.stack([O.circ(ny, nx, d, d, 0.4 * nx * d) * O.lens(ny, nx, d, d, l, 0.05) for l in lams])
    ref = O.propagate(x.astype(np.complex128) * np.exp(1j * phi.astype(np.float64)), d, d, lams, z, pad) * lm
    assert rel_l2(host(psi), ref) < TOL
    assert torch.equal(psi, T.top_propagate(dev(x), d, d, lams, z, pad, pre=pre, post=post))
    o_ref = O.overlap(ref, tgt, d, d)
    assert np.max(np.abs(host(ov) - o_ref)) < TOL * np.max(np.abs(o_ref))
    assert np.max(np.abs(host(pw) - O.power(ref, d, d))) < TOL * np.max(O.power(ref, d, d))
    # without keeping the field
    ov2, _, none = T.top_propagate_overlap(dev(x), dev(tgt), d, d, lams, z, pad, pre=pre, post=post)
    assert none is None and torch.equal(ov2, ov)


def gaussian(n, d, w, x0=0.0, y0=0.0):
    x = O.coords(n, d)[None, :]
    y = O.coords(n, d)[:, None]
    g = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (w * w))
    return g / math.sqrt(O.power(g, d, d)[0])


def test_beam_splitter_training_step(T):
    """A normalised Gaussian through three trainable phase masks (5 cm apart) to a target of four
    normalised Gaussian spots; loss of Eq. 7 and the gradients of all three masks, batch of 2
    wavelengths, against the oracle."""
    n, d, gap = 128, 8e-6, 0.05
    lams = [532e-9, 633e-9]
    w = 80e-6
    x = np.stack([gaussian(n, d, w)] * 2).astype(np.complex64)
    a = 0.2e-3
    tgt = sum(gaussian(n, d, 40e-6, sx * a, sy * a) for sx in (-1, 1) for sy in (-1, 1))
    tgt = (tgt / math.sqrt(O.power(tgt, d, d)[0])).astype(np.complex64)
    phases = S.uniform(124, (3, n, n), 0, 2 * np.pi).astype(np.float32)
    # forward on the GPU, keeping each mask's input
    ins = [dev(x)]
    cur = ins[0]
    for l in range(2):
        cur = T.top_propagate(cur, d, d, lams, gap, 2.0, pre=T.Modulation(phase=dev(phases[l])))
        ins.append(cur)
    ov, _, _ = T.top_propagate_overlap(cur, dev(tgt), d, d, lams, gap, 2.0, pre=T.Modulation(phase=dev(phases[2])))
    loss, g = T.top_overlap_loss(ov, dev(tgt), 2, n, n, d, d)
    grads = torch.zeros((3, n, n), dtype=torch.float32, device="cuda")
    for l in (2, 1, 0):
        g = T.top_propagate_backward(g, d, d, lams, gap, 2.0, pre=T.Modulation(phase=dev(phases[l])), saved_in=ins[l],
                                     want_grad_in=l > 0, grad_phase=grads[l])
    # the oracle
    cur = x.astype(np.complex128)
    ins_o = []
    for l in range(3):
        ins_o.append(cur)
        cur = O.propagate(cur * np.exp(1j * phases[l].astype(np.float64)), d, d, lams, gap, 2.0)
    l_ref, g_ref = O.overlap_loss(cur, tgt.astype(np.complex128), d, d)
    assert abs(float(loss) - l_ref) < 1e-5
    go = g_ref
    for l in (2, 1, 0):
        m = np.exp(1j * phases[l].astype(np.float64))
        gy = O.propagate_adjoint(go, d, d, lams, gap, 2.0)
        assert rel_l2(host(grads[l]), O.grad_modulation(ins_o[l], m, gy)[2]) < TOL
        go = gy * np.conj(m)
