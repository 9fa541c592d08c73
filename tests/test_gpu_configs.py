"""Full-size parity of the five workloads against the FP64 oracle (GPU, through the C ABI).

Where the oracle cannot process a whole batch in seconds, the GPU runs the full batch
in the launch configuration the bench uses and a seeded sample of its fields is
compared one by one (every field is independent, so a sampled field's result is the
same computation the oracle does on its own).
"""
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


# ----------------------------------------------------------------------------- config 2

def diffractive_gpu(T, x, phases, c):
    """Forward through 5 phase masks 5 cm apart to the detector, MSE, gradients of all masks."""
    d, lam, gap = c["d"], c["lam"], c["gap"]
    ins = [x]
    cur = x
    L = phases.shape[0]
    for l in range(L - 1):
        cur = T.top_propagate(cur, d, d, lam, gap, c["pad"], pre=T.Modulation(phase=phases[l]))
        ins.append(cur)
    inten, psi = T.top_propagate_intensity(cur, d, d, lam, c["detector"], c["pad"],
                                           pre=T.Modulation(phase=phases[L - 1]), keep_field=True)
    return inten, psi, ins


def diffractive_grads(T, psi, ins, phases, g_i, c):
    d, lam, gap = c["d"], c["lam"], c["gap"]
    L = phases.shape[0]
    grads = torch.zeros_like(phases)
    g = T.top_propagate_intensity_backward(psi, g_i, d, d, lam, c["detector"], c["pad"],
                                           pre=T.Modulation(phase=phases[L - 1]), saved_in=ins[L - 1],
                                           grad_phase=grads[L - 1])
    for l in range(L - 2, -1, -1):
        g = T.top_propagate_backward(g, d, d, lam, gap, c["pad"], pre=T.Modulation(phase=phases[l]),
                                     saved_in=ins[l], want_grad_in=l > 0, grad_phase=grads[l])
    return grads


def diffractive_oracle(x, phases, target, c):
    d, lam, gap = c["d"], c["lam"], c["gap"]
    L = phases.shape[0]
    ins, cur = [], x.astype(np.complex128)
    for l in range(L):
        ins.append(cur)
        z = gap if l < L - 1 else c["detector"]
        cur = O.propagate(cur * np.exp(1j * phases[l].astype(np.float64)), d, d, lam, z, c["pad"])
    loss, g_i = O.mse_loss(O.intensity(cur), target)
    g = O.grad_intensity(cur, g_i)
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        z = gap if l < L - 1 else c["detector"]
        gy = O.propagate_adjoint(g, d, d, lam, z, c["pad"])
        m = np.exp(1j * phases[l].astype(np.float64))
        grads[l] = np.imag(gy * np.conj(m * ins[l])).sum(axis=0)
        g = gy * np.conj(m)
    return loss, np.stack(grads), cur


def test_config2_diffractive_network_gradients(T):
    """5 trainable 512^2 phase masks, 8 um, 532 nm, 5 cm apart, MSE on intensity (batch 8 of the 64)."""
    c = S.cfg2_diffractive()
    b = 8
    x, phases, target = c["field"][:b], c["phases"], c["target"][:b]
    inten, psi, ins = diffractive_gpu(T, dev(x), dev(phases), c)
    loss, g_i = T.top_mse_loss(inten, dev(target))
    grads = diffractive_grads(T, psi, ins, dev(phases), g_i, c)
    l_ref, g_ref, out_ref = diffractive_oracle(x, phases, target, c)
    assert rel_l2(host(psi), out_ref) < TOL
    assert abs(float(loss) - l_ref) / l_ref < 1e-5
    assert rel_l2(host(grads), g_ref) < TOL


def test_config2_full_batch_forward_sampled(T):
    c = S.cfg2_diffractive()
    inten, psi, _ = diffractive_gpu(T, dev(c["field"]), dev(c["phases"]), c)
    out = host(psi)
    for i in (0, 37, 63):
        _, _, ref = diffractive_oracle(c["field"][i:i + 1], c["phases"], c["target"][i:i + 1], c)
        assert rel_l2(out[i:i + 1], ref) < TOL


# ----------------------------------------------------------------------------- config 3

def test_config3_ragged_batch_sampled(T):
    """200 fields of mixed sizes, spacings, wavelengths and distances; phase-screen inputs;
    forward and the gradient w.r.t. each field's input phase, two fields of every size."""
    fields = S.cfg3_ragged()
    sizes = sorted({f["n"] for f in fields})
    checked = 0
    for n in sizes:
        idx = [i for i, f in enumerate(fields) if f["n"] == n]
        for i in idx[:2]:
            f = fields[i]
            phi = S.smooth_noise(f["seed"], (n, n), 4.0, 1.0).astype(np.float32)
            ones = np.ones((1, n, n), np.complex64)
            out = T.top_propagate(dev(ones), f["d"], f["d"], f["lam"], f["z"], 2.0,
                                  pre=T.Modulation(phase=dev(phi[None])))
            ref = O.propagate(np.exp(1j * phi.astype(np.float64))[None], f["d"], f["d"], f["lam"], f["z"], 2.0)
            assert rel_l2(host(out), ref) < TOL
            tgt = S.uniform(S.sub_seed(f["seed"], 1), (1, n, n))
            g_out = (O.intensity(ref) - tgt)  # any fixed upstream gradient of the field intensity
            g_psi = O.grad_intensity(ref, g_out)
            gp = torch.zeros((1, n, n), dtype=torch.float32, device="cuda")
            T.top_propagate_backward(dev(g_psi.astype(np.complex64)), f["d"], f["d"], f["lam"], f["z"], 2.0,
                                     pre=T.Modulation(phase=dev(phi[None])), saved_in=dev(ones),
                                     want_grad_in=False, grad_phase=gp)
            gy = O.propagate_adjoint(g_psi.astype(np.complex64).astype(np.complex128), f["d"], f["d"], f["lam"],
                                     f["z"], 2.0)
            g_ref = np.imag(gy * np.conj(np.exp(1j * phi.astype(np.float64))[None]))
            assert rel_l2(host(gp), g_ref) < TOL
            checked += 1
    assert checked == 2 * len(sizes)


# ----------------------------------------------------------------------------- config 4

def fourf_setup(T, objects, comps, nl):
    from paper_2411_18591_gb300.fourf import FourF
    c = S.CFG4
    lams = S.cfg4_wavelengths(c["wavelengths"])[:nl] if nl < c["wavelengths"] else S.cfg4_wavelengths(nl)
    sysm = FourF(n=c["n"], d=c["d"], f=c["f"], lens_radius=c["lens_radius"], pupil_radius=c["pupil_radius"],
                 objects=objects, comps=comps, wavelengths=tuple(lams), pad=c["pad"])
    obj = S.cfg4_objects(objects, comps, c["n"]).reshape(-1, c["n"], c["n"]).astype(np.complex64)
    phase = S.cfg4_pupil_phase(c["n"]).astype(np.float32)
    target = S.cfg4_target(objects, c["n"]).astype(np.float32)
    return sysm, obj, phase, target, lams


def test_config4_fourf_loss_and_pupil_gradient(T):
    """The bench's 4f step on 1 object x 3 components x 2 wavelengths of 1024^2 (2048^2 FFTs)."""
    sysm, obj, phase, target, lams = fourf_setup(T, 1, 3, 2)
    gp = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    loss, inten = sysm.step(dev(obj), dev(phase), dev(target), gp)
    c = S.CFG4
    obj_f = np.repeat(obj, len(lams), axis=0)
    lam_f = np.tile(lams, 3)
    l_ref, g_ref, i_ref = O.fourf_loss_and_grad(obj_f.astype(np.complex128), lam_f, c["d"], c["f"],
                                                c["lens_radius"], c["pupil_radius"], phase.astype(np.float64),
                                                sysm.group, target, c["pad"])
    assert rel_l2(host(inten), i_ref) < TOL
    assert abs(float(loss) - l_ref) / l_ref < 1e-5
    assert rel_l2(host(gp), g_ref) < TOL


def test_config4_full_batch_intensity_sampled(T):
    """All 384 fields in the bench's launch configuration; object 0's summed intensity is checked."""
    sysm, obj, phase, target, lams = fourf_setup(T, 16, 3, 8)
    gp = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    loss, inten = sysm.step(dev(obj), dev(phase), dev(target), gp)
    c = S.CFG4
    obj_f = np.repeat(obj[:3], len(lams), axis=0).astype(np.complex128)
    lam_f = np.tile(lams, 3)
    p4, _ = O.fourf_forward(obj_f, lam_f, c["d"], c["f"], c["lens_radius"], c["pupil_radius"],
                            phase.astype(np.float64), c["pad"])
    assert rel_l2(host(inten)[0], O.intensity_sum(p4, sysm.group)[0]) < TOL
    assert np.isfinite(float(loss)) and np.isfinite(host(gp)).all()


def test_config4_full_batch_gradient_is_the_mean_over_objects(T):
    """The pupil gradient of the full 384-field step (the bench's launch) against the mean of the 16
    single-object steps' gradients (the MSE averages over objects, so the batch gradient is their
    mean: a property that holds at any size), and the loss against the mean of their losses.
    Object 0's step itself is the oracle-checked case above at two wavelengths; here the full eight."""
    sysm, obj, phase, target, lams = fourf_setup(T, 16, 3, 8)
    gp = torch.empty((1024, 1024), dtype=torch.float32, device="cuda")
    loss, _ = sysm.step(dev(obj), dev(phase), dev(target), gp)
    one, _, _, _, _ = fourf_setup(T, 1, 3, 8)
    acc = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")
    losses = []
    g1 = torch.empty_like(gp)
    for o in range(16):
        l1, _ = one.step(dev(obj[3 * o:3 * o + 3]), dev(phase), dev(target[o:o + 1]), g1)
        acc += g1.double()
        losses.append(float(l1))
    mean = acc / 16
    assert rel_l2(host(gp).astype(np.float64), host(mean)) < TOL
    assert abs(float(loss) - np.mean(losses)) / np.mean(losses) < 1e-6


# ----------------------------------------------------------------------------- config 5

def test_config5a_coherence_full_size(T):
    """GSM mutual coherence on a 64^4 grid through a trainable 64^2 mask, z = 0.2 m, fwd + bwd."""
    c = S.cfg5a_coherence()
    g0 = c["gamma"]
    d, lam, z = c["d"], c["lam"], c["z"]
    mask = T.Modulation(phase=dev(c["phase"]))
    gz = T.top_propagate_coherence(dev(g0), d, d, lam, z, c["pad"], mask=mask)
    inten = T.top_coherence_intensity(gz)
    m = np.exp(1j * c["phase"].astype(np.float64))
    gm = O.modulate_coherence(g0.astype(np.complex128), m)
    ref = O.propagate_coherence(gm, d, d, lam, z, c["pad"])
    assert rel_l2(host(gz), ref) < TOL
    i_ref = O.coherence_diag(ref)
    assert rel_l2(host(inten), i_ref) < TOL
    _, g_i = O.mse_loss(i_ref, c["target"])
    G = T.top_coherence_intensity_backward(dev(g_i.astype(np.float32)), gz)
    gp = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    T.top_propagate_coherence_backward(G, d, d, lam, z, c["pad"], mask=mask, saved_in=dev(g0), want_grad_in=False,
                                       grad_phase=gp)
    n = 64
    gd = np.zeros((n * n, n * n), np.complex128)
    gd[np.arange(n * n), np.arange(n * n)] = g_i.reshape(-1).astype(np.float32)
    gmg = O.propagate_coherence(gd.reshape(n, n, n, n), d, d, lam, z, c["pad"], adjoint=True)
    g_m = O.grad_modulate_coherence(g0.astype(np.complex128), m, gmg)
    assert rel_l2(host(gp), np.imag(np.conj(m) * g_m)) < TOL


@pytest.mark.slow
def test_config5b_large_field(T):
    """A single 4096^2 coherent field with 2x padding (8192^2 FFTs), forward and backward; tolerance 5e-5."""
    c = S.cfg5b_field()
    x = c["field"]
    d, lam, z = c["d"], c["lam"], c["z"]
    y = T.top_propagate(dev(x), d, d, lam, z, c["pad"])
    ref = O.propagate(x.astype(np.complex128), d, d, lam, z, c["pad"])
    assert rel_l2(host(y), ref) < 5e-5
    del ref
    g = T.top_propagate_backward(y, d, d, lam, z, c["pad"])
    back = O.propagate_adjoint(host(y).astype(np.complex128), d, d, lam, z, c["pad"])
    assert rel_l2(host(g), back) < 5e-5
