"""top_propagate_ragged: fields of different sizes, spacings, wavelengths and distances in one
call (GPU, through the C ABI). Checked against the FP64 oracle and, bit for bit, against the
same field propagated on its own."""
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_config3_whole_batch_in_one_call(T):
    """All 200 config-3 phase-screen fields (six sizes, 4-12 um, 450-700 nm, 1-50 cm), forward and
    backward in one call each; two fields of every size against the oracle, every field against
    its own top_propagate call."""
    descs = S.cfg3_ragged()
    xs = [torch.from_numpy(S.cfg3_field(d)).cuda() for d in descs]
    ds = [d["d"] for d in descs]
    lams = [d["lam"] for d in descs]
    zs = [d["z"] for d in descs]
    ys = T.top_propagate_ragged(xs, ds, lams, zs, 2.0)
    gs = T.top_propagate_ragged(ys, ds, lams, zs, 2.0, backward=True)
    seen = {}
    for i, d in enumerate(descs):
        single = T.top_propagate(xs[i], d["d"], d["d"], d["lam"], d["z"], 2.0)
        assert torch.equal(ys[i], single[0])
        if seen.get(d["n"], 0) < 2:
            seen[d["n"]] = seen.get(d["n"], 0) + 1
            x = S.cfg3_field(d).astype(np.complex128)
            ref = O.propagate(x, d["d"], d["d"], d["lam"], d["z"], 2.0)[0]
            assert rel_l2(host(ys[i]), ref) < 1e-5
            back = O.propagate_adjoint(host(ys[i]).astype(np.complex128), d["d"], d["d"], d["lam"], d["z"], 2.0)[0]
            assert rel_l2(host(gs[i]), back) < 1e-5
    assert len(seen) == len(S.CFG3_SIZES)


def test_ragged_mixed_methods_in_place_and_empty(T):
    descs = [(64, 64, 5e-6, 2.0, "as"), (48, 96, (4e-6, 6e-6), 2.667, "fresnel"), (64, 64, 8e-6, 2.0, "fresnel"),
             (48, 96, (4e-6, 6e-6), 2.667, "as")]
    xs = [torch.from_numpy(S.to_c64(S.normal(60 + i, (ny, nx)) + 1j * S.normal(70 + i, (ny, nx)))).cuda()
          for i, (ny, nx, *_) in enumerate(descs)]
    refs = []
    for i, (ny, nx, d, pad, m) in enumerate(descs):
        dy, dx = (d, d) if isinstance(d, float) else d
        refs.append(O.propagate(host(xs[i]).astype(np.complex128), dy, dx, 500e-9 + 50e-9 * i, 2e-3, pad,
                                O.AS if m == "as" else O.FRESNEL_TF)[0])
    # one call per (method, pad): the grid of every field carries both, so a call may mix them too
    by_method = {}
    for i, desc in enumerate(descs):
        by_method.setdefault(desc[4], []).append(i)
    for m, idx in by_method.items():
        pads = {descs[i][3] for i in idx}
        for pad in pads:
            sel = [i for i in idx if descs[i][3] == pad]
            fl = [xs[i] for i in sel]
            T.top_propagate_ragged(fl, [descs[i][2] for i in sel], [500e-9 + 50e-9 * i for i in sel], [2e-3] * len(sel),
                                   pad, m, out=fl)  # in place
    for i in range(len(descs)):
        assert rel_l2(host(xs[i]), refs[i]) < 1e-5


def test_ragged_call_mixing_methods_and_pads(T):
    """One call with two geometries and both methods: each field is grouped with its own kind."""
    specs = [(64, 64, 5e-6, 2.0, "as"), (48, 96, 4e-6, 2.667, "fresnel"), (64, 64, 8e-6, 2.0, "fresnel")]
    xs = [torch.from_numpy(S.to_c64(S.normal(80 + i, (ny, nx)) + 1j * S.normal(90 + i, (ny, nx)))).cuda()
          for i, (ny, nx, *_) in enumerate(specs)]
    import ctypes as C
    from paper_2411_18591_gb300 import _lib, binding as B
    n = len(specs)
    grids = (_lib.TopGrid * n)()
    outs = [torch.empty_like(x) for x in xs]
    ins = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    ous = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    for i, (ny, nx, d, pad, m) in enumerate(specs):
        grids[i] = B.make_grid(1, ny, nx, d, d, pad, m)
    lams = [520e-9, 610e-9, 700e-9]
    _lib.check(_lib.load().top_propagate_ragged(B.handle(), n, grids, ins, ous, _lib.doubles(lams), _lib.doubles([3e-3] * n),
                                                0, None))
    _lib.check(_lib.load().top_propagate_ragged(B.handle(), 0, None, None, None, None, None, 0, None))
    for i, (ny, nx, d, pad, m) in enumerate(specs):
        ref = O.propagate(host(xs[i]).astype(np.complex128), d, d, lams[i], 3e-3, pad, O.AS if m == "as" else O.FRESNEL_TF)
        assert rel_l2(host(outs[i]), ref[0]) < 1e-5
