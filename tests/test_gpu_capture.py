"""Library calls captured in a CUDA graph: the no-alloc call and a ragged batch.

Once a call's tables and workspace exist (an uncaptured call on the same sizes), the call does no
host-to-device copy and no allocation: its per-call data (twiddles, per-field lists) reach the
device through kernel parameters. Captured and replayed, it must give the uncaptured results bit
for bit, on replays in a row.
"""
import numpy as np
import pytest
import torch

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


def field(seed, shape):
    x = S.normal(seed, shape) + 1j * S.normal(S.sub_seed(seed, 1), shape)
    return torch.from_numpy(S.to_c64(x)).cuda()


def test_noalloc_call_replays_from_a_graph(T):
    lam = list(np.linspace(450e-9, 700e-9, 5))
    x = field(41, (5, 256, 256))
    ref = T.top_propagate(x, 4e-6, 4e-6, lam, 0.02, 2.0)
    out = torch.empty_like(x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        T.top_propagate_noalloc(x, 4e-6, 4e-6, lam, 0.02, 2.0, out=out)  # looks up the scratch
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.top_propagate_noalloc(x, 4e-6, 4e-6, lam, 0.02, 2.0, out=out)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_ragged_call_replays_from_a_graph(T):
    sizes = [64, 128, 250, 64, 128, 250, 250]
    fields = [field(50 + i, (n, n)) for i, n in enumerate(sizes)]
    spacing = [4e-6 + 1e-6 * i for i in range(len(sizes))]
    lams = list(np.linspace(450e-9, 700e-9, len(sizes)))
    zs = [0.01 + 0.005 * i for i in range(len(sizes))]
    refs = [T.top_propagate(f[None], d, d, l, z, 2.0)[0] for f, d, l, z in zip(fields, spacing, lams, zs)]
    outs = [torch.empty_like(f) for f in fields]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        T.top_propagate_ragged(fields, spacing, lams, zs, 2.0, out=outs)  # tables and workspace
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        T.top_propagate_ragged(fields, spacing, lams, zs, 2.0, out=outs)
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            assert torch.equal(o, r)
