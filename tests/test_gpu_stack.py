"""Per-layer checkpoints of a deep mask stack (the diffractive network of config 2): the gradients
with a plane kept every second layer (or only the input) equal those with every plane kept, bit for
bit, and match the FP64 oracle."""
import numpy as np
import pytest
import torch

import synthetic as S

from conftest import rel_l2
from test_gpu_configs import diffractive_oracle

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


def test_checkpointed_mask_stack_gradients(T):
    from paper_2411_18591_gb300.stack import MaskStack
    c = S.cfg2_diffractive()
    b = 4
    x, phases, target = dev(c["field"][:b]), dev(c["phases"]), dev(c["target"][:b])
    K = phases.shape[0]
    stack = MaskStack(c["d"], c["lam"], [c["gap"]] * (K - 1) + [c["detector"]], c["pad"])
    results = {}
    for every in (1, 2, K):
        inten, st = stack.forward(x, phases, checkpoint_every=every)
        loss, g_i = T.top_mse_loss(inten, target)
        grads, _ = stack.backward(st, phases, g_i)
        torch.cuda.synchronize()
        results[every] = (inten.clone(), float(loss), grads.clone(), st.planes_held())
    for every in (2, K):
        assert torch.equal(results[every][0], results[1][0])
        assert results[every][1] == results[1][1]
        assert torch.equal(results[every][2], results[1][2])
    # planes held for the backward besides the input: 1 + 4 kept, 1 + 2 kept, 1
    assert [results[e][3] for e in (1, 2, K)] == [5, 3, 1]
    l_ref, g_ref, _ = diffractive_oracle(c["field"][:b], c["phases"], c["target"][:b], c)
    assert abs(results[2][1] - l_ref) / l_ref < 1e-5
    assert rel_l2(results[2][2].cpu().numpy().astype(np.float64), g_ref) < 1e-5
