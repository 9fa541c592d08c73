"""Failure handling without a GPU fault: a workspace limit below one field's need is reported as
TOP_ERR_OOM before any launch, and calls write nothing outside their output buffers."""
import ctypes as C

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


def test_workspace_limit_gives_oom_before_any_launch(T):
    from paper_2411_18591_gb300 import _lib
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.top_create(C.byref(h), torch.cuda.current_device()) == 0
    try:
        assert lib.top_set_workspace_limit(h, 4096) == 1  # below the 1 MiB floor: TOP_ERR_INVALID_ARG
        assert lib.top_set_workspace_limit(h, 1 << 20) == 0
        assert lib.top_profile_enable(h, 1) == 0
        x = field(61, (1, 1024, 1024))  # one field at 2x padding needs 16 MiB of workspace
        out = torch.full_like(x, complex(7.0, -3.0))
        g = _lib.TopGrid(1, 1024, 1024, 5e-6, 5e-6, 2.0, _lib.TOP_AS, 0)
        lam, z = _lib.doubles([532e-9]), _lib.doubles([0.01])
        st = lib.top_propagate(h, C.byref(g), x.data_ptr(), out.data_ptr(), lam, z, 1, None, None,
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 3  # TOP_ERR_OOM
        assert b"workspace" in lib.top_last_error()
        kinds = (C.c_char_p * 8)()
        ms = (C.c_double * 8)()
        cnt = (C.c_int64 * 8)()
        n = C.c_int()
        assert lib.top_profile_read(h, 8, kinds, ms, cnt, C.byref(n)) == 0
        assert sum(cnt[i] for i in range(n.value)) == 0  # nothing was launched
        torch.cuda.synchronize()
        assert torch.all(out == complex(7.0, -3.0))
    finally:
        lib.top_destroy(h)


@pytest.mark.parametrize("n", [64, 250, 1024])
def test_calls_write_only_their_outputs(T, n):
    """Propagation, its backward and the grouped intensity, through the C ABI, into buffers with
    guard regions on both sides."""
    from paper_2411_18591_gb300 import _lib, binding
    lib = _lib.load()
    b, gs = 3, 4096  # fields, guard samples on each side
    x = field(70 + n, (b, n, n))
    plane = b * n * n
    h = binding.handle(x.device)
    g = _lib.TopGrid(b, n, n, 5e-6, 5e-6, 2.0, _lib.TOP_AS, 0)
    lam, z = _lib.doubles([600e-9]), _lib.doubles([0.02])
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    guard = complex(1.5, 2.5)
    buf = torch.full((plane + 2 * gs,), guard, dtype=torch.complex64, device="cuda")
    out = buf[gs:gs + plane]
    _lib.check(lib.top_propagate(h, C.byref(g), x.data_ptr(), out.data_ptr(), lam, z, 1, None, None, st))
    _lib.check(lib.top_propagate_backward(h, C.byref(g), x.data_ptr(), out.data_ptr(), lam, z, 1, None, None, None,
                                          st))
    fbuf = torch.full((n * n + 2 * gs,), 9.0, dtype=torch.float32, device="cuda")
    inten = fbuf[gs:gs + n * n]
    _lib.check(lib.top_propagate_intensity(h, C.byref(g), x.data_ptr(), None, inten.data_ptr(), b, None, lam, z, 1,
                                           None, None, st))
    torch.cuda.synchronize()
    assert torch.all(buf[:gs] == guard) and torch.all(buf[gs + plane:] == guard)
    assert torch.all(fbuf[:gs] == 9.0) and torch.all(fbuf[gs + n * n:] == 9.0)
    ref = T.top_propagate_backward(x, 5e-6, 5e-6, 600e-9, 0.02, 2.0)
    assert torch.equal(out.view(b, n, n), ref)
    assert torch.all(torch.isfinite(inten))
