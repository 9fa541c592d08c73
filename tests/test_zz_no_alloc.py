"""top_propagate_noalloc: the handle-free propagation through the library's static scratch.

Its results must equal top_propagate's bit for bit (same tables, same kernels), on calls in a
row, and it must leave the device's free memory untouched once its first call has loaded the
scratch.
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


def field(seed, b, n):
    x = S.normal(seed, (b, n, n)) + 1j * S.normal(S.sub_seed(seed, 1), (b, n, n))
    return torch.from_numpy(S.to_c64(x)).cuda()


def test_noalloc_equals_propagate_on_calls_in_a_row(T):
    """Six 1024^2 fields with their own wavelengths: two fields and their two tables fit the scratch at
    a time (three chunks)."""
    lam = list(np.linspace(450e-9, 700e-9, 6))
    z = [0.05] * 6
    xs = [field(11, 6, 1024), field(12, 6, 1024)]
    refs = [T.top_propagate(x, 5e-6, 5e-6, lam, z, 2.0) for x in xs]
    out = torch.empty_like(xs[0])
    for x, ref in zip(xs, refs):
        T.top_propagate_noalloc(x, 5e-6, 5e-6, lam, z, 2.0, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_allocates_nothing(T):
    x = field(13, 4, 256)
    out = torch.empty_like(x)
    T.top_propagate_noalloc(x, 4e-6, 4e-6, 532e-9, 0.01, 2.0, out=out)  # loads the scratch
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    T.top_propagate_noalloc(x, 4e-6, 4e-6, 532e-9, 0.01, 2.0, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, T.top_propagate(x, 4e-6, 4e-6, 532e-9, 0.01, 2.0))


def test_noalloc_many_parameter_sets_in_place_fresnel(T):
    """30 wavelengths in one batch (more than one launch's parameter sets), 48^2 fields padded to
    128^2 (the field off the centre of the padded grid), in place."""
    lam = list(np.linspace(400e-9, 700e-9, 30))
    x = field(14, 30, 48)
    ref = T.top_propagate(x, 6e-6, 6e-6, lam, 2e-3, 2.667, "fresnel")
    y = x.clone()
    for _ in range(2):
        y.copy_(x)
        T.top_propagate_noalloc(y, 6e-6, 6e-6, lam, 2e-3, 2.667, "fresnel", out=y)
        torch.cuda.synchronize()
        assert torch.equal(y, ref)


def test_noalloc_rejects_a_field_beyond_the_scratch(T):
    x = torch.zeros((1, 2048, 2048), dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TopError, match="static scratch"):
        T.top_propagate_noalloc(x, 1e-6, 1e-6, 500e-9, 1e-3, 2.0, out=x)
