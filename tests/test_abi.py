"""Host-side checks of the C-ABI library (no GPU needed).

The library must load and export every function that include/top.h declares;
host-only calls (plan query, validation, z_critical, status strings) must work
without a device; and nothing here launches a kernel.
"""
import ctypes as C
import math
import os
import re
import subprocess

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "top.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2411_18591_gb300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(top_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_calls():
    names = declared_functions()
    for required in ["top_propagate", "top_propagate_backward", "top_modulate", "top_modulate_backward",
                     "top_propagate_coherence", "top_propagate_coherence_backward", "top_propagate_intensity",
                     "top_propagate_intensity_backward", "top_zcritical", "top_create", "top_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    cdll = lib.load()
    names = declared_functions()
    missing = [n for n in names if not hasattr(cdll, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (top_[a-z_0-9]+)\b", out))
    assert set(names) <= exported
    # the ctypes signature table covers exactly the declared calls
    assert set(lib.SIGNATURES) == set(names)


def test_version_and_status_strings(lib):
    cdll = lib.load()
    assert cdll.top_version() == 1
    assert cdll.top_status_string(0) == b"TOP_OK"
    assert cdll.top_status_string(2) == b"TOP_ERR_UNSUPPORTED"


def test_zcritical_matches_eq6(lib):
    cdll = lib.load()
    for L, dx, lam in [(2.56e-3, 10e-6, 700e-9), (5.12e-3, 5e-6, 450e-9)]:
        assert cdll.top_zcritical(L, dx, lam) == pytest.approx(O.z_critical(L, dx, lam), rel=1e-15)


def plan(lib, **kw):
    g = lib.TopGrid(kw.get("batch", 1), kw.get("ny", 64), kw.get("nx", 64), kw.get("dy", 1e-5), kw.get("dx", 1e-5),
                    kw.get("pad", 2.0), kw.get("method", 0), kw.get("input_repeat", 0))
    py, px, ws = C.c_int64(), C.c_int64(), C.c_uint64()
    st = lib.load().top_plan_query(C.byref(g), C.byref(py), C.byref(px), C.byref(ws))
    return st, py.value, px.value, ws.value


@pytest.mark.parametrize("ny,nx,pad,py,px", [(64, 64, 2.0, 128, 128), (1024, 1024, 2.0, 2048, 2048),
                                             (250, 500, 2.0, 500, 1000), (768, 1000, 2.0, 1536, 2000),
                                             (24, 48, 1.34, 32, 64), (4096, 4096, 2.0, 8192, 8192)])
def test_plan_query_padded_sizes(lib, ny, nx, pad, py, px):
    st, gy, gx, ws = plan(lib, ny=ny, nx=nx, pad=pad)
    assert st == 0
    assert (gy, gx) == (py, px) == (O.padded_size(ny, pad), O.padded_size(nx, pad))
    assert ws == px * ny * 8


@pytest.mark.parametrize("ny,nx,pad,py,px", [(61, 61, 1.0, 61, 61), (20, 20, 1.7, 34, 34), (1021, 24, 2.0, 2042, 48)])
def test_plan_query_bluestein_sizes(lib, ny, nx, pad, py, px):
    """Padded sizes without a plan of their own go through Bluestein transforms (two field-sized
    buffers per field)."""
    st, gy, gx, ws = plan(lib, ny=ny, nx=nx, pad=pad)
    assert st == 0
    assert (gy, gx) == (py, px)
    assert ws == 2 * px * ny * 8


@pytest.mark.parametrize("kw,status", [
    (dict(batch=0), 1), (dict(ny=0), 1), (dict(dx=0.0), 1), (dict(dy=-1e-6), 1), (dict(dx=float("nan")), 1),
    (dict(pad=0.5), 1), (dict(pad=float("inf")), 1), (dict(method=7), 1), (dict(batch=6, input_repeat=4), 1),
    (dict(ny=16, nx=2500, pad=2.0), 2), (dict(ny=4097, nx=16, pad=1.0), 2),
])
def test_plan_query_rejects(lib, kw, status):
    st, *_ = plan(lib, **kw)
    assert st == status
    assert len(lib.load().top_last_error()) > 0


def test_null_handle_is_rejected_before_any_launch(lib):
    cdll = lib.load()
    g = lib.TopGrid(1, 64, 64, 1e-5, 1e-5, 2.0, 0, 0)
    lam = lib.doubles([5e-7])
    assert cdll.top_propagate(None, C.byref(g), None, None, lam, lam, 1, None, None, None) == 1
    assert cdll.top_propagate_backward(None, C.byref(g), None, None, lam, lam, 1, None, None, None, None) == 1
    assert cdll.top_modulate(None, C.byref(g), None, None, None, lam, 1, None) == 1
    assert cdll.top_propagate_coherence(None, C.byref(g), None, None, lam, lam, None, None) == 1
    assert cdll.top_mse_loss(None, 1, None, None, None, None, None) == 1
    assert cdll.top_destroy(None) == 1
    assert b"handle" in cdll.top_last_error()


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="only meaningful on a host without a GPU")
def test_create_without_gpu_reports_cuda_error(lib):
    cdll = lib.load()
    h = C.c_void_p()
    st = cdll.top_create(C.byref(h), 0)
    assert st in (1, 4)  # no device: TOP_ERR_CUDA (or INVALID_ARG when the runtime reports zero devices)
    assert h.value is None


def _jones(lib, name, *args):
    import numpy as np
    out = (C.c_double * 18)()
    st = getattr(lib.load(), name)(*args, out)
    v = np.frombuffer(out, dtype=np.float64)
    return st, (v[0::2] + 1j * v[1::2]).reshape(3, 3)


@pytest.mark.parametrize("theta", [0.0, 0.3, math.pi / 4, math.pi / 2, -1.1])
def test_jones_constructors_match_the_oracle(lib, theta):
    """The library's Jones matrices (host-only calls) against the oracle's matrix products (§5.1)."""
    import numpy as np
    st, m = _jones(lib, "top_jones_linear_polarizer", C.c_double(theta))
    assert st == 0 and np.abs(m - O.linear_polarizer(theta)).max() < 1e-15
    for ret in (math.pi / 2, math.pi, 0.7):
        st, m = _jones(lib, "top_jones_waveplate", C.c_double(ret), C.c_double(theta))
        assert st == 0 and np.abs(m - O.waveplate(ret, theta)).max() < 1e-15
    for hand in (1, -1):
        st, m = _jones(lib, "top_jones_circular_polarizer", hand)
        assert st == 0 and np.abs(m - O.circular_polarizer(hand)).max() < 1e-15


def test_jones_constructors_reject_bad_arguments(lib):
    cdll = lib.load()
    assert _jones(lib, "top_jones_circular_polarizer", 0)[0] == 1
    assert _jones(lib, "top_jones_linear_polarizer", C.c_double(float("nan")))[0] == 1
    assert cdll.top_jones_waveplate(C.c_double(1.0), C.c_double(0.0), None) == 1


def test_autotune_table_round_trip_and_corruption(lib, tmp_path):
    """The autotune cache file: what is saved loads back; an altered, truncated or malformed file
    is refused with TOP_ERR_INVALID_ARG and leaves the table as it was (host-only calls)."""
    cdll = lib.load()
    assert cdll.top_autotune_clear() == 0
    entries = {1024: 0x1 | 0x8, 512: 0x2 | (3 << 8), 250: 0, 64: 0x800}  # 0x800: TOP_TUNE_THREE_PASS
    for m, f in entries.items():
        assert cdll.top_autotune_set(m, f) == 0
    assert cdll.top_autotune_set(1024, 0x8000) == 1  # unknown flag bit
    assert cdll.top_autotune_set(1024, 0x1000) == 1
    assert cdll.top_autotune_set(0, 0) == 1
    path = tmp_path / "tune.txt"
    assert cdll.top_autotune_save(str(path).encode()) == 0
    assert cdll.top_autotune_clear() == 0

    def get(m):
        v = C.c_uint32()
        assert cdll.top_autotune_get(m, C.byref(v)) == 0
        return v.value

    assert get(1024) == 0
    assert cdll.top_autotune_load(str(path).encode()) == 0
    assert {m: get(m) for m in entries} == entries
    text = path.read_text()
    assert text.startswith("top-autotune 1\n") and "checksum" in text
    # an altered entry, a truncated file, a bad header and a missing file are all refused
    cdll.top_autotune_set(2048, 0x4)
    bad = {"altered": text.replace("1024 9", "1024 1"), "truncated": text[: len(text) // 2],
           "header": text.replace("top-autotune 1", "top-autotune 9"), "empty": ""}
    for name, body in bad.items():
        p = tmp_path / f"{name}.txt"
        p.write_text(body)
        assert cdll.top_autotune_load(str(p).encode()) == 1, name
        assert b"autotune cache" in cdll.top_last_error()
        assert get(2048) == 0x4 and get(1024) == entries[1024]  # unchanged
    assert cdll.top_autotune_load(str(tmp_path / "missing.txt").encode()) == 1
    assert cdll.top_autotune_clear() == 0
