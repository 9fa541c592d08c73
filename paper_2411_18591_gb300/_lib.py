"""ctypes view of the C ABI declared in include/top.h (loads the in-tree libtop.so)."""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtop.so")

TOP_OK = 0
STATUS = {0: "TOP_OK", 1: "TOP_ERR_INVALID_ARG", 2: "TOP_ERR_UNSUPPORTED", 3: "TOP_ERR_OOM", 4: "TOP_ERR_CUDA",
          5: "TOP_ERR_TIMEOUT", 6: "TOP_ERR_INTERNAL"}

TOP_AS = 0
TOP_FRESNEL_TF = 1
TOP_DI = 2
TOP_AUTO = 3
TOP_NEAREST = 0
TOP_BILINEAR = 1
TOP_MOD_COMPLEX = 0x1
TOP_MOD_AMPLITUDE = 0x2
TOP_MOD_PHASE = 0x4
TOP_MOD_LENS = 0x8
TOP_MOD_CIRC = 0x10


class TopGrid(C.Structure):
    _fields_ = [("batch", C.c_int64), ("ny", C.c_int32), ("nx", C.c_int32), ("dy", C.c_double),
                ("dx", C.c_double), ("pad", C.c_double), ("method", C.c_int32), ("input_repeat", C.c_int32)]


class TopMod(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("reserved", C.c_int32), ("mask", C.c_void_p), ("amplitude", C.c_void_p),
                ("phase", C.c_void_p), ("batch_stride", C.c_int64), ("focal_length", C.c_double),
                ("radius", C.c_double)]


class TopModGrads(C.Structure):
    _fields_ = [("saved_in", C.c_void_p), ("grad_phase", C.c_void_p), ("grad_amplitude", C.c_void_p),
                ("grad_mask", C.c_void_p)]


class TopStage(C.Structure):
    _fields_ = [("z", C.c_double), ("pre", C.POINTER(TopMod)), ("keep", C.c_void_p)]


class TopError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.c_int64
_GRID = C.POINTER(TopGrid)
_MOD = C.POINTER(TopMod)
_GRADS = C.POINTER(TopModGrads)

SIGNATURES = {
    "top_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "top_destroy": (C.c_int, [_P]),
    "top_last_error": (C.c_char_p, []),
    "top_status_string": (C.c_char_p, [C.c_int]),
    "top_version": (C.c_int, []),
    "top_set_workspace_limit": (C.c_int, [_P, C.c_uint64]),
    "top_plan_query": (C.c_int, [_GRID, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)]),
    "top_zcritical": (C.c_double, [C.c_double, C.c_double, C.c_double]),
    "top_propagate": (C.c_int, [_P, _GRID, _P, _P, _D, _D, _I64, _MOD, _MOD, _P]),
    "top_propagate_noalloc": (C.c_int, [_GRID, _P, _P, _D, _D, _I64, _P]),
    "top_propagate_ragged": (C.c_int, [_P, C.c_int, _GRID, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), _D, _D,
                                       C.c_int, _P]),
    "top_fused_chain": (C.c_int, [_P, _GRID, _P, _P, _P, _I64, _D, _I64, C.POINTER(TopStage), C.c_int, _P]),
    "top_fused_chain_backward": (C.c_int, [_P, _GRID, _P, _P, _I64, _D, _I64, C.POINTER(TopStage), C.c_int, _GRADS,
                                           _P, _P]),
    "top_propagate_backward": (C.c_int, [_P, _GRID, _P, _P, _D, _D, _I64, _MOD, _MOD, _GRADS, _P]),
    "top_propagate_intensity": (C.c_int, [_P, _GRID, _P, _P, _P, _I64, _P, _D, _D, _I64, _MOD, _MOD, _P]),
    "top_propagate_intensity_backward": (C.c_int, [_P, _GRID, _P, _P, _P, _I64, _P, _D, _D, _I64, _MOD, _MOD,
                                                   _GRADS, _P]),
    "top_modulate": (C.c_int, [_P, _GRID, _MOD, _P, _P, _D, _I64, _P]),
    "top_modulate_backward": (C.c_int, [_P, _GRID, _MOD, _P, _P, _GRADS, _D, _I64, _P]),
    "top_mse_loss": (C.c_int, [_P, _I64, _P, _P, _P, _P, _P]),
    "top_resample": (C.c_int, [_P, _GRID, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _P, _P, _P]),
    "top_jones": (C.c_int, [_P, _GRID, _I64, _P, _D, _P, _P, _P]),
    "top_jones_backward": (C.c_int, [_P, _GRID, _I64, _P, _D, _P, _P, _P, _P, _P]),
    "top_field_power": (C.c_int, [_P, _GRID, _P, _P, _P]),
    "top_jones_linear_polarizer": (C.c_int, [C.c_double, _D]),
    "top_jones_circular_polarizer": (C.c_int, [C.c_int, _D]),
    "top_jones_waveplate": (C.c_int, [C.c_double, C.c_double, _D]),
    "top_propagate_overlap": (C.c_int, [_P, _GRID, _P, _P, _P, _I64, _P, _P, _D, _D, _I64, _MOD, _MOD, _P]),
    "top_overlap_loss": (C.c_int, [_P, _GRID, _P, _P, _I64, _P, _P, _P]),
    "top_propagate_coherence": (C.c_int, [_P, _GRID, _P, _P, _D, _D, _MOD, _P]),
    "top_propagate_coherence_backward": (C.c_int, [_P, _GRID, _P, _P, _D, _D, _MOD, _GRADS, _P]),
    "top_intensity": (C.c_int, [_P, _GRID, _P, _P, _I64, _P, _P]),
    "top_intensity_backward": (C.c_int, [_P, _GRID, _P, _P, _P, _I64, _P, _P]),
    "top_coherence_intensity": (C.c_int, [_P, _GRID, _P, _P, _P]),
    "top_coherence_intensity_backward": (C.c_int, [_P, _GRID, _P, _P, _P]),
    "top_autotune": (C.c_int, [_P, _GRID, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "top_autotune_set": (C.c_int, [C.c_int, C.c_uint32]),
    "top_autotune_get": (C.c_int, [C.c_int, C.POINTER(C.c_uint32)]),
    "top_autotune_clear": (C.c_int, []),
    "top_autotune_save": (C.c_int, [C.c_char_p]),
    "top_autotune_load": (C.c_int, [C.c_char_p]),
    "top_profile_enable": (C.c_int, [_P, C.c_int]),
    "top_profile_read": (C.c_int, [_P, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libtop.so (built by ``paper_2411_18591_gb300.build.build()``); fails loudly if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != TOP_OK:
        msg = load().top_last_error().decode(errors="replace")
        raise TopError(status, msg)


def doubles(values) -> C.Array:
    vals = [float(v) for v in values]
    return (C.c_double * len(vals))(*vals)
