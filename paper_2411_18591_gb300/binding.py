"""Python binding of the C ABI with the same call names, for torch CUDA tensors.

Argument marshalling only: every step of the computation runs in libtop.so's
CUDA kernels. Tensors must live on a CUDA device; fields are complex64
[batch, ny, nx] (a single [ny, nx] field is treated as batch 1), phases,
amplitudes and intensities float32. Calls run on torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import TopGrid, TopMod, TopModGrads, TopStage, check, doubles

METHODS = {"as": _lib.TOP_AS, "angular_spectrum": _lib.TOP_AS, "fresnel": _lib.TOP_FRESNEL_TF,
           "fresnel_tf": _lib.TOP_FRESNEL_TF, "di": _lib.TOP_DI, "direct": _lib.TOP_DI, "auto": _lib.TOP_AUTO,
           _lib.TOP_AS: _lib.TOP_AS, _lib.TOP_FRESNEL_TF: _lib.TOP_FRESNEL_TF, _lib.TOP_DI: _lib.TOP_DI,
           _lib.TOP_AUTO: _lib.TOP_AUTO}

_handles: dict = {}
_handle_lock = threading.Lock()


def handle(device: Optional[torch.device] = None) -> C.c_void_p:
    """The library handle of a CUDA device (created on first use, kept for the process)."""
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    with _handle_lock:
        h = _handles.get(idx)
        if h is None:
            h = C.c_void_p()
            check(lib.top_create(C.byref(h), idx))
            _handles[idx] = h
    return h


def _stream(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _field(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.complex64:
        raise ValueError(f"{name} must be complex64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _real(t: Optional[torch.Tensor], name: str) -> Optional[torch.Tensor]:
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def _shape3(t: torch.Tensor):
    if t.dim() == 2:
        return 1, t.shape[0], t.shape[1]
    if t.dim() == 3:
        return t.shape[0], t.shape[1], t.shape[2]
    raise ValueError("fields must be [ny, nx] or [batch, ny, nx]")


def make_grid(batch: int, ny: int, nx: int, dy: float, dx: float, pad: float = 2.0, method="as",
              input_repeat: int = 1) -> TopGrid:
    return TopGrid(int(batch), int(ny), int(nx), float(dy), float(dx), float(pad), METHODS[method],
                   int(input_repeat))


@dataclass
class Modulation:
    """Element modulation of Eq. 1: product of the factors that are set.

    mask: complex64 [ny, nx] or [batch, ny, nx]; amplitude / phase: float32 of the same shapes;
    focal_length: thin lens f (m); radius: circular aperture radius R (m).
    """
    mask: Optional[torch.Tensor] = None
    amplitude: Optional[torch.Tensor] = None
    phase: Optional[torch.Tensor] = None
    focal_length: Optional[float] = None
    radius: Optional[float] = None

    def to_c(self) -> TopMod:
        m = TopMod()
        flags = 0
        stride = 0
        for t, flag, name in ((self.mask, _lib.TOP_MOD_COMPLEX, "mask"),
                              (self.amplitude, _lib.TOP_MOD_AMPLITUDE, "amplitude"),
                              (self.phase, _lib.TOP_MOD_PHASE, "phase")):
            if t is None:
                continue
            if flag == _lib.TOP_MOD_COMPLEX:
                _field(t, name)
            else:
                _real(t, name)
            flags |= flag
            s = t.shape[-1] * t.shape[-2] if t.dim() == 3 else 0
            stride = max(stride, s)
        m.mask = _ptr(self.mask)
        m.amplitude = _ptr(self.amplitude)
        m.phase = _ptr(self.phase)
        if self.focal_length is not None:
            flags |= _lib.TOP_MOD_LENS
            m.focal_length = float(self.focal_length)
        if self.radius is not None:
            flags |= _lib.TOP_MOD_CIRC
            m.radius = float(self.radius)
        m.flags = flags
        m.batch_stride = stride
        return m


def _mod(m: Optional[Modulation]):
    return None if m is None else C.byref(m.to_c())


def _lz(lam, z, batch):
    lam = [lam] if isinstance(lam, (int, float)) else list(lam)
    zs = [z] if isinstance(z, (int, float)) else list(z)
    n = max(len(lam), len(zs))
    if len(lam) == 1 and n > 1:
        lam = lam * n
    if len(zs) == 1 and n > 1:
        zs = zs * n
    return doubles(lam), doubles(zs), n


def top_propagate(field: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0, method="as",
                  pre: Optional[Modulation] = None, post: Optional[Modulation] = None,
                  out: Optional[torch.Tensor] = None, input_repeat: int = 1) -> torch.Tensor:
    """out = post * P_z(pre * field) (Eq. 1 and Eq. 4-5).

    With input_repeat = k each input field feeds k consecutive output fields (batch_out = k batch_in).
    """
    _field(field, "field")
    b, ny, nx = _shape3(field)
    b *= input_repeat
    if out is None:
        out = torch.empty((b, ny, nx), dtype=field.dtype, device=field.device)
    else:
        _field(out, "out")
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method, input_repeat)
    check(_lib.load().top_propagate(handle(field.device), C.byref(g), field.data_ptr(), out.data_ptr(), lams, zs, n,
                                    _mod(pre), _mod(post), _stream(field)))
    return out


def top_propagate_overlap(field: torch.Tensor, target: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0,
                          method="as", pre: Optional[Modulation] = None, post: Optional[Modulation] = None,
                          keep_field: bool = False):
    """Overlaps O_b = sum psi_b conj(phi) dx dy of Eq. 7 and powers sum |psi_b|^2 dx dy of
    psi_b = post * P_z(pre * field_b); returns (overlap complex128 [batch], power float64 [batch],
    psi or None). ``target`` is [ny, nx] (shared) or [batch, ny, nx]."""
    _field(field, "field")
    _field(target, "target")
    b, ny, nx = _shape3(field)
    stride = ny * nx if target.dim() == 3 else 0
    ov = torch.empty((b, 2), dtype=torch.float64, device=field.device)
    pw = torch.empty((b,), dtype=torch.float64, device=field.device)
    psi = torch.empty_like(field) if keep_field else None
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method)
    check(_lib.load().top_propagate_overlap(handle(field.device), C.byref(g), field.data_ptr(), _ptr(psi),
                                            target.data_ptr(), stride, ov.data_ptr(), pw.data_ptr(), lams, zs, n,
                                            _mod(pre), _mod(post), _stream(field)))
    return torch.view_as_complex(ov), pw, psi


def top_overlap_loss(overlap: torch.Tensor, target: torch.Tensor, batch: int, ny: int, nx: int, dy: float, dx: float,
                     want_grad: bool = True):
    """Eq. 7 loss mean_b (1 - |O_b|^2) (device float64 scalar) and dL/dpsi (complex64 [batch, ny, nx])."""
    _field(target, "target")
    ov = torch.view_as_real(overlap.to(torch.complex128)).contiguous()
    stride = ny * nx if target.dim() == 3 else 0
    loss = torch.empty((1,), dtype=torch.float64, device=target.device)
    grad = torch.empty((batch, ny, nx), dtype=torch.complex64, device=target.device) if want_grad else None
    g = make_grid(batch, ny, nx, dy, dx)
    check(_lib.load().top_overlap_loss(handle(target.device), C.byref(g), ov.data_ptr(), target.data_ptr(), stride,
                                       loss.data_ptr(), _ptr(grad), _stream(target)))
    return loss[0], grad


def top_resample(field: torch.Tensor, dy: float, dx: float, ny_out: int, nx_out: int, dy_out: float, dx_out: float,
                 mode: str = "bilinear") -> torch.Tensor:
    """Interpolate [..., ny, nx] fields on spacing (dy, dx) onto the centred grid (ny_out, nx_out,
    dy_out, dx_out) (§3), nearest or bilinear."""
    _field(field, "field")
    ny, nx = field.shape[-2:]
    b = field.numel() // (ny * nx)
    out = torch.empty(field.shape[:-2] + (ny_out, nx_out), dtype=field.dtype, device=field.device)
    g = make_grid(b, ny, nx, dy, dx)
    check(_lib.load().top_resample(handle(field.device), C.byref(g), ny_out, nx_out, dy_out, dx_out, _interp(mode), 0,
                                   field.data_ptr(), out.data_ptr(), _stream(field)))
    return out


def top_resample_backward(grad_out: torch.Tensor, ny: int, nx: int, dy: float, dx: float, dy_out: float, dx_out: float,
                          mode: str = "bilinear") -> torch.Tensor:
    """Gradient of top_resample: from [..., ny_out, nx_out] on (dy_out, dx_out) back to [..., ny, nx] on (dy, dx)."""
    _field(grad_out, "grad_out")
    ny_out, nx_out = grad_out.shape[-2:]
    b = grad_out.numel() // (ny_out * nx_out)
    out = torch.empty(grad_out.shape[:-2] + (ny, nx), dtype=grad_out.dtype, device=grad_out.device)
    g = make_grid(b, ny, nx, dy, dx)
    check(_lib.load().top_resample(handle(grad_out.device), C.byref(g), ny_out, nx_out, dy_out, dx_out, _interp(mode), 1,
                                   grad_out.data_ptr(), out.data_ptr(), _stream(grad_out)))
    return out


def _interp(mode: str) -> int:
    return {"nearest": _lib.TOP_NEAREST, "bilinear": _lib.TOP_BILINEAR}[mode]


# ----------------------------------------------------------------------------- polarisation


def _jones_matrix(call, *args):
    """A 3x3 Jones matrix from one of the library's constructors, as complex128 [3, 3]."""
    import numpy as np
    out = (C.c_double * 18)()
    check(call(*args, out))
    v = np.frombuffer(out, dtype=np.float64)
    return (v[0::2] + 1j * v[1::2]).reshape(3, 3)


def linear_polarizer(theta: float):
    """Linear polariser with its transmission axis at theta to x (§5.1)."""
    return _jones_matrix(_lib.load().top_jones_linear_polarizer, float(theta))


def circular_polarizer(handedness: int = 1):
    """Circular polariser passing (1, i handedness) / sqrt 2 (§5.1)."""
    return _jones_matrix(_lib.load().top_jones_circular_polarizer, int(handedness))


def waveplate(retardance: float, theta: float = 0.0):
    """Waveplate of the given retardance with its fast axis at theta (quarter-wave: pi/2, half-wave: pi)."""
    return _jones_matrix(_lib.load().top_jones_waveplate, float(retardance), float(theta))


def _jones_args(jones):
    if isinstance(jones, torch.Tensor):
        _field(jones, "jones")
        return jones.data_ptr(), None
    import numpy as np
    j = np.asarray(jones, dtype=np.complex128).reshape(9)
    return None, doubles([v for z in j for v in (z.real, z.imag)])


def top_jones(field: torch.Tensor, jones, inner: int = 1, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """J |psi> per pixel on three-component fields. ``field``: complex64 [..., ny, nx] with
    3 * inner * K leading entries (component c of polarised field (o, i) at (o 3 + c) inner + i).
    ``jones``: a 3x3 matrix (uniform) or a complex64 [3, 3, ny, nx] tensor (spatially varying)."""
    _field(field, "field")
    ny, nx = field.shape[-2:]
    b = field.numel() // (ny * nx)
    out = torch.empty_like(field) if out is None else _field(out, "out")
    jp, ju = _jones_args(jones)
    g = make_grid(b, ny, nx, 1.0, 1.0)
    check(_lib.load().top_jones(handle(field.device), C.byref(g), inner, jp, ju, field.data_ptr(), out.data_ptr(),
                                _stream(field)))
    return out


def top_jones_backward(saved_in: torch.Tensor, grad_out: torch.Tensor, jones, inner: int = 1, want_grad_in: bool = True,
                       want_grad_jones: bool = False):
    """(grad_in, grad_jones) of top_jones; grad_jones only for a spatially varying [3, 3, ny, nx] tensor."""
    _field(grad_out, "grad_out")
    ny, nx = grad_out.shape[-2:]
    b = grad_out.numel() // (ny * nx)
    gin = torch.empty_like(grad_out) if want_grad_in else None
    gj = torch.empty((3, 3, ny, nx), dtype=torch.complex64, device=grad_out.device) if want_grad_jones else None
    jp, ju = _jones_args(jones)
    g = make_grid(b, ny, nx, 1.0, 1.0)
    check(_lib.load().top_jones_backward(handle(grad_out.device), C.byref(g), inner, jp, ju, _ptr(saved_in),
                                         grad_out.data_ptr(), _ptr(gin), _ptr(gj), _stream(grad_out)))
    return gin, gj


def top_field_power(field: torch.Tensor, dy: float, dx: float) -> torch.Tensor:
    """sum |psi_b|^2 dx dy for every [ny, nx] plane of ``field`` (float64 device tensor)."""
    _field(field, "field")
    ny, nx = field.shape[-2:]
    b = field.numel() // (ny * nx)
    power = torch.empty((b,), dtype=torch.float64, device=field.device)
    g = make_grid(b, ny, nx, dy, dx)
    check(_lib.load().top_field_power(handle(field.device), C.byref(g), field.data_ptr(), power.data_ptr(),
                                      _stream(field)))
    return power


def top_propagate_ragged(fields: Sequence[torch.Tensor], spacings, lams, zs, pad: float = 2.0, method="as",
                         backward: bool = False, out: Optional[Sequence[torch.Tensor]] = None):
    """Propagate (or back-propagate) fields of different sizes in one call: field i ([ny, nx]
    complex64) with spacing spacings[i] (a number or a (dy, dx) pair), wavelength lams[i] and
    distance zs[i]. Returns the output fields (``out`` if given)."""
    n = len(fields)
    if n == 0:
        return []
    if out is None:
        out = [torch.empty_like(f) for f in fields]
    if not (len(spacings) == len(lams) == len(zs) == len(out) == n):
        raise ValueError("fields, spacings, lams, zs and out must have the same length")
    grids = (TopGrid * n)()
    ins = (C.c_void_p * n)()
    outs = (C.c_void_p * n)()
    for i, (f, o) in enumerate(zip(fields, out)):
        _field(f, "field")
        _field(o, "out")
        if f.dim() != 2 or o.shape != f.shape:
            raise ValueError("ragged fields are [ny, nx] and out[i] must match field i")
        sp = spacings[i]
        dy, dx = (sp, sp) if isinstance(sp, (int, float)) else sp
        grids[i] = make_grid(1, f.shape[0], f.shape[1], dy, dx, pad, method)
        ins[i] = f.data_ptr()
        outs[i] = o.data_ptr()
    dev = fields[0].device if n else torch.device("cuda", torch.cuda.current_device())
    check(_lib.load().top_propagate_ragged(handle(dev), n, grids, ins, outs, doubles([float(v) for v in lams]),
                                           doubles([float(v) for v in zs]), 1 if backward else 0,
                                           C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))
    return out


@dataclass
class Stage:
    """One stage of a system chain: multiply by ``pre`` (Eq. 1), then propagate by ``z`` (Eq. 4);
    ``keep`` (complex64, the batch's shape) receives the stage's output field."""
    z: float
    pre: Optional[Modulation] = None
    keep: Optional[torch.Tensor] = None


def top_fused_chain(field: torch.Tensor, dy: float, dx: float, lam, stages: Sequence[Stage], pad: float = 2.0,
                    method="as", out: Optional[torch.Tensor] = None, intensity_group: Optional[int] = None,
                    input_repeat: int = 1, want_field: bool = True):
    """x_K of x_k = P_{z_k}(pre_k x_{k-1}), x_0 = field, with the row passes between stages fused.

    Returns (out, intensity): ``out`` the last field (None if ``want_field`` is False and an
    intensity is asked for), ``intensity`` the sum of |x_K|^2 over each ``intensity_group``
    consecutive fields (Eq. 14) or None.
    """
    _field(field, "field")
    b, ny, nx = _shape3(field)
    b *= input_repeat
    if out is None and (want_field or intensity_group is None):
        out = torch.empty((b, ny, nx), dtype=field.dtype, device=field.device)
    elif out is not None:
        _field(out, "out")
    inten = None
    group = 1
    if intensity_group is not None:
        group = int(intensity_group)
        if group < 1 or b % group:
            raise ValueError("intensity_group must divide the batch")
        inten = torch.empty((b // group, ny, nx), dtype=torch.float32, device=field.device)
    lams = [lam] if isinstance(lam, (int, float)) else list(lam)
    mods = []
    arr = (TopStage * len(stages))()
    for i, st in enumerate(stages):
        arr[i].z = float(st.z)
        if st.pre is not None:
            m = st.pre.to_c()
            mods.append(m)
            arr[i].pre = C.pointer(m)
        if st.keep is not None:
            _field(st.keep, "keep")
            arr[i].keep = st.keep.data_ptr()
    g = make_grid(b, ny, nx, dy, dx, pad, method, input_repeat)
    check(_lib.load().top_fused_chain(handle(field.device), C.byref(g), field.data_ptr(), _ptr(out), _ptr(inten), group,
                                      doubles(lams), len(lams), arr, len(stages), _stream(field)))
    return out, inten


def top_fused_chain_backward(field: torch.Tensor, grad_intensity: torch.Tensor, dy: float, dx: float, lam,
                             stages: Sequence[Stage], pad: float = 2.0, method="as", intensity_group: int = 1,
                             saved_in: Optional[torch.Tensor] = None, want_grad_in: bool = True,
                             grad_phase: Optional[torch.Tensor] = None, grad_amplitude: Optional[torch.Tensor] = None,
                             grad_mask: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    """Backward of top_fused_chain's grouped intensity: ``field`` is the chain's last field x_K,
    ``grad_intensity`` dL/dI; ``stages`` in forward order. Returns dL/dx_0 (None if not
    ``want_grad_in``) and fills the gradients of stages[0].pre given ``saved_in`` = x_0."""
    _field(field, "field")
    _real(grad_intensity, "grad_intensity")
    b, ny, nx = _shape3(field)
    grad_in = torch.empty_like(field) if want_grad_in else None
    lams = [lam] if isinstance(lam, (int, float)) else list(lam)
    mods = []
    arr = (TopStage * len(stages))()
    for i, st in enumerate(stages):
        arr[i].z = float(st.z)
        if st.pre is not None:
            m = st.pre.to_c()
            mods.append(m)
            arr[i].pre = C.pointer(m)
    grads = None
    if grad_phase is not None or grad_amplitude is not None or grad_mask is not None:
        if saved_in is None:
            raise ValueError("modulation gradients need saved_in (the chain's input)")
        _field(saved_in, "saved_in")
        grads = C.byref(TopModGrads(saved_in.data_ptr(), _ptr(_real(grad_phase, "grad_phase")),
                                    _ptr(_real(grad_amplitude, "grad_amplitude")), _ptr(grad_mask)))
    g = make_grid(b, ny, nx, dy, dx, pad, method)
    check(_lib.load().top_fused_chain_backward(handle(field.device), C.byref(g), field.data_ptr(),
                                               grad_intensity.data_ptr(), int(intensity_group), doubles(lams),
                                               len(lams), arr, len(stages), grads, _ptr(grad_in), _stream(field)))
    return grad_in


def top_propagate_noalloc(field: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0, method="as", *,
                          out: torch.Tensor) -> torch.Tensor:
    """out = P_z(field) through the library's static device scratch: no handle, no device allocation.

    ``out`` is required (complex64, the shape of ``field``; ``out is field`` allowed), so the call
    allocates nothing. Calls on one device must not overlap (they share the scratch)."""
    _field(field, "field")
    _field(out, "out")
    b, ny, nx = _shape3(field)
    if _shape3(out) != (b, ny, nx):
        raise ValueError("out must have the shape of field")
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method)
    with torch.cuda.device(field.device):
        check(_lib.load().top_propagate_noalloc(C.byref(g), field.data_ptr(), out.data_ptr(), lams, zs, n,
                                                _stream(field)))
    return out


def top_propagate_backward(grad_out: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0, method="as",
                           pre: Optional[Modulation] = None, post: Optional[Modulation] = None,
                           saved_in: Optional[torch.Tensor] = None, want_grad_in: bool = True,
                           grad_phase: Optional[torch.Tensor] = None, grad_amplitude: Optional[torch.Tensor] = None,
                           grad_mask: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    """Adjoint of top_propagate; fills grad_phase / grad_amplitude / grad_mask of ``pre`` if given."""
    _field(grad_out, "grad_out")
    b, ny, nx = _shape3(grad_out)
    grad_in = torch.empty_like(grad_out) if want_grad_in else None
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method)
    grads = None
    if grad_phase is not None or grad_amplitude is not None or grad_mask is not None:
        if saved_in is None:
            raise ValueError("modulation gradients need saved_in (the forward input)")
        _field(saved_in, "saved_in")
        grads = C.byref(TopModGrads(saved_in.data_ptr(), _ptr(_real(grad_phase, "grad_phase")),
                                    _ptr(_real(grad_amplitude, "grad_amplitude")), _ptr(grad_mask)))
    check(_lib.load().top_propagate_backward(handle(grad_out.device), C.byref(g), grad_out.data_ptr(), _ptr(grad_in),
                                             lams, zs, n, _mod(pre), _mod(post), grads, _stream(grad_out)))
    return grad_in


def top_propagate_intensity(field: torch.Tensor, dy: float, dx: float, lam, z, pad: float = 2.0, method="as",
                            group: int = 1, weights: Optional[torch.Tensor] = None,
                            pre: Optional[Modulation] = None, post: Optional[Modulation] = None,
                            keep_field: bool = False, input_repeat: int = 1):
    """I[b/group] = sum_group w_b |post * P_z(pre * field_b)|^2 (Eq. 14); returns (I, field or None)."""
    _field(field, "field")
    b, ny, nx = _shape3(field)
    b *= input_repeat
    inten = torch.empty((b // group, ny, nx), dtype=torch.float32, device=field.device)
    fout = torch.empty((b, ny, nx), dtype=field.dtype, device=field.device) if keep_field else None
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method, input_repeat)
    check(_lib.load().top_propagate_intensity(handle(field.device), C.byref(g), field.data_ptr(), _ptr(fout),
                                              inten.data_ptr(), group, _ptr(_real(weights, "weights")), lams, zs,
                                              n, _mod(pre), _mod(post), _stream(field)))
    return inten, fout


def top_intensity(field: torch.Tensor, group: int = 1, weights: Optional[torch.Tensor] = None) -> torch.Tensor:
    """I[b/group] = sum over each group of `group` fields of w_b |field_b|^2 (Eq. 14, no propagation)."""
    _field(field, "field")
    b, ny, nx = _shape3(field)
    inten = torch.empty((b // max(1, group), ny, nx), dtype=torch.float32, device=field.device)
    g = make_grid(b, ny, nx, 1.0, 1.0, 1.0, "as")
    check(_lib.load().top_intensity(handle(field.device), C.byref(g), field.data_ptr(), inten.data_ptr(), group,
                                    _ptr(_real(weights, "weights")), _stream(field)))
    return inten


def top_intensity_backward(field: torch.Tensor, grad_intensity: torch.Tensor, group: int = 1,
                           weights: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Backward of top_intensity: grad_field_b = 2 w_b grad_I[b/group] field_b."""
    _field(field, "field")
    _real(grad_intensity, "grad_intensity")
    b, ny, nx = _shape3(field)
    if out is None:
        out = torch.empty_like(field)
    else:
        _field(out, "out")
    g = make_grid(b, ny, nx, 1.0, 1.0, 1.0, "as")
    check(_lib.load().top_intensity_backward(handle(field.device), C.byref(g), field.data_ptr(),
                                             grad_intensity.data_ptr(), out.data_ptr(), group,
                                             _ptr(_real(weights, "weights")), _stream(field)))
    return out


def top_propagate_intensity_backward(field: torch.Tensor, grad_intensity: torch.Tensor, dy: float, dx: float, lam,
                                     z, pad: float = 2.0, method="as", group: int = 1,
                                     weights: Optional[torch.Tensor] = None, pre: Optional[Modulation] = None,
                                     post: Optional[Modulation] = None, saved_in: Optional[torch.Tensor] = None,
                                     want_grad_in: bool = True, grad_phase: Optional[torch.Tensor] = None,
                                     grad_amplitude: Optional[torch.Tensor] = None,
                                     grad_mask: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    """Backward of top_propagate_intensity given the saved output field."""
    _field(field, "field")
    _real(grad_intensity, "grad_intensity")
    b, ny, nx = _shape3(field)
    grad_in = torch.empty_like(field) if want_grad_in else None
    lams, zs, n = _lz(lam, z, b)
    g = make_grid(b, ny, nx, dy, dx, pad, method)
    grads = None
    if grad_phase is not None or grad_amplitude is not None or grad_mask is not None:
        _field(saved_in, "saved_in")
        grads = C.byref(TopModGrads(saved_in.data_ptr(), _ptr(_real(grad_phase, "grad_phase")),
                                    _ptr(_real(grad_amplitude, "grad_amplitude")), _ptr(grad_mask)))
    check(_lib.load().top_propagate_intensity_backward(handle(field.device), C.byref(g), field.data_ptr(),
                                                       grad_intensity.data_ptr(), _ptr(grad_in), group,
                                                       _ptr(_real(weights, "weights")), lams, zs, n, _mod(pre),
                                                       _mod(post), grads, _stream(field)))
    return grad_in


def top_modulate(field: torch.Tensor, mod: Modulation, dy: float, dx: float, lam=1.0,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """out = M * field (Eq. 1)."""
    _field(field, "field")
    b, ny, nx = _shape3(field)
    out = torch.empty_like(field) if out is None else _field(out, "out")
    lams, _, n = _lz(lam, 0.0, b)
    g = make_grid(b, ny, nx, dy, dx, 1.0, "as")
    check(_lib.load().top_modulate(handle(field.device), C.byref(g), C.byref(mod.to_c()), field.data_ptr(),
                                   out.data_ptr(), lams, n, _stream(field)))
    return out


def top_modulate_backward(grad_out: torch.Tensor, mod: Modulation, dy: float, dx: float, lam=1.0,
                          saved_in: Optional[torch.Tensor] = None, want_grad_in: bool = True,
                          grad_phase: Optional[torch.Tensor] = None, grad_amplitude: Optional[torch.Tensor] = None,
                          grad_mask: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    """Backward of top_modulate: conj(M) grad_out and the gradients of M's parameters."""
    _field(grad_out, "grad_out")
    b, ny, nx = _shape3(grad_out)
    grad_in = torch.empty_like(grad_out) if want_grad_in else None
    lams, _, n = _lz(lam, 0.0, b)
    g = make_grid(b, ny, nx, dy, dx, 1.0, "as")
    grads = None
    if grad_phase is not None or grad_amplitude is not None or grad_mask is not None:
        _field(saved_in, "saved_in")
        grads = C.byref(TopModGrads(saved_in.data_ptr(), _ptr(_real(grad_phase, "grad_phase")),
                                    _ptr(_real(grad_amplitude, "grad_amplitude")), _ptr(grad_mask)))
    check(_lib.load().top_modulate_backward(handle(grad_out.device), C.byref(g), C.byref(mod.to_c()),
                                            grad_out.data_ptr(), _ptr(grad_in), grads, lams, n, _stream(grad_out)))
    return grad_in


def top_mse_loss(intensity: torch.Tensor, target: torch.Tensor, want_grad: bool = True):
    """(loss as a float64 device scalar, dL/dI or None) for L = mean((I - T)^2)."""
    _real(intensity, "intensity")
    _real(target, "target")
    loss = torch.empty(2, dtype=torch.float64, device=intensity.device)  # 16-byte aligned scalar
    grad = torch.empty_like(intensity) if want_grad else None
    check(_lib.load().top_mse_loss(handle(intensity.device), intensity.numel(), intensity.data_ptr(),
                                   target.data_ptr(), loss.data_ptr(), _ptr(grad), _stream(intensity)))
    return loss[0], grad


def _coh_grid(gamma: torch.Tensor, dy, dx, pad, method) -> TopGrid:
    if gamma.dim() == 4:
        b, ny, nx = 1, gamma.shape[0], gamma.shape[1]
    elif gamma.dim() == 5:
        b, ny, nx = gamma.shape[0], gamma.shape[1], gamma.shape[2]
    else:
        raise ValueError("coherence tensors are [ny, nx, ny, nx] or [batch, ny, nx, ny, nx]")
    return make_grid(b, ny, nx, dy, dx, pad, method)


def top_propagate_coherence(gamma: torch.Tensor, dy: float, dx: float, lam: float, z: float, pad: float = 2.0,
                            method="as", mask: Optional[Modulation] = None) -> torch.Tensor:
    """Gamma_z = P (M M* Gamma) P^H (Eq. 12-13)."""
    _field(gamma, "gamma")
    out = torch.empty_like(gamma)
    g = _coh_grid(gamma, dy, dx, pad, method)
    check(_lib.load().top_propagate_coherence(handle(gamma.device), C.byref(g), gamma.data_ptr(), out.data_ptr(),
                                              doubles([lam]), doubles([z]), _mod(mask), _stream(gamma)))
    return out


def top_propagate_coherence_backward(grad_out: torch.Tensor, dy: float, dx: float, lam: float, z: float,
                                     pad: float = 2.0, method="as", mask: Optional[Modulation] = None,
                                     saved_in: Optional[torch.Tensor] = None, want_grad_in: bool = True,
                                     grad_phase: Optional[torch.Tensor] = None,
                                     grad_amplitude: Optional[torch.Tensor] = None,
                                     grad_mask: Optional[torch.Tensor] = None) -> Optional[torch.Tensor]:
    _field(grad_out, "grad_out")
    grad_in = torch.empty_like(grad_out) if want_grad_in else None
    g = _coh_grid(grad_out, dy, dx, pad, method)
    grads = None
    if grad_phase is not None or grad_amplitude is not None or grad_mask is not None:
        _field(saved_in, "saved_in")
        grads = C.byref(TopModGrads(saved_in.data_ptr(), _ptr(_real(grad_phase, "grad_phase")),
                                    _ptr(_real(grad_amplitude, "grad_amplitude")), _ptr(grad_mask)))
    check(_lib.load().top_propagate_coherence_backward(handle(grad_out.device), C.byref(g), grad_out.data_ptr(),
                                                       _ptr(grad_in), doubles([lam]), doubles([z]), _mod(mask),
                                                       grads, _stream(grad_out)))
    return grad_in


def top_coherence_intensity(gamma: torch.Tensor) -> torch.Tensor:
    _field(gamma, "gamma")
    g = _coh_grid(gamma, 1.0, 1.0, 1.0, "as")
    out = torch.empty((g.batch, g.ny, g.nx), dtype=torch.float32, device=gamma.device)
    check(_lib.load().top_coherence_intensity(handle(gamma.device), C.byref(g), gamma.data_ptr(), out.data_ptr(),
                                              _stream(gamma)))
    return out.reshape(gamma.shape[:-2]) if gamma.dim() == 4 else out


def top_coherence_intensity_backward(grad_intensity: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    _real(grad_intensity, "grad_intensity")
    g = _coh_grid(like, 1.0, 1.0, 1.0, "as")
    out = torch.empty_like(like)
    check(_lib.load().top_coherence_intensity_backward(handle(like.device), C.byref(g), grad_intensity.data_ptr(),
                                                       out.data_ptr(), _stream(like)))
    return out


def top_plan_query(batch: int, ny: int, nx: int, dy: float, dx: float, pad: float = 2.0, method="as"):
    """(Py, Px, workspace bytes per field); host only, no GPU needed."""
    g = make_grid(batch, ny, nx, dy, dx, pad, method)
    py, px, ws = C.c_int64(), C.c_int64(), C.c_uint64()
    check(_lib.load().top_plan_query(C.byref(g), C.byref(py), C.byref(px), C.byref(ws)))
    return py.value, px.value, ws.value


def top_zcritical(L: float, dx: float, lam: float) -> float:
    return _lib.load().top_zcritical(L, dx, lam)


def profile_enable(enable: bool = True, device=None) -> None:
    check(_lib.load().top_profile_enable(handle(device), 1 if enable else 0))


def profile_read(device=None) -> dict:
    """{kernel kind: (milliseconds, launches)} accumulated since the last read (synchronises)."""
    cap = 8
    kinds = (C.c_char_p * cap)()
    ms = (C.c_double * cap)()
    cnt = (C.c_int64 * cap)()
    n = C.c_int()
    check(_lib.load().top_profile_read(handle(device), cap, kinds, ms, cnt, C.byref(n)))
    return {kinds[i].decode(): (ms[i], cnt[i]) for i in range(n.value)}


# ----------------------------------------------------------------------------- autotuning

def top_autotune(batch: int, ny: int, nx: int, dy: float, dx: float, pad: float = 2.0, method="as",
                 device=None):
    """Measure the pass variants on this geometry (``batch`` scratch fields) and record the fastest
    in the process-wide table; returns (row flags of Px/2, column flags of Py/2)."""
    g = make_grid(batch, ny, nx, dy, dx, pad, method)
    rf, cf = C.c_uint32(), C.c_uint32()
    check(_lib.load().top_autotune(handle(device), C.byref(g), C.byref(rf), C.byref(cf)))
    return rf.value, cf.value


def autotune_set(line_length: int, flags: int) -> None:
    check(_lib.load().top_autotune_set(int(line_length), int(flags)))


def autotune_get(line_length: int) -> int:
    v = C.c_uint32()
    check(_lib.load().top_autotune_get(int(line_length), C.byref(v)))
    return v.value


def autotune_clear() -> None:
    check(_lib.load().top_autotune_clear())


def autotune_save(path: str) -> None:
    check(_lib.load().top_autotune_save(str(path).encode()))


def autotune_load(path: str) -> None:
    check(_lib.load().top_autotune_load(str(path).encode()))
