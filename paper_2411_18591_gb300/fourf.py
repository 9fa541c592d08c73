"""Polarised, polychromatic 4f imaging system with a trainable pupil phase (Fig. 1, Listing 5).

A sequence of library calls, no arithmetic of its own:

  F1  psi1 = lens1 * P_f(obj)               (object broadcast over the wavelengths, input_repeat)
  F2  psi2 = P_f(psi1)                       (kept for the pupil gradient)
  F3  psi3 = lens2 * P_f(pupil * psi2)       (pupil = circ(R) exp(i phi))
  F4  psi4 = P_f(psi3), I = sum over each object's component and wavelength fields of |psi4|^2 (Eq. 14)
      (F1-F4 run as one fused chain: the row passes between consecutive propagations are one kernel)
  L   = mean((I - T)^2), dL/dI
  B4  g3 = P_f^H(2 dL/dI psi4)               (intensity backward)
  B3  dL/dphi = sum_b Im(g_y conj(pupil psi2)),  g_y = P_f^H(conj(lens2) g3)
      (B4-B3 run as one fused backward chain: the row passes between the two adjoint
      propagations are one kernel)

Fields are ordered (object, component, wavelength), so each object's fields are
consecutive (one intensity group) and each (object, component) input feeds its
consecutive wavelength fields. Four forward and two backward propagations per
field per step.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B


@dataclass
class FourF:
    n: int = 1024
    d: float = 5e-6
    f: float = 0.2
    lens_radius: float = 2.56e-3
    pupil_radius: float = 1.0e-3
    objects: int = 16
    comps: int = 3
    wavelengths: tuple = ()
    pad: float = 2.0
    method: str = "as"

    @property
    def repeat(self) -> int:
        return len(self.wavelengths)

    @property
    def batch(self) -> int:
        return self.objects * self.comps * self.repeat

    @property
    def group(self) -> int:
        return self.comps * self.repeat

    def field_lambdas(self):
        return list(self.wavelengths) * (self.objects * self.comps)

    FWD_PROPS = 4
    BWD_PROPS = 2

    def lens(self) -> B.Modulation:
        return B.Modulation(focal_length=self.f, radius=self.lens_radius)

    def pupil(self, phase: torch.Tensor) -> B.Modulation:
        return B.Modulation(phase=phase, radius=self.pupil_radius)

    def _forward(self, obj, phase, target, buffers):
        lam = self.field_lambdas()
        d, f, pad, m = self.d, self.f, self.pad, self.method
        bufs = buffers if buffers is not None else {}
        shape = (self.batch, self.n, self.n)
        if "a" not in bufs:
            bufs["a"] = torch.empty(shape, dtype=torch.complex64, device=obj.device)
            bufs["b"] = torch.empty(shape, dtype=torch.complex64, device=obj.device)
        a, b = bufs["a"], bufs["b"]
        lens, pupil = self.lens(), self.pupil(phase)
        # F1-F4 as one fused chain: psi2 kept in a, psi4 and the grouped intensity out of the last stage
        stages = [B.Stage(f), B.Stage(f, pre=lens, keep=a), B.Stage(f, pre=pupil), B.Stage(f, pre=lens)]
        _, inten = B.top_fused_chain(obj, d, d, lam, stages, pad, m, out=b, intensity_group=self.group,
                                     input_repeat=self.repeat)
        loss, g_i = B.top_mse_loss(inten, target)
        return lam, a, b, inten, loss, g_i, lens, pupil

    def step(self, obj: torch.Tensor, phase: torch.Tensor, target: torch.Tensor, grad_phase: torch.Tensor,
             buffers: dict | None = None):
        """One forward + backward pass; returns (loss device scalar, intensity). grad_phase is overwritten."""
        lam, a, b, inten, loss, g_i, lens, pupil = self._forward(obj, phase, target, buffers)
        # B4-B3: the backward of the last two stages, from psi4 (in b) to the pupil's phase gradient
        B.top_fused_chain_backward(b, g_i, self.d, self.d, lam, [B.Stage(self.f, pre=pupil), B.Stage(self.f, pre=lens)],
                                   self.pad, self.method, intensity_group=self.group, saved_in=a,
                                   want_grad_in=False, grad_phase=grad_phase)
        return loss, inten

    def step_unfused_backward(self, obj: torch.Tensor, phase: torch.Tensor, target: torch.Tensor,
                              grad_phase: torch.Tensor, buffers: dict | None = None):
        """``step`` with the backward as two separate calls (intensity backward, then propagation
        backward through the pupil): the same results, for comparison."""
        lam, a, b, inten, loss, g_i, lens, pupil = self._forward(obj, phase, target, buffers)
        _intensity_backward_into(b, g_i, b, self, lam)                                                # B4 (g3 in b)
        B.top_propagate_backward(b, self.d, self.d, lam, self.f, self.pad, self.method, pre=pupil, post=lens,
                                 saved_in=a, want_grad_in=False, grad_phase=grad_phase)               # B3
        return loss, inten


def _intensity_backward_into(psi, g_i, grad_in, sysm: FourF, lam):
    import ctypes as C
    from . import _lib
    b, ny, nx = psi.shape
    lams, zs, n = B._lz(lam, sysm.f, b)
    g = B.make_grid(b, ny, nx, sysm.d, sysm.d, sysm.pad, sysm.method)
    _lib.check(_lib.load().top_propagate_intensity_backward(B.handle(psi.device), C.byref(g), psi.data_ptr(),
                                                            g_i.data_ptr(), grad_in.data_ptr(), sysm.group, None,
                                                            lams, zs, n, None, None, None, B._stream(psi)))
    return grad_in
