"""A stack of trainable phase masks with free-space propagation after each (a diffractive network,
§4 and Listing 2), trained through its detector intensity, with per-layer checkpoints.

Layer k (k = 1 .. K) multiplies the field by exp(i phi_k) (Eq. 1) and propagates it by z_k (Eq. 4):
x_k = P_{z_k}(exp(i phi_k) x_{k-1}); the detector sees I = |x_K|^2, summed over each `group` of
consecutive fields (Eq. 14). The gradient of phi_k needs the layer's input x_{k-1}. With
``checkpoint_every = c`` the forward keeps x_j only for j a multiple of c (x_0 is the caller's
input), and the backward recomputes the others from the nearest kept plane, one segment of at
most c - 1 planes at a time, when it reaches them: the gradients are the same bit for bit as
with every plane kept (c = 1), for K - 1 - floor((K - 1) / c) fewer stored planes and at most
c - 1 recomputed ones alive at once.

A sequence of library calls (a fused chain forward, intensity and propagation backwards), no
arithmetic of its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from . import binding as B


@dataclass
class StackState:
    """What the forward leaves for the backward."""
    x0: torch.Tensor
    xK: torch.Tensor
    kept: dict = field(default_factory=dict)  # layer output index j -> x_j
    every: int = 1

    def planes_held(self) -> int:
        """Field planes held for the backward besides the input: the last field and the kept ones."""
        return 1 + len(self.kept)


@dataclass
class MaskStack:
    d: float
    lam: object
    zs: Sequence[float]
    pad: float = 2.0
    method: str = "as"

    def _stage(self, phases: torch.Tensor, k: int, keep: Optional[torch.Tensor] = None) -> B.Stage:
        return B.Stage(float(self.zs[k - 1]), pre=B.Modulation(phase=phases[k - 1]), keep=keep)

    def forward(self, x0: torch.Tensor, phases: torch.Tensor, group: int = 1, checkpoint_every: int = 1):
        """Returns (intensity [batch / group, ny, nx], state)."""
        K = len(self.zs)
        c = int(checkpoint_every)
        if c < 1:
            raise ValueError("checkpoint_every must be >= 1")
        kept = {j: torch.empty_like(x0) for j in range(c, K, c)}
        stages = [self._stage(phases, k, kept.get(k)) for k in range(1, K + 1)]
        xK, inten = B.top_fused_chain(x0, self.d, self.d, self.lam, stages, self.pad, self.method,
                                      intensity_group=group)
        return inten, StackState(x0=x0, xK=xK, kept=kept, every=c)

    def _segment(self, st: StackState, phases: torch.Tensor, j: int) -> dict:
        """x_{c0+1} .. x_j recomputed from the kept x_{c0} (c0 the last multiple of the checkpoint
        interval below j), through one fused chain."""
        c0 = (j // st.every) * st.every
        base = st.x0 if c0 == 0 else st.kept[c0]
        seg = {i: torch.empty_like(base) for i in range(c0 + 1, j)}
        stages = [self._stage(phases, k, seg.get(k)) for k in range(c0 + 1, j + 1)]
        seg[j], _ = B.top_fused_chain(base, self.d, self.d, self.lam, stages, self.pad, self.method)
        return seg

    def backward(self, st: StackState, phases: torch.Tensor, grad_intensity: torch.Tensor, group: int = 1,
                 want_grad_in: bool = False):
        """Gradients of every layer's phase ([K, ny, nx]) and, if asked, of the input field."""
        K = len(self.zs)
        grads = torch.empty_like(phases)
        seg: dict = {}
        g = None
        for k in range(K, 0, -1):
            j = k - 1
            if j == 0:
                xin = st.x0
            elif j in st.kept:
                xin = st.kept[j]
            else:
                if j not in seg:
                    seg = self._segment(st, phases, j)
                xin = seg[j]
            pre = B.Modulation(phase=phases[k - 1])
            need_in = k > 1 or want_grad_in
            if k == K:
                g = B.top_propagate_intensity_backward(st.xK, grad_intensity, self.d, self.d, self.lam,
                                                       float(self.zs[k - 1]), self.pad, self.method, group=group,
                                                       pre=pre, saved_in=xin, want_grad_in=need_in,
                                                       grad_phase=grads[k - 1])
            else:
                g = B.top_propagate_backward(g, self.d, self.d, self.lam, float(self.zs[k - 1]), self.pad,
                                             self.method, pre=pre, saved_in=xin, want_grad_in=need_in,
                                             grad_phase=grads[k - 1])
        return grads, g
