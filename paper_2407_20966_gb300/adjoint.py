"""Reverse mode of the limited SSP-RK3 integration, as torch.autograd.Functions.

Every step of the forward and reverse passes runs in libkbl's CUDA kernels
(kbl_step_fixed, kbl_adjoint_segment, kbl_entropy, kbl_entropy_vjp); this module
only sequences the calls and keeps the checkpoints.

* :func:`trajectory` -- w(t_end) from w0 through fixed time steps ``dts`` (take them
  from :func:`cfl_time_steps`).  Checkpointing: the forward pass keeps every
  ``checkpoint_every``-th state (and, by default, every stage's bounds); the backward
  pass runs kbl_adjoint_segment once per segment, which recomputes the segment's states
  and walks them backwards.
* :func:`entropy` -- the integrated entropy sum |J_e| W_n rho ln(P rho^-gamma).

The time steps are held fixed in the derivative (the CFL rule is not differentiated).
Subgradients at ties of the method's min / max operations follow the rule stated in
include/kbl.h (the first element in the natural order wins).
"""
from __future__ import annotations

import torch

from . import kbl


def cfl_time_steps(kctx: "kbl.Context", w0: torch.Tensor, n_steps: int, cfl: float) -> list:
    """The time steps of n_steps CFL-limited steps from w0 (runs the forward pass once)."""
    w = w0.detach().clone()
    dt_dev = torch.zeros(1, dtype=torch.float64, device=w.device)
    dts = []
    for _ in range(n_steps):
        kctx.dt(w, cfl, dt_dev)
        dt = float(dt_dev.item())
        kctx.step_fixed(w, dt)
        dts.append(dt)
    kctx.check()
    return dts


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(fctx, w0, kctx, dts, every, keep_bounds):
        w = w0.detach().clone()
        n = len(dts)
        segs = []
        for a in range(0, n, every):
            seg = dts[a:a + every]
            bnd = None
            if keep_bounds:
                bnd = torch.empty((len(seg), 3, 2, kctx.nv, kctx.E), dtype=torch.float64, device=w.device)
            segs.append((w.clone(), seg, bnd))
            kctx.forward_segment(w, seg, bnd)
        fctx.kctx, fctx.segs = kctx, segs
        return w

    @staticmethod
    def backward(fctx, wbar):
        g = wbar.detach().contiguous().clone()
        for ckpt, seg, bnd in reversed(fctx.segs):
            fctx.kctx.adjoint_segment(ckpt, seg, g, bnd)
        fctx.segs = None
        return g, None, None, None, None


def trajectory(w0: torch.Tensor, kctx: "kbl.Context", dts, checkpoint_every: int = 10,
               keep_bounds: bool = True) -> torch.Tensor:
    """The state after len(dts) fixed-dt steps from w0, differentiable in w0.

    Every ``checkpoint_every``-th state is kept; with ``keep_bounds`` the stage bounds of every
    step are kept too (8 values per element and stage, an eighth of a P3 state), so that the
    backward pass does not recompute them."""
    if checkpoint_every < 1:
        raise ValueError("checkpoint_every must be >= 1")
    return _Trajectory.apply(w0, kctx, list(dts), int(checkpoint_every), bool(keep_bounds))


class _Entropy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, w, kctx):
        J = torch.zeros(1, dtype=torch.float64, device=w.device)
        kctx.entropy(w.detach(), J)
        fctx.save_for_backward(w)
        fctx.kctx = kctx
        return J[0]

    @staticmethod
    def backward(fctx, Jb):
        (w,) = fctx.saved_tensors
        g = torch.empty_like(w)
        fctx.kctx.entropy_vjp(w.detach(), float(Jb), g)
        return g, None


def entropy(w: torch.Tensor, kctx: "kbl.Context") -> torch.Tensor:
    """Integrated entropy sum |J_e| W_n rho ln(P rho^-gamma) of w (a 0-dim tensor), differentiable in w."""
    return _Entropy.apply(w, kctx)
