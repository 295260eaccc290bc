"""torch.autograd binding of the spline evaluation and its hand-written adjoint.

    beta, beta_lap = spl.coefficient_parameters()      # leaf tensors, requires_grad
    val, grad, lap = evaluate(spl, pos, beta, beta_lap)
    loss = f(val, grad, lap); loss.backward()
    # pos.grad: dL/dr [P, 3] (forces);  beta.grad, beta_lap.grad: dL/dbeta (canonical
    # layout [Nx, Ny, Nz, O]), both from qmcspl_eval_vgl_backward.

The forward pass reads the coefficient tables held by the handle; `beta` / `beta_lap`
stand for those tables in the autograd graph (they must hold the same values, which
is what coefficient_parameters() returns).  Stencil weights are recomputed in the
backward kernel rather than saved.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from .api import OrbitalSplines


class SplineOrbitalFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, beta, beta_lap, spl: OrbitalSplines):
        val, grad, lap = spl.eval_vgl(pos)
        ctx.spl = spl
        ctx.save_for_backward(pos)
        return val, grad, lap

    @staticmethod
    def backward(ctx, gv, gg, gl):
        spl: OrbitalSplines = ctx.spl
        (pos,) = ctx.saved_tensors
        need_pos = ctx.needs_input_grad[0]
        need_coef = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        inf = spl.info()
        # Lagrange and B-splines with separate gradient tables: five tables; pp: eight entries
        n_multi = 5 if inf["n_tables"] == 5 else (8 if inf["entries_per_point"] == 8 else 0)
        sep = bool(inf["separate_lap"]) and not n_multi
        dcoef = dcoef_lap = None
        if need_coef:
            shape = ((n_multi,) if n_multi else ()) + spl.coef_shape()
            dcoef = torch.zeros(shape, dtype=spl.out_dtype, device=spl.device)
            if sep:
                dcoef_lap = torch.zeros_like(dcoef)
        dpos = None
        if need_pos or need_coef:
            dpos = spl.backward(pos, gv, gg, gl, dcoef=dcoef, dcoef_lap=dcoef_lap, want_dpos=need_pos)
        return (dpos if need_pos else None, dcoef if ctx.needs_input_grad[1] else None,
                dcoef_lap if ctx.needs_input_grad[2] else None, None)


def coefficient_parameters(spl: OrbitalSplines):
    """Leaf tensors (requires_grad) holding the handle's coefficient tables in canonical
    layout [Nx, Ny, Nz, O], in the output dtype: (beta, beta_lap or None).  Five-table
    handles (Lagrange, B-splines with separate gradient tables) give all five tables as one
    [5, Nx, Ny, Nz, O] tensor and None, pp handles their eight entries as [8, Nx, Ny, Nz, O]."""
    inf = spl.info()
    n_multi = 5 if inf["n_tables"] == 5 else (8 if inf["entries_per_point"] == 8 else 0)
    if n_multi:
        t = torch.from_numpy(np.stack([spl.get_table(i) for i in range(n_multi)]))
        return t.to(device=spl.device, dtype=spl.out_dtype).requires_grad_(True), None
    out = []
    for idx in range(2):
        if idx == 1 and not inf["separate_lap"]:
            out.append(None)
            continue
        t = torch.from_numpy(spl.get_table(idx)).to(device=spl.device, dtype=spl.out_dtype)
        out.append(t.requires_grad_(True))
    return tuple(out)


def evaluate(spl: OrbitalSplines, pos: torch.Tensor, beta: Optional[torch.Tensor] = None,
             beta_lap: Optional[torch.Tensor] = None):
    """(val, grad, lap) with autograd to positions and (if given) coefficients."""
    if beta is None:
        beta = torch.zeros((), device=spl.device)   # no coefficient gradient requested
    if beta_lap is None:
        beta_lap = torch.zeros((), device=spl.device)
    return SplineOrbitalFunction.apply(pos, beta, beta_lap, spl)
