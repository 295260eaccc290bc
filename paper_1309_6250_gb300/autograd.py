"""torch.autograd binding of the spline evaluation and its hand-written adjoint.

    beta, beta_lap = spl.coefficient_parameters()      # leaf tensors, requires_grad
    val, grad, lap = evaluate(spl, pos, beta, beta_lap)
    loss = f(val, grad, lap); loss.backward()
    # pos.grad: dL/dr [P, 3] (forces);  beta.grad, beta_lap.grad: dL/dbeta (canonical
    # layout [Nx, Ny, Nz, O]), both from qmcspl_eval_vgl_backward.

The forward pass evaluates the coefficient tables held by the handle.  `beta` / `beta_lap`
are those tables in the autograd graph: whenever a tensor passed as `beta` or `beta_lap`
differs from the one last uploaded to the handle (another tensor, or the same tensor changed
in place since, e.g. by an optimiser step: torch's version counter), forward first writes it
into the handle's tables (qmcspl_set_table, with the storage type's rounding).  So

    opt = torch.optim.SGD([beta], lr=...)
    for _ in range(n):
        opt.zero_grad(); loss(evaluate(spl, pos, beta)).backward(); opt.step()

optimises the orbitals' coefficients.  Stencil weights are recomputed in the backward kernel
rather than saved.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from .api import OrbitalSplines


def _is_table(t) -> bool:
    return t is not None and t.dim() >= 4


def upload_if_changed(spl: OrbitalSplines, index: int, t: torch.Tensor) -> None:
    """Write `t` into table `index` of the handle unless it is the tensor, at the version, that
    was written last."""
    key = (t.data_ptr(), t._version, tuple(t.shape), t.dtype)
    seen = spl.__dict__.setdefault("_uploaded", {})
    if seen.get(index) != key:
        spl.set_table(index, t)
        seen[index] = key


def sync_tables(spl: OrbitalSplines, beta, beta_lap) -> None:
    """Upload the coefficient tensors of the autograd graph that changed since the last upload:
    beta [Nx, Ny, Nz, F] is table 0 (beta_lap table 1); a stacked [5 or 8, Nx, Ny, Nz, F] beta
    holds every table of a five-table or pp handle."""
    shape = spl.coef_shape()
    if _is_table(beta):
        if tuple(beta.shape) == shape:
            upload_if_changed(spl, 0, beta)
        else:
            for i in range(beta.shape[0]):
                upload_if_changed(spl, i, beta[i])
    if _is_table(beta_lap):
        upload_if_changed(spl, 1, beta_lap)


class SplineOrbitalFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, beta, beta_lap, spl: OrbitalSplines):
        sync_tables(spl, beta, beta_lap)
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
    layout [Nx, Ny, Nz, O], in the output dtype: (beta, beta_lap or None).  They are recorded
    as the handle's current tables (nothing is uploaded until one of them changes).  Five-table
    handles (Lagrange, B-splines with separate gradient tables) give all five tables as one
    [5, Nx, Ny, Nz, O] tensor and None, pp handles their eight entries as [8, Nx, Ny, Nz, O]."""
    inf = spl.info()
    n_multi = 5 if inf["n_tables"] == 5 else (8 if inf["entries_per_point"] == 8 else 0)
    seen = spl.__dict__.setdefault("_uploaded", {})
    if n_multi:
        t = torch.from_numpy(np.stack([spl.get_table(i) for i in range(n_multi)]))
        t = t.to(device=spl.device, dtype=spl.out_dtype).requires_grad_(True)
        for i in range(n_multi):
            v = t[i]
            seen[i] = (v.data_ptr(), v._version, tuple(v.shape), v.dtype)
        return t, None
    out = []
    for idx in range(2):
        if idx == 1 and not inf["separate_lap"]:
            out.append(None)
            continue
        t = torch.from_numpy(spl.get_table(idx)).to(device=spl.device, dtype=spl.out_dtype)
        t.requires_grad_(True)
        seen[idx] = (t.data_ptr(), t._version, tuple(t.shape), t.dtype)
        out.append(t)
    return tuple(out)


def evaluate(spl: OrbitalSplines, pos: torch.Tensor, beta: Optional[torch.Tensor] = None,
             beta_lap: Optional[torch.Tensor] = None):
    """(val, grad, lap) with autograd to positions and (if given) coefficients."""
    if beta is None:
        beta = torch.zeros((), device=spl.device)   # no coefficient gradient requested
    if beta_lap is None:
        beta_lap = torch.zeros((), device=spl.device)
    return SplineOrbitalFunction.apply(pos, beta, beta_lap, spl)
