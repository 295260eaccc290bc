"""Synthetic analogue of Fig. 1 (Sec. III A): relative mean absolute error of the orbital,
its gradient and its Laplacian against the planewave sum, as a function of the planewave
cutoff at the natural grid spacing h = pi / G_max (Eq. natural_spacing), for the four
methods, with derivatives of the approximation ("der") and with separate approximations
of the gradient and Laplacian ("sep", Sec. III C).

Workload (a stand-in for the paper's LDA orbitals of rock-salt MgO, which are not
available): the 8-atom conventional cubic cell of MgO, a = 7.96 bohr; 16 real synthetic
orbitals per cutoff from the seeded generator (c_G ~ N(0,1) exp(-|G|^2/8) over the cutoff
sphere, the MgO-like decay of the workload recipe); 2000 uniform positions.

The approximations are evaluated by the GPU library through its C ABI; the reference is
the oracle's direct planewave sum (CPU, FP64).  With use_oracle=True the approximations come
from the oracle as well (no GPU needed).  tests/test_fig1_analogue.py runs both.
"""
from __future__ import annotations

import math
import os
import sys
from typing import Dict, List, Sequence

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1309_6250_gb300 import inputs  # noqa: E402

A_MGO = 7.96          # bohr, conventional rock-salt cell of MgO
DECAY = 8.0           # c_G envelope exp(-|G|^2 / DECAY)
ECUTS = (10.0, 15.0, 20.0, 30.0, 40.0)
# (row label, method, separate approximations)
ROWS = (("lagrange", "lagrange", True), ("pp", "pp", False), ("interp", "interp", False),
        ("interp_sep", "interp", True), ("smooth", "smooth", False), ("smooth_sep", "smooth", True))


def natural_dims(lattice: np.ndarray, ecut: float) -> tuple:
    """Grid points per lattice vector at the natural spacing h = pi / sqrt(2 Ecut)."""
    h = math.pi / math.sqrt(2.0 * ecut)
    return tuple(max(4, int(math.ceil(np.linalg.norm(lattice[:, i]) / h))) for i in range(3))


def workload(ecut: float, n_orb: int = 16, n_pos: int = 2000, seed: int = 1001):
    lat = np.eye(3) * A_MGO
    mil = inputs.miller_set(lat, ecut)
    coef = inputs.pw_coefficients(lat, mil, n_orb, DECAY, seed)
    pos = inputs.positions(lat, n_pos, seed + 1)
    return lat, mil, coef, pos


def _oracle_outputs(method, sep, lat, mil, coef, dims, pos):
    if method == "lagrange":
        return oracle.lagrange_eval(oracle.lagrange_tables(lat, mil, coef, dims), lat, pos)
    if method == "pp":
        return oracle.pp_eval(oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims)), lat, pos)
    if sep:
        return oracle.bspline_eval_separate(oracle.derivative_tables(method, lat, mil, coef, dims), lat, pos)
    tb = oracle.smoothing_tables if method == "smooth" else oracle.interpolating_tables
    beta, _ = tb(lat, mil, coef, dims)
    return oracle.bspline_eval(beta, lat, pos)


def _gpu_outputs(method, sep, lat, mil, coef, dims, pos, storage, device):
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    spl = OrbitalSplines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep,
                         separate_grad=sep and method in ("smooth", "interp"), device=device)
    v, g, l = spl.eval_vgl(torch.from_numpy(np.ascontiguousarray(pos)).to(device))
    spl.sync()
    out = tuple(x.double().cpu().numpy() for x in (v, g, l))
    spl.close()
    return out


def run(ecuts: Sequence[float] = ECUTS, storage: str = "f64", use_oracle: bool = False,
        n_orb: int = 16, n_pos: int = 2000, device=None) -> List[Dict]:
    """One dict per (cutoff, row): relative MAE of value, gradient and Laplacian."""
    rows = []
    for ecut in ecuts:
        lat, mil, coef, pos = workload(ecut, n_orb, n_pos)
        dims = natural_dims(lat, ecut)
        pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
        for label, method, sep in ROWS:
            if use_oracle:
                v, g, l = _oracle_outputs(method, sep, lat, mil, coef, dims, pos)
            else:
                v, g, l = _gpu_outputs(method, sep, lat, mil, coef, dims, pos, storage, device)
            m = oracle.relative_mean_absolute_error
            rows.append({"ecut": ecut, "dims": dims, "n_pw": int(mil.shape[0]), "row": label,
                         "value": m(v, pv), "grad": m(g, pg), "lap": m(l, pl)})
    return rows


def run_degrees(ecuts: Sequence[float] = ECUTS, degrees: Sequence[int] = (1, 3, 5, 7), storage: str = "f64",
                n_orb: int = 16, n_pos: int = 2000, device=None) -> List[Dict]:
    """Relative MAE of interpolating B-splines of each odd degree at the natural spacing
    (derivatives of the spline; the Laplacian from a separate table and from the Hessian)."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    rows = []
    for ecut in ecuts:
        lat, mil, coef, pos = workload(ecut, n_orb, n_pos)
        dims = natural_dims(lat, ecut)
        pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
        m = oracle.relative_mean_absolute_error
        for deg in degrees:
            res = {"ecut": ecut, "dims": dims, "n_pw": int(mil.shape[0]), "row": "degree%d" % deg}
            for sep in (False, True):
                spl = OrbitalSplines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=sep,
                                     degree=deg, device=device)
                v, g, l = (x.double().cpu().numpy() for x in spl.eval_vgl(torch.from_numpy(pos).to(device)))
                spl.sync()
                spl.close()
                if not sep:
                    res.update(value=m(v, pv), grad=m(g, pg), lap=m(l, pl))
                else:
                    res["lap_sep"] = m(l, pl)
            rows.append(res)
    return rows
