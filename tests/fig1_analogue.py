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
the oracle's direct planewave sum (CPU, FP64).  With --oracle the approximations come from
the oracle as well (no GPU needed).

    python tests/fig1_analogue.py [--storage f32] [--ecut 10 15 20 30 40] [--oracle]
"""
from __future__ import annotations

import argparse
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


def degree_table(rows: List[Dict]) -> str:
    out = ["| Ecut (Ha) | N | degree | value | grad | lap (Hessian) | lap (separate table) |",
           "|---|---|---|---|---|---|---|"]
    for r in rows:
        out.append("| %g | %d | %s | %.2e | %.2e | %.2e | %.2e |" % (r["ecut"], r["dims"][0], r["row"][6:],
                                                                  r["value"], r["grad"], r["lap"], r["lap_sep"]))
    return "\n".join(out)


def table(rows: List[Dict]) -> str:
    """Markdown: one table per quantity, cutoffs down, rows of ROWS across."""
    out = []
    for what in ("value", "grad", "lap"):
        out += ["", "%s:" % what, "",
                "| Ecut (Ha) | N | PWs | " + " | ".join(r[0] for r in ROWS) + " |",
                "|---|---|---|" + "---|" * len(ROWS)]
        for ecut in sorted({r["ecut"] for r in rows}):
            rs = {r["row"]: r for r in rows if r["ecut"] == ecut}
            first = next(iter(rs.values()))
            out.append("| %g | %d | %d | " % (ecut, first["dims"][0], first["n_pw"]) +
                       " | ".join("%.2e" % rs[lab][what] for lab, _, _ in ROWS) + " |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--storage", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--ecut", type=float, nargs="*", default=list(ECUTS))
    ap.add_argument("--oracle", action="store_true", help="approximations from the oracle (no GPU)")
    ap.add_argument("--degrees", action="store_true",
                    help="also tabulate interpolating B-splines of degree 1, 3, 5, 7 (GPU)")
    args = ap.parse_args()
    device = None
    if not args.oracle:
        import torch
        device = torch.device("cuda", 0)
    rows = run(args.ecut, args.storage, args.oracle, device=device)
    print("approximations: %s%s" % ("oracle" if args.oracle else "GPU", "" if args.oracle else " " + args.storage))
    print(table(rows))
    if args.degrees and not args.oracle:
        print("\ninterpolating B-splines by degree (GPU %s):\n" % args.storage)
        print(degree_table(run_degrees(args.ecut, storage=args.storage, device=device)))


if __name__ == "__main__":
    main()
