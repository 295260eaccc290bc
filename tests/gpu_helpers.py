"""Shared helpers of the GPU parity tests (no spline arithmetic of their own)."""
import numpy as np

import oracle

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "bf16": 1e-2}
NONORTHO = np.array([[5.0, 1.0, 0.5],
                     [0.0, 6.0, 0.3],
                     [0.0, 0.0, 7.0]])


def dev():
    import torch
    return torch.device("cuda", 0)


def splines(*a, **k):
    from paper_1309_6250_gb300.api import OrbitalSplines
    return OrbitalSplines(*a, device=dev(), **k)


def rounded(a, storage):
    """A table as the GPU stores it, back in float64 (the oracle's single round-to-nearest-even)."""
    return oracle.round_to_storage(a, storage)


def gpu_eval(spl, pos):
    import torch
    v, g, l = spl.eval_vgl(torch.from_numpy(np.ascontiguousarray(pos)).to(dev()))
    spl.sync()
    return v.double().cpu().numpy(), g.double().cpu().numpy(), l.double().cpu().numpy()


def assert_parity(got, ref, tol, what=""):
    errs = [oracle.relative_error(g, r) for g, r in zip(got, ref)]
    for n, e in zip(("val", "grad", "lap"), errs):
        assert e <= tol, "%s %s: relative error %.3e > %.1e" % (what, n, e, tol)
    return errs


def oracle_tables(lat, mil, coef, dims, method="smooth", storage="f64", sep=False, separate_grad=False,
                  kpoint=None, degree=3, knots=None):
    """The tables a handle with these options stores, built by the oracle from the planewave
    coefficients (never read back from the GPU) and rounded the way the GPU stores them (FP32,
    BF16; FP64 and double-float as they are: a double-float pair holds the FP64 value to about
    2^-48).  Laid out as get_table gives them: (beta, beta_lap or None) for B-splines, one
    stacked [5, ...] array for five-table handles, [8, ...] for pp; Bloch tables interleaved."""
    if degree != 3 or knots is not None:
        kn = knots if knots is not None else (None, None, None)
        if method == "smooth":
            tabs = oracle.smoothing_tables_degree(lat, mil, coef, dims, degree, laplacian=sep)
        else:
            tabs = oracle.general_interp_tables(lat, mil, coef, dims, degree, kn, laplacian=sep, kpoint=kpoint)
    elif kpoint is not None:
        tabs = oracle.bloch_tables(method, lat, mil, coef, kpoint, dims, laplacian=sep, gradient=separate_grad)
    elif separate_grad:
        tabs = oracle.derivative_tables(method, lat, mil, coef, dims)
    elif method == "lagrange":
        tabs = oracle.lagrange_tables(lat, mil, coef, dims)
    elif method == "pp":
        tabs = oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims))
    elif method == "smooth":
        tabs = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=sep)
    else:
        tabs = oracle.interpolating_tables(lat, mil, coef, dims, laplacian=sep)
    if isinstance(tabs, tuple):
        return tuple(rounded(x, storage) for x in tabs)
    return rounded(tabs, storage)
