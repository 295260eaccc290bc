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
    import torch
    if a is None or storage in ("f64", "df64"):
        return a
    if storage == "f32":
        return a.astype(np.float32).astype(np.float64)
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).double().numpy()


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
