"""GPU parity of B-spline construction and evaluation against the FP64 oracle.

Tolerances (max |gpu - oracle| / max |oracle|, per output): 1e-12 for FP64 tables,
2e-6 for FP32 tables and 1e-2 for BF16 tables (FP32 accumulation).  Tables are
compared after the same rounding to the stored type.
"""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "bf16": 1e-2}
NONORTHO = np.array([[5.0, 1.0, 0.5],
                     [0.0, 6.0, 0.3],
                     [0.0, 0.0, 7.0]])


def dev():
    return torch.device("cuda", 0)


def splines(*a, **k):
    from paper_1309_6250_gb300.api import OrbitalSplines
    return OrbitalSplines(*a, device=dev(), **k)


def oracle_tables(method, lattice, miller, coef, dims, sep):
    if method == "smooth":
        return oracle.smoothing_tables(lattice, miller, coef, dims, laplacian=sep)
    return oracle.interpolating_tables(lattice, miller, coef, dims, laplacian=sep)


def rounded(a, storage):
    return oracle.round_to_storage(a, storage)


def gpu_eval(spl, pos):
    v, g, l = spl.eval_vgl(torch.from_numpy(np.ascontiguousarray(pos)).to(dev()))
    spl.sync()
    return v.double().cpu().numpy(), g.double().cpu().numpy(), l.double().cpu().numpy()


def assert_parity(got, ref, tol, what=""):
    names = ("val", "grad", "lap")
    errs = [oracle.relative_error(g, r) for g, r in zip(got, ref)]
    for n, e in zip(names, errs):
        assert e <= tol, "%s %s: relative error %.3e > %.1e" % (what, n, e, tol)
    return errs


@pytest.mark.parametrize("method", ["smooth", "interp"])
@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
def test_tables_match_oracle(method, storage):
    """Construction (frequency grid, symbol division, inverse DFT, layout) against the
    oracle's tables: FP64 to 1e-13, lower precisions to their rounding."""
    dims = (10, 12, 14)
    lat, mil, coef = inputs.random_cell(21, dims, 7, 9.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=True)
    beta, blap = oracle_tables(method, lat, mil, coef, dims, True)
    for idx, ref in ((0, beta), (1, blap)):
        got = spl.get_table(idx)
        tol = {"f64": 1e-13, "df64": 1e-13, "f32": 1e-7, "bf16": 8e-3}[storage]
        assert oracle.relative_error(got, ref) <= tol
    info = spl.info()
    assert info["n_tables"] == 2 and info["table_bytes"] > 0


def test_c1_fp64_interpolating_16cube():
    """FP64 interpolating B-spline, cubic a = 10.26 bohr, 16^3 grid, 8 orbitals with
    |G|^2/2 <= 15 Ha (aliasing at n = 8 = N/2), 1000 uniform positions."""
    w = inputs.make_workload("c1")
    dims = w.cell.grid
    spl = splines(w.lattice, dims, w.miller, w.coef, method="interp", storage="f64",
                  separate_lap=False)
    beta, _ = oracle.interpolating_tables(w.lattice, w.miller, w.coef, dims)
    ref = oracle.bspline_eval(beta, w.lattice, w.pos)
    got = gpu_eval(spl, w.pos)
    assert_parity(got, ref, TOL["f64"], "c1")
    # the interpolant reproduces the planewave sum at the grid points
    idx = np.stack(np.meshgrid(*[np.arange(0, d, 3) for d in dims], indexing="ij"), -1).reshape(-1, 3)
    gp = (idx / np.array(dims)) @ w.lattice.T
    pv, _, _, _ = oracle.pw_eval(w.lattice, w.miller, w.coef, gp)
    assert oracle.relative_error(gpu_eval(spl, gp)[0], pv) < 1e-12


@pytest.mark.parametrize("method", ["smooth", "interp"])
@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
@pytest.mark.parametrize("sep", [False, True])
@pytest.mark.parametrize("n_orb", [1, 3, 13, 40])
def test_eval_ragged_nonorthogonal(method, storage, sep, n_orb):
    """Non-orthogonal cell, unequal grid, orbital counts that leave ragged rows, positions
    inside and outside the cell (wrapped, Eq. reducedcoordinate), P not a multiple of
    anything."""
    dims = (9, 11, 13)
    lat, mil, coef = inputs.random_cell(100 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep)
    beta, blap = oracle_tables(method, lat, mil, coef, dims, sep)
    beta = rounded(beta, storage)
    blap = None if blap is None else rounded(blap, storage)
    pos = np.vstack([inputs.positions(lat, 301, 7), inputs.positions(lat, 70, 8, -3.0, 4.0)])
    ref = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
    got = gpu_eval(spl, pos)
    assert_parity(got, ref, TOL[storage], "%s/%s/sep=%d/O=%d" % (method, storage, sep, n_orb))


def test_edge_cases_empty_single_nan_and_far():
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_cell(5, dims, 6, 5.0, 4.0, np.eye(3) * 6.0)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=True)
    beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
    # P = 0 is a no-op
    empty = torch.zeros((0, 3), dtype=torch.float64, device=dev())
    v, g, l = spl.eval_vgl(empty)
    spl.sync()
    assert v.shape == (0, 6)
    # P = 1, at a grid point, and far outside the cell
    for p in (np.array([[0.0, 0.0, 0.0]]), np.array([[0.75, 1.5, 2.25]]),
              np.array([[6.0 * 1000 + 0.3, -6.0 * 777 + 0.1, 6.0 * 12345 + 5.9]])):
        ref = oracle.bspline_eval(beta, lat, p, beta_lap=blap)
        assert_parity(gpu_eval(spl, p), ref, 1e-11)
    # a non-finite position: NaN outputs for that row only, error reported at sync
    pos = inputs.positions(lat, 40, 3)
    pos[17, 1] = np.nan
    v, g, l = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    from paper_1309_6250_gb300 import _lib
    with pytest.raises(_lib.QmcsplError) as ei:
        spl.sync()
    assert ei.value.code == _lib.ERR_DEVICE
    spl.sync()                      # the flag is cleared once reported
    v = v.cpu().numpy()
    assert np.all(np.isnan(v[17])) and np.all(np.isfinite(np.delete(v, 17, axis=0)))
    ok = np.delete(np.arange(40), 17)
    ref = oracle.bspline_eval(beta, lat, pos[ok], beta_lap=blap)
    assert oracle.relative_error(v[ok], ref[0]) < 1e-12


@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
def test_c2_si8_smoothing_with_laplacian_table(storage):
    """Si-like 8-atom cell, 16 orbitals on 48^3, smoothing B-spline + separate Laplacian
    table; 4096 of the 1024 x 32 positions.  Also reports the kinetic-energy effect of
    the Laplacian error, T_n = -1/2 <phi lap phi>/<phi^2>."""
    w = inputs.make_workload("c2", n_pos=4096)
    dims = w.cell.grid
    spl = splines(w.lattice, dims, w.miller, w.coef, method="smooth", storage=storage, separate_lap=True)
    beta, blap = oracle.smoothing_tables(w.lattice, w.miller, w.coef, dims, laplacian=True)
    ref = oracle.bspline_eval(beta, w.lattice, w.pos, beta_lap=blap)
    got = gpu_eval(spl, w.pos)
    assert_parity(got, ref, TOL[storage], "c2/" + storage)
    dT = np.abs(oracle.kinetic_energy(got[0], got[2]) - oracle.kinetic_energy(ref[0], ref[2]))
    print("c2 %s: max |dT_n| = %.3e mHa" % (storage, 1e3 * dT.max()))
    assert 1e3 * dT.max() < {"f64": 1e-9, "df64": 1e-9, "f32": 1e-2, "bf16": 50.0}[storage]


def test_host_buffers_match_device_path():
    """qmcspl_eval_vgl_host (chunked copies + kernels) returns exactly the device path."""
    w = inputs.make_workload("c2", n_pos=150_000)
    spl = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                  separate_lap=True)
    pos_h = torch.from_numpy(w.pos).pin_memory()
    hv, hg, hl = spl.eval_vgl_host(pos_h)
    dv, dg, dl = spl.eval_vgl(pos_h.to(dev()))
    torch.cuda.synchronize()
    assert torch.equal(hv, dv.cpu()) and torch.equal(hg, dg.cpu()) and torch.equal(hl, dl.cpu())


def _oracle_c3_sample(w, sample, sep=True):
    """Oracle outputs at sampled positions for a large cell, built in orbital chunks."""
    outs = [[], [], []]
    for o0 in range(0, w.coef.shape[0], 16):
        c = w.coef[o0:o0 + 16]
        beta, blap = oracle.smoothing_tables(w.lattice, w.miller, c, w.cell.grid, laplacian=sep)
        r = oracle.bspline_eval(beta, w.lattice, w.pos[sample], beta_lap=blap)
        for k in range(3):
            outs[k].append(r[k])
    return (np.concatenate(outs[0], axis=-1), np.concatenate(outs[1], axis=-1),
            np.concatenate(outs[2], axis=-1))


@pytest.mark.slow
def test_c3_mgo64_full_size_sampled():
    """MgO-like 64-atom cell: 128 orbitals on 96^3, 2048 x 256 positions, smoothing +
    Laplacian table in FP32 and BF16 (the benchmark's launch), checked on a sample of
    the outputs against the oracle."""
    w = inputs.make_workload("c3")
    P = w.pos.shape[0]
    sample = np.unique(np.concatenate([np.arange(0, P, 8191), np.arange(P - 5, P)]))
    ref = _oracle_c3_sample(w, sample)
    pos = torch.from_numpy(w.pos).to(dev())
    for storage in ("f32", "bf16", "df64"):
        spl = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage=storage,
                      separate_lap=True)
        v, g, l = spl.eval_vgl(pos)
        spl.sync()
        s = torch.from_numpy(sample).to(dev())
        got = (v[s].double().cpu().numpy(), g[s].double().cpu().numpy(), l[s].double().cpu().numpy())
        errs = assert_parity(got, ref, TOL[storage], "c3/" + storage)
        print("c3 %s sampled errors: %s" % (storage, ["%.2e" % e for e in errs]))
        spl.close()


def test_out_of_memory_is_reported_not_faulted():
    """A table far larger than the device reports QMCSPL_ERR_OOM (or a CUDA error) from
    qmcspl_create and leaves the context usable."""
    from paper_1309_6250_gb300 import _lib
    mil = np.zeros((1, 3), dtype=np.int32)
    coef = np.ones((4096, 1))
    with pytest.raises(_lib.QmcsplError) as ei:
        splines(np.eye(3) * 10.0, (512, 512, 512), mil, coef, method="smooth", storage="f64",
                separate_lap=True)
    assert ei.value.code in (_lib.ERR_OOM, _lib.ERR_CUDA)
    # the device still works
    lat, mil, coef = inputs.random_cell(1, (8, 8, 8), 2, 4.0, 4.0, np.eye(3) * 6.0)
    spl = splines(lat, (8, 8, 8), mil, coef, method="smooth", storage="f64", separate_lap=False)
    beta, _ = oracle.smoothing_tables(lat, mil, coef, (8, 8, 8))
    pos = inputs.positions(lat, 10, 1)
    assert_parity(gpu_eval(spl, pos), oracle.bspline_eval(beta, lat, pos), 1e-12)
