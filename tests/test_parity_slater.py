"""GPU Slater-determinant consumer (qmcspl_slater_kinetic) against the oracle's definition
(numpy slogdet / inv) on the same orbital values, real and complex (Bloch orbitals).

The orbital values both sides consume are the oracle's spline outputs (its own tables and
evaluation), rounded to the dtype the consumer reads; nothing the oracle sees comes from the
GPU."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def consumer(v, g, l, W, n_elec, n_up, arith="df64"):
    from paper_1309_6250_gb300.api import slater_kinetic
    out = slater_kinetic(v, g, l, W, n_elec, n_up, arith=arith)
    torch.cuda.synchronize()
    return tuple(None if x is None else x.cpu().numpy() for x in out)


def oracle_orbitals(lat, mil, coef, dims, pos, storage, kpoint=None):
    """Smoothing B-spline outputs (with the Laplacian table) of the oracle at `pos`, as the
    consumer reads them: float64, or rounded to float32 for storage 'f32' (what an FP32-table
    handle would hand the consumer).  Returns (numpy arrays as the oracle sees them, device
    tensors for the GPU)."""
    if kpoint is None:
        beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
        out = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
    else:
        beta, blap = oracle.bloch_tables("smooth", lat, mil, coef, kpoint, dims, laplacian=True)
        out = oracle.bloch_eval("smooth", beta, lat, kpoint, pos, tables_lap=blap)
    dt = {"f64": np.float64, "f32": np.float32}[storage]
    if kpoint is not None:
        dt = {np.float64: np.complex128, np.float32: np.complex64}[dt]
    dev_out = tuple(torch.from_numpy(np.ascontiguousarray(x.astype(dt))).to(dev()) for x in out)
    ref_in = tuple(x.astype(dt).astype(np.complex128 if kpoint is not None else np.float64) for x in out)
    return ref_in, dev_out


def compare(got, ref, rel=1e-9):
    ld, sg, kin, dr = got
    rld, rsg, rkin, rdr = ref
    np.testing.assert_array_equal(sg, rsg)
    assert np.max(np.abs(ld - rld)) <= rel * max(1.0, np.max(np.abs(rld)))
    assert oracle.relative_error(kin, rkin) < rel * 10
    assert oracle.relative_error(dr, rdr) < rel * 10


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("n_elec,n_up,n_orb", [(13, 7, 9), (8, 0, 8), (2, 1, 3), (40, 20, 24)])
def test_consumer_matches_oracle(storage, n_elec, n_up, n_orb, arith):
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_cell(1300 + n_elec, dims, n_orb, 8.0, 6.0, NONORTHO)
    W = 6
    pos = inputs.positions(lat, W * n_elec, 1301 + n_elec)
    ref_in, (v, g, l) = oracle_orbitals(lat, mil, coef, dims, pos, storage)
    got = consumer(v, g, l, W, n_elec, n_up, arith)
    ref = oracle.slater_kinetic(*ref_in, W, n_elec, n_up)
    compare(got, ref)


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_consumer_largest_block_and_singular_walker(arith):
    """Blocks of QMCSPL_SLATER_MAX_BLOCK electrons; a walker whose up block has a zero row
    is exactly singular: sign 0, logdet -inf, NaN kinetic energy and drift, the other
    walkers unaffected."""
    from paper_1309_6250_gb300 import _lib
    n = _lib.SLATER_MAX_BLOCK
    rng = np.random.default_rng(7)
    W, n_elec = 3, 2 * n
    val = rng.standard_normal((W * n_elec, n)) + 4.0 * np.tile(np.eye(n), (2 * W, 1))
    grad = rng.standard_normal((W * n_elec, 3, n))
    lap = rng.standard_normal((W * n_elec, n))
    val[1 * n_elec + 5] = 0.0                      # walker 1, up block: zero row
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev())
    ld, sg, kin, dr = consumer(t(val), t(grad), t(lap), W, n_elec, n, arith)
    assert sg[1] == 0 and ld[1] == -np.inf and np.isnan(kin[1]) and np.all(np.isnan(dr[1]))
    keep = [0, 2]
    rows = np.concatenate([np.arange(w * n_elec, (w + 1) * n_elec) for w in keep])
    ref = oracle.slater_kinetic(val[rows], grad[rows], lap[rows], 2, n_elec, n)
    compare((ld[keep], sg[keep], kin[keep], dr[keep]), ref)


def test_consumer_rejects_bad_arguments():
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import slater_kinetic
    v = torch.zeros((4, 3), dtype=torch.float64, device=dev())
    with pytest.raises(_lib.QmcsplError):
        slater_kinetic(v, None, v, 1, 4, 5)          # n_up > n_elec
    with pytest.raises(_lib.QmcsplError):
        slater_kinetic(v, None, v, 1, 4, 0)          # a block of 4 electrons, rows of 3 orbitals
    big = torch.zeros((2 * 161, 161), dtype=torch.float64, device=dev())
    with pytest.raises(_lib.QmcsplError) as ei:
        slater_kinetic(big, None, big, 1, 2 * 161, 161)
    assert ei.value.code == _lib.ERR_UNSUPPORTED


@pytest.mark.slow
@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_consumer_c3_mgo64_full_batch(arith):
    """The MgO-like 64-atom workload as a QMC walker batch: 2048 walkers x 256 electrons,
    128 up and 128 down, each block using all 128 orbitals of the smoothing spline with the
    Laplacian table (the oracle's outputs rounded to FP32, as an FP32-table handle gives them);
    every 7th walker against the oracle."""
    w = inputs.make_workload("c3")
    ref_in, (v, g, l) = oracle_orbitals(w.lattice, w.miller, w.coef, w.cell.grid, w.pos, "f32")
    W, n_elec = w.cell.n_walkers, w.cell.n_elec
    got = consumer(v, g, l, W, n_elec, n_elec // 2, arith)
    sample = np.arange(0, W, 7)
    rows = np.concatenate([np.arange(s * n_elec, (s + 1) * n_elec) for s in sample])
    ref = oracle.slater_kinetic(*(x[rows] for x in ref_in), len(sample), n_elec, n_elec // 2)
    compare(tuple(x[sample] for x in got), ref, rel=1e-8)


# ---------------------------------------------------------------------------
# complex orbitals (outputs of a Bloch handle): complex determinants, FP64 elimination
# ---------------------------------------------------------------------------

def compare_complex(got, ref, rel=1e-9):
    ld, sg, kin, dr = got
    rld, rsg, rkin, rdr = ref
    assert np.max(np.abs(ld - rld)) <= rel * max(1.0, np.max(np.abs(rld)))
    assert np.max(np.abs(sg - rsg)) <= rel * 100
    assert oracle.relative_error(kin, rkin) < rel * 10
    assert oracle.relative_error(dr, rdr) < rel * 10


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("n_elec,n_up,n_orb", [(13, 7, 9), (8, 0, 8), (2, 1, 3), (40, 20, 24)])
def test_complex_consumer_matches_oracle(storage, n_elec, n_up, n_orb, arith):
    k = inputs.KPOINTS["generic"]
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_bloch_cell(1900 + n_elec, n_orb, 8.0, 6.0, k, NONORTHO)
    W = 6
    pos = inputs.positions(lat, W * n_elec, 1901 + n_elec, -1, 2)
    ref_in, (v, g, l) = oracle_orbitals(lat, mil, coef, dims, pos, storage, kpoint=k)
    assert v.is_complex()
    got = consumer(v, g, l, W, n_elec, n_up, arith=arith)
    ref = oracle.slater_kinetic(*ref_in, W, n_elec, n_up)
    compare_complex(got, ref)


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_complex_consumer_largest_block_singular_walker_and_rejections(arith):
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import slater_kinetic
    n = _lib.SLATER_MAX_COMPLEX_BLOCK
    rng = np.random.default_rng(1910)
    W, n_elec = 3, 2 * n
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    val = c(W * n_elec, n) + 4.0 * np.tile(np.eye(n), (2 * W, 1))
    grad = c(W * n_elec, 3, n)
    lap = c(W * n_elec, n)
    val[2 * n_elec + n + 3] = 0.0                  # walker 2, down block: zero row
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev())
    ld, sg, kin, dr = consumer(tt(val), tt(grad), tt(lap), W, n_elec, n, arith)
    assert sg[2] == 0 and ld[2] == -np.inf and np.isnan(kin[2]) and np.all(np.isnan(dr[2]))
    keep = [0, 1]
    rows = np.concatenate([np.arange(w * n_elec, (w + 1) * n_elec) for w in keep])
    ref = oracle.slater_kinetic(val[rows], grad[rows], lap[rows], 2, n_elec, n)
    compare_complex((ld[keep], sg[keep], kin[keep], dr[keep]), ref)
    v = tt(val[: 2 * n])
    big = torch.zeros((2 * (n + 1), n + 1), dtype=torch.complex128, device=dev())
    with pytest.raises(_lib.QmcsplError) as ei:
        slater_kinetic(big, None, big, 1, 2 * (n + 1), n + 1, arith=arith)   # a block over the limit
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    with pytest.raises(_lib.QmcsplError) as ei:
        slater_kinetic(v, None, v, 1, 2 * n, 2 * n + 1, arith=arith)         # n_up > n_elec
    assert ei.value.code == _lib.ERR_ARG
