"""Staged evaluation (pencil order: stencil planes copied into shared memory by tensor
copies) against the gather kernel (cell order, bit for bit) and the oracle."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def both_orders(spl, pos):
    out = {}
    for mode in ("cell", "pencil"):
        spl.set_order(mode)
        out[mode] = [t.clone() for t in spl.eval_vgl(pos)]
        spl.sync()
    return out


def assert_identical(out):
    for a, b in zip(out["cell"], out["pencil"]):
        assert torch.equal(a, b)


# orbital counts giving rows of 512, 256 and 128 bytes (32, 16 and 8 lanes per position)
@pytest.mark.parametrize("storage,n_orb", [("f32", 128), ("f32", 61), ("f32", 32),
                                           ("bf16", 256), ("bf16", 128), ("bf16", 64)])
@pytest.mark.parametrize("sep", [True, False])
def test_staged_bit_identical_to_gather(storage, n_orb, sep):
    """Odd grid sizes (the last pencil of x and y is one cell wide), a non-orthogonal
    cell, positions inside and far outside the cell."""
    dims = (13, 11, 12)
    lat, mil, coef = inputs.random_cell(2100 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=sep)
    assert spl.info()["staged"] == 1
    pos = torch.from_numpy(np.vstack([inputs.positions(lat, 30000, 2101),
                                      inputs.positions(lat, 3000, 2102, -5, 6)])).to(dev())
    assert_identical(both_orders(spl, pos))
    spl.close()


@pytest.mark.parametrize("storage,n_orb", [("f32", 128), ("f32", 32), ("bf16", 64)])
def test_staged_sparse_and_clustered(storage, n_orb):
    """Few positions per pencil (the positions of one warp task may span more planes than the
    ring holds: they are then evaluated one group per round), all positions in one pencil
    (long items), a single position, and non-finite positions."""
    from paper_1309_6250_gb300 import _lib
    dims = (16, 16, 40)
    lat, mil, coef = inputs.random_cell(2200 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=True)
    assert spl.info()["staged"] == 1
    sparse = inputs.positions(lat, 300, 2201)
    s = np.random.default_rng(2202).random((5000, 3)) * np.array([0.1, 0.1, 1.0])
    clustered = s @ lat.T                       # crystal x, y < 0.1: pencil 0 and its neighbours
    for pos in (sparse, clustered, sparse[:1]):
        assert_identical(both_orders(spl, torch.from_numpy(pos).to(dev())))
    pos = inputs.positions(lat, 2000, 2203)
    pos[[3, 700]] = [np.inf, 0.0, 0.0], [0.0, np.nan, 1.0]
    spl.set_order("pencil")
    v, g, l = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    with pytest.raises(_lib.QmcsplError) as ei:
        spl.sync()
    assert ei.value.code == _lib.ERR_DEVICE
    v = v.cpu().numpy()
    assert np.all(np.isnan(v[[3, 700]])) and np.isfinite(np.delete(v, [3, 700], axis=0)).all()
    keep = torch.from_numpy(np.delete(np.arange(2000), [3, 700])).to(dev())
    spl.set_order("cell")
    ref = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    with pytest.raises(_lib.QmcsplError):
        spl.sync()
    assert torch.equal(ref[0][keep], torch.from_numpy(v).to(dev())[keep])
    spl.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_staged_matches_oracle(storage):
    """128 orbitals on a 24^3 grid, 65,536 positions in pencil order: a sample of positions
    against the oracle within the storage tolerance."""
    dims = (24, 24, 24)
    lat, mil, coef = inputs.random_cell(2300, dims, 128, 8.0, 6.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    spl.set_order("pencil")
    pos = inputs.positions(lat, 65536, 2301)
    got = gpu_eval(spl, pos)
    sample = np.arange(0, 65536, 97)
    beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
    ref = oracle.bspline_eval(rounded(beta, storage), lat, pos[sample], beta_lap=rounded(blap, storage))
    assert_parity([x[sample] for x in got], ref, TOL[storage], storage)
    spl.set_order("cell")
    cell = gpu_eval(spl, pos)
    for a, b in zip(got, cell):
        np.testing.assert_array_equal(a, b)
    spl.close()


def test_pencil_order_falls_back_where_staging_does_not_apply():
    """FP64 and double-float tables, several orbital tiles per position, rows of 64 bytes,
    separate gradient tables, Lagrange, pp and degree-5 splines: pencil order evaluates in cell
    order."""
    dims = (10, 10, 10)
    lat, mil, coef = inputs.random_cell(2350, dims, 48, 6.0, 5.0, NONORTHO)
    cases = [dict(method="smooth", storage="f64", separate_lap=True),
             dict(method="smooth", storage="df64", separate_lap=True),
             dict(method="smooth", storage="f32", separate_lap=True),            # 48 orbitals: 3 tiles
             dict(method="smooth", storage="f32", separate_lap=True, lanes=8),   # 128 orbitals below
             dict(method="smooth", storage="bf16", separate_lap=True, lanes=4),  # 32 orbitals below
             dict(method="smooth", storage="f32", separate_lap=True, separate_grad=True),
             dict(method="lagrange", storage="f32", separate_lap=True),
             dict(method="pp", storage="f32", separate_lap=False),
             dict(method="interp", storage="f32", separate_lap=True, degree=5)]
    pos = torch.from_numpy(inputs.positions(lat, 3000, 2351)).to(dev())
    for kw in cases:
        n_orb = {8: 128, 4: 32}.get(kw.get("lanes"), 48)
        _, m, c = inputs.random_cell(2352, dims, n_orb, 6.0, 5.0, NONORTHO)
        spl = splines(lat, dims, m, c, **kw)
        assert spl.info()["staged"] == 0, kw
        assert_identical(both_orders(spl, pos))
        spl.close()


def test_staged_bloch_bit_identical():
    dims = (12, 14, 16)
    k = inputs.KPOINTS["generic"]
    lat, mil, coef = inputs.random_bloch_cell(2400, 64, 6.0, 5.0, k, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True, kpoint=k)
    assert spl.info()["staged"] == 1          # 64 complex orbitals: 128 stored functions
    pos = torch.from_numpy(inputs.positions(lat, 20000, 2401, -2, 3)).to(dev())
    assert_identical(both_orders(spl, pos))
    spl.close()


def test_staged_graph_capture():
    """The pencil-order evaluation -- records, sort into pencils, staged kernel -- captured in
    a CUDA graph after one eager call; replays give the eager results."""
    dims = (20, 20, 20)
    lat, mil, coef = inputs.random_cell(2500, dims, 128, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True)
    spl.set_order("pencil")
    pos = torch.from_numpy(inputs.positions(lat, 50000, 2501)).to(dev())
    ref = [t.clone() for t in spl.eval_vgl(pos)]
    spl.sync()
    out = spl.alloc_outputs(pos.shape[0])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        spl.eval_vgl(pos, out=out, stream=s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            spl.eval_vgl(pos, out=out, stream=s)
    for t in out:
        t.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    spl.close()


def test_stalled_pipeline_times_out_and_recovers():
    """A producer that copies nothing (test hook): every consumer wait runs out after about a
    second, the launch ends by itself, qmcspl_sync reports QMCSPL_ERR_TIMEOUT, and the next
    evaluation on the same handle is correct."""
    from paper_1309_6250_gb300 import _lib
    L = _lib.load()
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_cell(2600, dims, 32, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True)
    spl.set_order("pencil")
    pos = torch.from_numpy(inputs.positions(lat, 4000, 2601)).to(dev())
    ref = [t.clone() for t in spl.eval_vgl(pos)]
    spl.sync()
    try:
        L.qmcspl_debug_stall_pipeline(1)
        spl.eval_vgl(pos)
        with pytest.raises(_lib.QmcsplError) as ei:
            spl.sync()
        assert ei.value.code == _lib.ERR_TIMEOUT
    finally:
        L.qmcspl_debug_stall_pipeline(0)
    again = spl.eval_vgl(pos)
    spl.sync()
    for a, b in zip(again, ref):
        assert torch.equal(a, b)
    spl.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_staged_full_size_bit_identical(storage):
    """The MgO-like 128-orbital workload at full size (96^3, 2,048 x 256 positions): 221,184
    pencil bins, two z segments per pencil; pencil order gives exactly the cell-order outputs."""
    w = inputs.make_workload("c3")
    spl = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage=storage,
                  separate_lap=True)
    assert spl.info()["staged"] == 1
    assert_identical(both_orders(spl, torch.from_numpy(w.pos).to(dev())))
    spl.close()
