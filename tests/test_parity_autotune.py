"""Tile shapes (lanes per position) and the autotuner on the GPU: every shape returns the
same bits, the tuned handle included."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
def test_every_lane_count_gives_identical_results(storage):
    dims = (10, 11, 12)
    lat, mil, coef = inputs.random_cell(910, dims, 37, 6.0, 5.0, NONORTHO)
    pos = inputs.positions(lat, 999, 3, -1, 2)
    ref = None
    beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
    for L in (1, 2, 4, 8, 16, 32):
        spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True, lanes=L)
        info = spl.info()
        assert info["lanes"] == L and info["n_orb_padded"] % L == 0
        got = gpu_eval(spl, pos)
        if ref is None:
            ref = got
            assert_parity(got, oracle.bspline_eval(rounded(beta, storage), lat, pos,
                                                   beta_lap=rounded(blap, storage)), TOL[storage])
        else:
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), L


def test_invalid_lanes_rejected():
    from paper_1309_6250_gb300 import _lib
    lat, mil, coef = inputs.random_cell(1, (8, 8, 8), 2, 4.0, 4.0, np.eye(3) * 6.0)
    with pytest.raises(_lib.QmcsplError) as ei:
        splines(lat, (8, 8, 8), mil, coef, lanes=3)
    assert ei.value.code == _lib.ERR_ARG


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    from paper_1309_6250_gb300 import autotune
    w = inputs.make_workload("c4-al32", n_pos=20000)
    cache = str(tmp_path / "tune.json")
    t = autotune.tune(w.lattice, w.cell.grid, w.miller, w.coef, w.pos, storage="f32", separate_lap=True,
                      device=dev(), repeats=3, cache_path=cache)
    assert t["lanes"] in autotune.candidate_lanes(48, "f32") and t["order"] in ("input", "cell")
    assert t["threads"] in autotune.candidate_threads("f32")
    assert len(t["trials"]) == 2 * len(autotune.candidate_threads("f32")) * len(autotune.candidate_lanes(48, "f32"))
    again = autotune.tune(w.lattice, w.cell.grid, w.miller, w.coef, w.pos, storage="f32",
                          separate_lap=True, device=dev(), cache_path=cache)
    assert again == t
    spl, t2 = autotune.tuned_splines(w.lattice, w.cell.grid, w.miller, w.coef, w.pos, storage="f32",
                                     separate_lap=True, device=dev(), cache_path=cache)
    assert t2 == t and spl.info()["lanes"] == t["lanes"] and spl.info()["block_threads"] == t["threads"]
    base = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                   separate_lap=True)
    for a, b in zip(gpu_eval(spl, w.pos), gpu_eval(base, w.pos)):
        assert np.array_equal(a, b)


def test_batched_with_cell_order_matches_single_launches():
    from paper_1309_6250_gb300.api import eval_batched
    ws = [inputs.make_workload(k, n_pos=n) for k, n in (("c4-al32", 30000), ("c4-mgo16", 12000))]
    spls = [splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                    separate_lap=True) for w in ws]
    for s in spls:
        s.set_order("cell")
    pos = [torch.from_numpy(w.pos).to(dev()) for w in ws]
    outs = eval_batched(spls, pos)
    torch.cuda.synchronize()
    for s, p, o in zip(spls, pos, outs):
        s.set_order("input")
        single = s.eval_vgl(p)
        s.sync()
        for a, b in zip(o, single):
            assert torch.equal(a, b)


@pytest.mark.parametrize("method,storage,sep", [("smooth", "f32", True), ("interp", "df64", False),
                                                ("pp", "bf16", False), ("lagrange", "f64", True)])
def test_save_load_round_trip(tmp_path, method, storage, sep):
    """qmcspl_save / qmcspl_load: the loaded handle evaluates to the same bits; a flipped
    byte in the tables fails the checksum."""
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import OrbitalSplines
    dims = (10, 11, 12)
    lat, mil, coef = inputs.random_cell(950, dims, 9, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep, lanes=4)
    path = tmp_path / "t.qmcspl"
    spl.save(path)
    loaded = OrbitalSplines.load(path, device=dev())
    assert loaded.info() == spl.info()
    pos = inputs.positions(lat, 20000, 4, -1, 2)
    for a, b in zip(gpu_eval(spl, pos), gpu_eval(loaded, pos)):
        assert np.array_equal(a, b)
    raw = bytearray(path.read_bytes())
    raw[-100] ^= 0x01
    path.write_bytes(bytes(raw))
    with pytest.raises(_lib.QmcsplError) as ei:
        OrbitalSplines.load(path, device=dev())
    assert ei.value.code == _lib.ERR_ARG
