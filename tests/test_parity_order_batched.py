"""Cell-ordered evaluation returns exactly the input-order results; the batched
multi-cell launch returns exactly the per-cell results (and matches the oracle)."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,storage,sep", [("smooth", "f32", True), ("smooth", "bf16", True),
                                                ("smooth", "df64", True), ("interp", "df64", False),
                                                ("interp", "f64", False), ("lagrange", "f32", True),
                                                ("pp", "f32", False)])
def test_cell_order_is_bit_identical(method, storage, sep):
    dims = (20, 22, 24)
    lat, mil, coef = inputs.random_cell(77, dims, 20, 8.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep)
    pos = torch.from_numpy(np.vstack([inputs.positions(lat, 30000, 6),
                                      inputs.positions(lat, 1000, 7, -5, 6)])).to(dev())
    outs = {}
    for mode in ("input", "cell", "auto"):
        spl.set_order(mode)
        outs[mode] = [t.clone() for t in spl.eval_vgl(pos)]
        spl.sync()
    for mode in ("cell", "auto"):
        for a, b in zip(outs["input"], outs[mode]):
            assert torch.equal(a, b), mode


def test_cell_order_small_and_nan():
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_cell(78, dims, 4, 5.0, 4.0, np.eye(3) * 6.0)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=True)
    spl.set_order("cell")
    beta, blap = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
    for n in (1, 2, 33):
        pos = inputs.positions(lat, n, 10 + n)
        assert_parity(gpu_eval(spl, pos), oracle.bspline_eval(beta, lat, pos, beta_lap=blap), 1e-12)
    pos = inputs.positions(lat, 100, 3)
    pos[5] = np.inf
    v, _, _ = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    from paper_1309_6250_gb300 import _lib
    with pytest.raises(_lib.QmcsplError):
        spl.sync()
    v = v.cpu().numpy()
    assert np.all(np.isnan(v[5])) and np.isfinite(np.delete(v, 5, axis=0)).all()


def test_batched_uneven_cells_full_size():
    """Al-like 32-atom (48 orbitals, 64^3, 512 x 96 e), Si-like 64-atom (128, 80^3,
    1024 x 256 e) and MgO-like 16-atom (32, 64^3, 2048 x 64 e), FP32 smoothing + Laplacian
    table, in one launch: identical to three separate launches, and on a sample of each
    cell equal to the oracle within the FP32 tolerance."""
    from paper_1309_6250_gb300.api import eval_batched
    keys = ("c4-al32", "c4-si64", "c4-mgo16")
    ws = [inputs.make_workload(k) for k in keys]
    spls = [splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                    separate_lap=True) for w in ws]
    for s in spls:
        s.set_order("input")
    pos = [torch.from_numpy(w.pos).to(dev()) for w in ws]
    outs = eval_batched(spls, pos)
    torch.cuda.synchronize()
    for s, p, o, w in zip(spls, pos, outs, ws):
        single = s.eval_vgl(p)
        s.sync()
        for a, b in zip(o, single):
            assert torch.equal(a, b), w.cell.name
        sample = np.arange(0, w.pos.shape[0], max(1, w.pos.shape[0] // 40))
        ref = [[], [], []]
        for o0 in range(0, w.coef.shape[0], 32):
            beta, blap = oracle.smoothing_tables(w.lattice, w.miller, w.coef[o0:o0 + 32], w.cell.grid,
                                                 laplacian=True)
            r = oracle.bspline_eval(rounded(beta, "f32"), w.lattice, w.pos[sample],
                                    beta_lap=rounded(blap, "f32"))
            for k in range(3):
                ref[k].append(r[k])
        ref = [np.concatenate(r, axis=-1) for r in ref]
        s_t = torch.from_numpy(sample).to(dev())
        got = [t[s_t].double().cpu().numpy() for t in o]
        assert_parity(got, ref, TOL["f32"], w.cell.name)


def test_batched_graph_capture_and_validation():
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import eval_batched
    cells = []
    for i, dims in enumerate(((12, 12, 12), (10, 14, 16))):
        lat, mil, coef = inputs.random_cell(500 + i, dims, 7 + 9 * i, 6.0, 5.0, NONORTHO)
        cells.append((splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True),
                      torch.from_numpy(inputs.positions(lat, 1000 + 777 * i, 9)).to(dev())))
    spls = [c[0] for c in cells]
    pos = [c[1] for c in cells]
    outs = [s.alloc_outputs(p.shape[0]) for s, p in zip(spls, pos)]
    ref = eval_batched(spls, pos)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        eval_batched(spls, pos, outs=outs, stream=s)   # warm up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            eval_batched(spls, pos, outs=outs, stream=s)
    for o in outs:
        for t in o:
            t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    # mixed storage types are rejected before any launch
    lat, mil, coef = inputs.random_cell(9, (8, 8, 8), 3, 5.0, 4.0, np.eye(3) * 6.0)
    other = splines(lat, (8, 8, 8), mil, coef, method="smooth", storage="f64", separate_lap=True)
    with pytest.raises(_lib.QmcsplError) as ei:
        eval_batched([spls[0], other], [pos[0], pos[0]])
    assert ei.value.code == _lib.ERR_ARG


def test_eval_vgl_cell_order_captured_in_cuda_graph():
    """After one call at a size (scratch allocated) qmcspl_eval_vgl -- records, sort and
    evaluation -- can be captured in a CUDA graph; replays give the eager results."""
    w = inputs.make_workload("c2", n_pos=20000)
    spl = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32", separate_lap=True)
    pos = torch.from_numpy(w.pos).to(dev())
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
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)


def test_batched_mixes_own_and_shared_launches():
    """A call with one cell large enough for its own launch (over four rounds of warp tasks)
    and two small cells sharing the batched launch: every cell equals its own eval_vgl, also
    when the call is captured in a CUDA graph and replayed."""
    from paper_1309_6250_gb300.api import eval_batched
    cells = []
    for i, (dims, n_orb, n_pos) in enumerate((((12, 12, 12), 16, 90_000), ((10, 14, 16), 7, 1000),
                                              ((8, 8, 12), 20, 3001))):
        lat, mil, coef = inputs.random_cell(520 + i, dims, n_orb, 6.0, 5.0, NONORTHO)
        cells.append((splines(lat, dims, mil, coef, method="interp", storage="f32", separate_lap=True),
                      torch.from_numpy(inputs.positions(lat, n_pos, 30 + i, -1, 2)).to(dev())))
    spls = [c[0] for c in cells]
    pos = [c[1] for c in cells]
    singles = [s.eval_vgl(p) for s, p in zip(spls, pos)]
    torch.cuda.synchronize()
    outs = eval_batched(spls, pos)
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        eval_batched(spls, pos, outs=outs, stream=st)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            eval_batched(spls, pos, outs=outs, stream=st)
    for o in outs:
        for t in o:
            t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        for x, y in zip(a, b):
            assert torch.equal(x, y)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f64"])
def test_launch_plans_and_block_shapes_give_the_same_bits(storage):
    """qmcspl_eval_batched_ex: one launch per cell, every cell in the one persistent batched
    launch with 512 or (float / bfloat16 tables) 640 threads per block, and the automatic rule
    all give each cell exactly its own qmcspl_eval_vgl outputs, whatever the block shape set on
    the handles (qmcspl_set_block); the single launch also as a CUDA-graph replay."""
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import eval_batched
    cells = []
    for i, (dims, n_orb, n_pos) in enumerate((((12, 12, 12), 16, 60_000), ((10, 14, 16), 7, 1000),
                                              ((8, 8, 12), 20, 9001))):
        lat, mil, coef = inputs.random_cell(540 + i, dims, n_orb, 6.0, 5.0, NONORTHO)
        cells.append((splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=i != 1),
                      torch.from_numpy(inputs.positions(lat, n_pos, 40 + i, -1, 2)).to(dev())))
    # one separate_lap setting per batch: the middle cell goes to its own calls only
    spls = [cells[0][0], cells[2][0]]
    pos = [cells[0][1], cells[2][1]]
    singles = [[t.clone() for t in s.eval_vgl(p)] for s, p in zip(spls, pos)]
    torch.cuda.synchronize()
    shapes = [0, 512] + ([640] if storage in ("f32", "bf16") else [])
    for th in shapes:
        for s in spls:
            s.set_block(th)
            assert s.info()["block_threads"] == th
        for s, p, ref in zip(spls, pos, singles):
            got = s.eval_vgl(p)
            torch.cuda.synchronize()
            assert all(torch.equal(x, y) for x, y in zip(got, ref))
        for plan in [{"launch": "auto"}, {"launch": "split"}] + [{"launch": "single", "threads": t} for t in shapes]:
            outs = eval_batched(spls, pos, plan=plan)
            torch.cuda.synchronize()
            for a, b in zip(outs, singles):
                assert all(torch.equal(x, y) for x, y in zip(a, b)), (th, plan)
    # the single persistent launch captured in a CUDA graph
    plan = {"launch": "single", "threads": shapes[-1]}
    outs = [s.alloc_outputs(p.shape[0]) for s, p in zip(spls, pos)]
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        eval_batched(spls, pos, outs=outs, stream=st, plan=plan)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=st):
            eval_batched(spls, pos, outs=outs, stream=st, plan=plan)
    for o in outs:
        for t in o:
            t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        assert all(torch.equal(x, y) for x, y in zip(a, b))
    # rejected plans and shapes
    with pytest.raises(_lib.QmcsplError) as ei:
        eval_batched(spls, pos, plan={"launch": "single", "threads": 256})
    assert ei.value.code == _lib.ERR_ARG
    if storage == "f64":
        with pytest.raises(_lib.QmcsplError) as ei:
            spls[0].set_block(640)
        assert ei.value.code == _lib.ERR_UNSUPPORTED
        with pytest.raises(_lib.QmcsplError) as ei:
            eval_batched(spls, pos, plan={"launch": "single", "threads": 640})
        assert ei.value.code == _lib.ERR_UNSUPPORTED



def test_batched_refuses_a_handle_twice():
    """Each cell's visiting order lives in its handle's scratch, so a handle may appear only once
    in a batch; cells of 8192 positions or more (records, and the sort for the first and last)
    give the bytes of per-cell eval_vgl."""
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import eval_batched
    spec = (((16, 16, 16), 8, 40_000), ((20, 18, 16), 24, 9_000), ((12, 12, 12), 5, 20_000))
    spls, pos = [], []
    for i, (dims, n_orb, n) in enumerate(spec):
        lat, mil, coef = inputs.random_cell(2450 + i, dims, n_orb, 6.0, 5.0, NONORTHO)
        spls.append(splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True))
        pos.append(torch.from_numpy(inputs.positions(lat, n, 2460 + i, -1, 2)).to(dev()))
    assert [s.resolved_order(p.shape[0]) for s, p in zip(spls, pos)] == ["cell", "input", "cell"]
    ref = [s.eval_vgl(p) for s, p in zip(spls, pos)]
    got = eval_batched(spls, pos)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    with pytest.raises(_lib.QmcsplError) as ei:
        eval_batched([spls[0], spls[1], spls[0]], [pos[0], pos[1], pos[0]])
    assert ei.value.code == _lib.ERR_ARG
    for s in spls:
        s.close()


def test_batched_with_an_empty_cell():
    """A cell of no positions in the middle of a batch (its pointers may be NULL) changes nothing
    for the others under every launch plan; the host-buffer call with no positions is a no-op."""
    from paper_1309_6250_gb300.api import eval_batched
    spec = (((16, 16, 16), 8, 20_000), ((10, 11, 12), 5, 0), ((12, 12, 12), 6, 1_000))
    spls, pos = [], []
    for i, (dims, n_orb, n) in enumerate(spec):
        lat, mil, coef = inputs.random_cell(2490 + i, dims, n_orb, 6.0, 5.0, NONORTHO)
        spls.append(splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True))
        p = inputs.positions(lat, max(n, 1), 2495 + i, -1, 2)[:n]
        pos.append(torch.from_numpy(np.ascontiguousarray(p)).to(dev()).reshape(-1, 3))
    ref = [s.eval_vgl(p) if p.shape[0] else None for s, p in zip(spls, pos)]
    torch.cuda.synchronize()
    for plan in (None, {"launch": "split"}, {"launch": "single", "threads": 512}):
        got = eval_batched(spls, pos, plan=plan)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            if r is None:
                assert all(t.shape[0] == 0 for t in g)
                continue
            for x, y in zip(g, r):
                assert torch.equal(x, y), plan
    v, g_, l = spls[0].eval_vgl_host(torch.zeros((0, 3), dtype=torch.float64))
    assert v.shape[0] == 0 and g_.shape[0] == 0 and l.shape[0] == 0
    for s in spls:
        s.close()
