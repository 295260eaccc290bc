"""GPU Bloch orbitals at k != 0 (Sec. II: phi = u exp(i k.r)) against the oracle.

Every case goes through the C ABI (OrbitalSplines with a kpoint).  The oracle builds the
tables of the complex periodic part u from the same planewaves and evaluates them with
its own loops, then multiplies by exp(i k.r) with the product rule."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, oracle_tables, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KGEN = inputs.KPOINTS["generic"]


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def gpu_eval_c(spl, pos):
    v, g, l = spl.eval_vgl(t(pos))
    spl.sync()
    return (v.cpu().numpy().astype(np.complex128), g.cpu().numpy().astype(np.complex128),
            l.cpu().numpy().astype(np.complex128))


def oracle_reference(method, storage, lat, mil, coef, kp, dims, pos, sep):
    """Oracle evaluation of the oracle's own tables, rounded the way the GPU stores them."""
    tabs = oracle_tables(lat, mil, coef, dims, method, storage, sep, kpoint=kp)
    if method in ("smooth", "interp"):
        return oracle.bloch_eval(method, tabs[0], lat, kp, pos, tables_lap=tabs[1])
    return oracle.bloch_eval(method, tabs, lat, kp, pos)


CASES = ([("smooth", s, sep) for s in ("f64", "f32", "bf16", "df64") for sep in (False, True)] +
         [("interp", s, sep) for s in ("f64", "f32", "df64") for sep in (False, True)] +
         [("lagrange", s, False) for s in ("f64", "f32", "bf16")] +
         [("pp", s, False) for s in ("f64", "f32", "bf16")])


@pytest.mark.parametrize("method,storage,sep", CASES)
def test_bloch_tables_and_outputs_match_oracle(method, storage, sep):
    """Ragged band count (5 bands = 10 stored functions), non-orthogonal cell, positions
    outside the cell (the phase uses the unwrapped position)."""
    dims = (9, 10, 11)
    lat, mil, coef = inputs.random_bloch_cell(900, 5, 6.0, 5.0, KGEN, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep, kpoint=KGEN)
    inf = spl.info()
    assert inf["bloch"] == 1 and inf["n_orb"] == 5 and np.allclose(inf["kpoint"], KGEN)
    # tables: the stored values are the oracle's tables rounded to the storage type
    ref_t = oracle.bloch_tables(method, lat, mil, coef, KGEN, dims, laplacian=sep)
    if method in ("smooth", "interp"):
        pairs = [(spl.get_table(0), ref_t[0])] + ([(spl.get_table(1), ref_t[1])] if sep else [])
    else:
        pairs = [(spl.get_table(i), ref_t[i]) for i in range(ref_t.shape[0])]
    ttol = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-7, "bf16": 8e-3}[storage]
    for got, ref in pairs:
        assert oracle.relative_error(got, ref) < ttol
    pos = inputs.positions(lat, 300, 901, -1, 2)
    got = gpu_eval_c(spl, pos)
    ref = oracle_reference(method, storage, lat, mil, coef, KGEN, dims, pos, sep)
    assert_parity(got, ref, TOL[storage], "bloch %s/%s/sep=%d" % (method, storage, sep))
    # the planewave sum itself, within the approximation error (grid above natural spacing)
    if storage == "f64" and method != "lagrange":
        pv, _, _ = oracle.bloch_pw_eval(lat, mil, coef, KGEN, pos)
        assert oracle.relative_mean_absolute_error(got[0], pv) < 5e-2
    spl.close()


def test_bloch_orders_lanes_and_graph_are_bit_identical():
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_bloch_cell(910, 24, 6.0, 5.0, KGEN, NONORTHO)
    pos = t(inputs.positions(lat, 20000, 911, -2, 3))
    ref = None
    for lanes in (0, 4):
        spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True,
                      kpoint=KGEN, lanes=lanes)
        for order in ("input", "cell"):
            spl.set_order(order)
            out = spl.eval_vgl(pos)
            spl.sync()
            if ref is None:
                ref = [o.clone() for o in out]
            else:
                assert all(torch.equal(a, b) for a, b in zip(out, ref))
        # CUDA graph replay of the whole step (per-position pass + evaluation)
        outs = spl.alloc_outputs(pos.shape[0])
        spl.eval_vgl(pos, out=outs)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                spl.eval_vgl(pos, out=outs, stream=side)
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(outs, ref))
        spl.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_bloch_at_gamma_equals_the_real_path(storage):
    """k = 0 with Hermitian coefficients: the real part is the real path's output, the
    imaginary part vanishes."""
    dims = (10, 10, 12)
    lat, mil, coef = inputs.random_cell(920, dims, 6, 6.0, 5.0, NONORTHO)
    pos = inputs.positions(lat, 500, 921, -1, 2)
    real = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    cplx = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True,
                   kpoint=(0.0, 0.0, 0.0))
    rv = [o.cpu().numpy().astype(np.float64) for o in real.eval_vgl(t(pos))]
    cv = gpu_eval_c(cplx, pos)
    for a, b in zip(cv, rv):
        assert oracle.relative_error(a.real, b) < (1e-15 if storage == "f64" else 1e-6)
        assert np.abs(a.imag).max() < 1e-6 * np.abs(b).max()


def test_bloch_batched_and_host_buffers():
    """Two Bloch cells with different k in one batched launch equal their own launches;
    the host-buffer path equals the device path."""
    from paper_1309_6250_gb300.api import eval_batched
    cells = []
    for i, (kp, dims, nb) in enumerate([(KGEN, (10, 11, 12), 7), (inputs.KPOINTS["X"], (12, 12, 12), 16)]):
        lat, mil, coef = inputs.random_bloch_cell(930 + i, nb, 6.0, 5.0, kp, NONORTHO)
        spl = splines(lat, dims, mil, coef, method="interp", storage="f32", separate_lap=True, kpoint=kp)
        pos = t(inputs.positions(lat, 5000 + 3000 * i, 940 + i, -1, 2))
        cells.append((spl, pos))
    outs = eval_batched([c[0] for c in cells], [c[1] for c in cells])
    torch.cuda.synchronize()
    for (spl, pos), o in zip(cells, outs):
        ref = spl.eval_vgl(pos)
        spl.sync()
        assert all(torch.equal(a, b) for a, b in zip(o, ref))
    spl, pos = cells[1]
    hv, hg, hl = spl.eval_vgl_host(pos.cpu())
    dv, dg, dl = spl.eval_vgl(pos)
    torch.cuda.synchronize()
    assert torch.equal(hv, dv.cpu()) and torch.equal(hg, dg.cpu()) and torch.equal(hl, dl.cpu())


def test_bloch_rejections_and_checkpoint(tmp_path):
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import OrbitalSplines, eval_batched
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_bloch_cell(950, 3, 5.0, 4.0, KGEN, np.eye(3) * 6.0)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=False, kpoint=KGEN)
    pos = t(inputs.positions(lat, 64, 951, -1, 2))
    lib = _lib.load()
    out = spl.alloc_outputs(64)
    rc = lib.qmcspl_eval_vgl_noalloc(spl.handle, pos.data_ptr(), 64, out[0].data_ptr(),
                                     out[1].data_ptr(), out[2].data_ptr(), None)
    assert rc == _lib.ERR_UNSUPPORTED
    # real and Bloch handles do not share a batch
    rl, rm, rc_ = inputs.random_cell(952, dims, 2, 5.0, 4.0, np.eye(3) * 6.0)
    real = splines(rl, dims, rm, rc_, method="smooth", storage="f64", separate_lap=False)
    with pytest.raises(_lib.QmcsplError) as ei:
        eval_batched([spl, real], [pos, pos])
    assert ei.value.code == _lib.ERR_ARG
    # save / load keeps the k point and gives identical outputs
    path = tmp_path / "bloch.qmcspl"
    spl.save(str(path))
    back = OrbitalSplines.load(str(path), device=dev())
    assert back.bloch and np.allclose(back.kpoint, KGEN)
    a = spl.eval_vgl(pos)
    b = back.eval_vgl(pos)
    torch.cuda.synchronize()
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    back.close()
    spl.close()


@pytest.mark.slow
def test_bloch_c3_mgo64_full_size_sampled():
    """MgO-like 64-atom cell with 64 complex bands at the zone corner R on 96^3 (the same
    table bytes as the 128 real orbitals), 2048 x 256 positions, smoothing + Laplacian
    table in FP32, checked on a sample against the oracle."""
    kp = inputs.KPOINTS["R"]
    w = inputs.make_bloch_workload("c3", kp)
    P = w.pos.shape[0]
    sample = np.unique(np.concatenate([np.arange(0, P, 8191), np.arange(P - 5, P)]))
    outs = [[], [], []]
    for o0 in range(0, w.coef.shape[0], 8):
        beta, blap = oracle.bloch_tables("smooth", w.lattice, w.miller, w.coef[o0:o0 + 8], kp,
                                         w.cell.grid, laplacian=True)
        r = oracle.bloch_eval("smooth", beta, w.lattice, kp, w.pos[sample], tables_lap=blap)
        for k in range(3):
            outs[k].append(r[k])
    ref = tuple(np.concatenate(o, axis=-1) for o in outs)
    spl = splines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                  separate_lap=True, kpoint=kp)
    v, g, l = spl.eval_vgl(t(w.pos))
    spl.sync()
    s = torch.from_numpy(sample).to(dev())
    got = tuple(x[s].cpu().numpy().astype(np.complex128) for x in (v, g, l))
    errs = assert_parity(got, ref, TOL["f32"], "bloch c3/f32")
    print("bloch c3 f32 sampled errors: %s" % ["%.2e" % e for e in errs])
    spl.close()
