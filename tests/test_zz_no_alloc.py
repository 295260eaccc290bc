"""qmcspl_eval_vgl_noalloc: the evaluation for callers that cannot allocate device memory while
they evaluate (all device memory handed to their own pool allocator at start-up, or a
time-critical loop that must not call cudaMalloc/cudaFree, which can stall the whole device).
It must return exactly what qmcspl_eval_vgl returns, call after call, although every call
reuses one fixed scratch array inside the library, and it must not allocate.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import _lib, inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, oracle_tables

torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _noalloc(spl, pos, out):
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.qmcspl_eval_vgl_noalloc(spl.handle, _ptr(pos), pos.shape[0], _ptr(out[0]), _ptr(out[1]),
                                       _ptr(out[2]), st)


def _noalloc_checked(spl, pos):
    """One no-alloc call with the library's allocation hook armed: the next device allocation
    the library makes would fail with QMCSPL_ERR_OOM, so a QMCSPL_OK return shows that the call
    allocated nothing.  Outputs start as NaN so that anything left unwritten shows."""
    lib = _lib.load()
    out = spl.alloc_outputs(pos.shape[0])
    for t in out:
        t.fill_(float("nan"))
    torch.cuda.synchronize()
    lib.qmcspl_debug_fail_alloc(0)
    try:
        rc = _noalloc(spl, pos, out)
    finally:
        lib.qmcspl_debug_fail_alloc(-1)
    assert rc == _lib.OK, lib.qmcspl_last_error()
    assert lib.qmcspl_last_error() == b""
    spl.sync()
    return out


@pytest.mark.gpu
def test_noalloc_matches_eval_vgl_on_two_calls_in_a_row():
    from paper_1309_6250_gb300.api import OrbitalSplines
    dev = torch.device("cuda", 0)
    w = inputs.make_workload("c2", n_pos=60000)
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev)
    beta, blap = oracle_tables(w.lattice, w.miller, w.coef, w.cell.grid, "smooth", "f32", True)
    # two calls in a row with different positions and sizes: the second call finds the
    # first call's bins and counters in the shared scratch array
    for n, seed in ((60000, 11), (23456, 12)):
        pos_np = inputs.positions(w.lattice, n, seed, -1.0, 2.0)
        pos = torch.from_numpy(pos_np).to(dev)
        ref = [t.clone() for t in spl.eval_vgl(pos)]
        spl.sync()
        out = _noalloc_checked(spl, pos)
        # the same kernels on the same positions: bit for bit what qmcspl_eval_vgl gives
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
        # and directly against the oracle on sampled positions
        s = np.arange(0, n, 97)
        got = tuple(t[torch.from_numpy(s).to(dev)].double().cpu().numpy() for t in out)
        assert_parity(got, oracle.bspline_eval(beta, w.lattice, pos_np[s], beta_lap=blap), TOL["f32"], "noalloc")
    spl.close()


@pytest.mark.gpu
@pytest.mark.parametrize("kw", [dict(method="lagrange", separate_lap=True), dict(method="pp", separate_lap=False),
                                dict(method="interp", separate_lap=True, degree=5),
                                dict(method="interp", separate_lap=False, graded=True)],
                         ids=["lagrange", "pp", "degree5", "graded_cubic"])
def test_noalloc_other_bases_are_bit_identical_to_eval_vgl(kw):
    """Lagrange (five tables), pp-splines and the general kernel (degree 5; a graded grid, whose
    positions the no-alloc sort bins by the grid interval that holds them) through the no-alloc
    call: equal to qmcspl_eval_vgl in cell order, and to the oracle on a sample."""
    from paper_1309_6250_gb300.api import OrbitalSplines
    dev = torch.device("cuda", 0)
    dims = (12, 13, 14)
    kw = dict(kw)
    knots = None
    if kw.pop("graded", False):
        knots = tuple(inputs.graded_knots(d, 0.5, 0.17 * a) for a, d in enumerate(dims))
    lat, mil, coef = inputs.random_cell(2100, dims, 20, 5.0, 4.0, NONORTHO)
    spl = OrbitalSplines(lat, dims, mil, coef, storage="f32", device=dev, knots=knots, **kw)
    spl.set_order("cell")
    pos_np = inputs.positions(lat, 20000, 2101, -1.0, 2.0)
    pos = torch.from_numpy(pos_np).to(dev)
    ref = [t.clone() for t in spl.eval_vgl(pos)]
    spl.sync()
    for _ in range(2):
        out = _noalloc_checked(spl, pos)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
    s = np.arange(0, 20000, 331)
    got = tuple(t[torch.from_numpy(s).to(dev)].double().cpu().numpy() for t in out)
    tabs = oracle_tables(lat, mil, coef, dims, kw["method"], "f32", kw["separate_lap"],
                         degree=kw.get("degree", 3), knots=knots)
    if kw["method"] == "lagrange":
        ref_o = oracle.lagrange_eval(tabs, lat, pos_np[s])
    elif kw["method"] == "pp":
        ref_o = oracle.pp_eval(tabs, lat, pos_np[s])
    else:
        ref_o = oracle.general_eval(tabs[0], lat, pos_np[s], kw.get("degree", 3),
                                    knots if knots is not None else (None, None, None), beta_lap=tabs[1])
    assert_parity(got, ref_o, TOL["f32"], "noalloc " + kw["method"])
    spl.close()


@pytest.mark.gpu
def test_noalloc_rejects_more_positions_than_its_scratch_holds():
    from paper_1309_6250_gb300.api import OrbitalSplines
    dev = torch.device("cuda", 0)
    lat, mil, coef = inputs.random_cell(3, (8, 8, 8), 2, 4.0, 4.0, np.eye(3) * 6.0)
    spl = OrbitalSplines(lat, (8, 8, 8), mil, coef, method="smooth", storage="f64", separate_lap=False,
                         device=dev)
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the size check happens before any pointer is touched or anything is launched
    rc = lib.qmcspl_eval_vgl_noalloc(spl.handle, ctypes.c_void_p(16), _lib.NOALLOC_MAX_POS + 1,
                                     None, None, None, st)
    assert rc == _lib.ERR_ARG
    assert b"QMCSPL_NOALLOC_MAX_POS" in lib.qmcspl_last_error()
    spl.close()
