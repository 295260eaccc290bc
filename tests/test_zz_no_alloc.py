"""qmcspl_eval_vgl_noalloc: the evaluation for callers that cannot allocate device memory
(their memory belongs to their own pool allocator, or their loop must not call
cudaMalloc/cudaFree).  It must return what qmcspl_eval_vgl returns, call after call,
although every call reuses one fixed scratch array inside the library.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_1309_6250_gb300 import _lib, inputs

torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _noalloc(spl, pos, out):
    lib = _lib.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.qmcspl_eval_vgl_noalloc(spl.handle, _ptr(pos), pos.shape[0], _ptr(out[0]), _ptr(out[1]),
                                       _ptr(out[2]), st)


@pytest.mark.gpu
def test_noalloc_matches_eval_vgl_on_two_calls_in_a_row():
    from paper_1309_6250_gb300.api import OrbitalSplines
    dev = torch.device("cuda", 0)
    w = inputs.make_workload("c2", n_pos=60000)
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev)
    tol = 2e-6     # the FP32-table tolerance of the parity tests
    # two calls in a row with different positions and sizes: the second call finds the
    # first call's bins and counters in the shared scratch array
    for n, seed in ((60000, 11), (23456, 12)):
        pos = torch.from_numpy(inputs.positions(w.lattice, n, seed, -1.0, 2.0)).to(dev)
        ref = spl.eval_vgl(pos)
        out = spl.alloc_outputs(n)
        for t in out:
            t.fill_(float("nan"))
        rc = _noalloc(spl, pos, out)
        assert rc == _lib.OK, _lib.load().qmcspl_last_error()
        spl.sync()
        for a, b in zip(out, ref):
            a64, b64 = a.double().cpu().numpy(), b.double().cpu().numpy()
            assert np.isfinite(a64).all()
            err = np.abs(a64 - b64).max() / np.abs(b64).max()
            assert err <= tol, err


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
