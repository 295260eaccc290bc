"""The C-ABI library loads and exports every entry point of include/qmcspl.h; host-side
validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1309_6250_gb300 import _lib, build as pkg_build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qmcspl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qmcspl_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "qmcspl_create" in names and "qmcspl_eval_vgl_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    assert {p[0] for p in _lib.PROTOTYPES} == set(names)


def test_version_and_empty_error(lib):
    assert lib.qmcspl_version() >= 10000
    assert lib.qmcspl_last_error() == b""


def _create(lib, lattice, dims, miller, coef, method=0, storage=0, sep=0, bloch=0, kpoint=(0.0, 0.0, 0.0),
            sep_grad=0):
    h = ctypes.c_void_p()
    lat = np.ascontiguousarray(lattice, dtype=np.float64)
    dm = np.ascontiguousarray(dims, dtype=np.int32)
    mil = np.ascontiguousarray(miller, dtype=np.int32)
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.complex128)).view(np.float64)
    opts = _lib.Opts(method, storage, sep, 0, sep_grad, bloch, (ctypes.c_double * 3)(*kpoint))
    rc = lib.qmcspl_create(ctypes.byref(h), lat.ctypes.data, dm.ctypes.data, mil.shape[0],
                           mil.ctypes.data, c.shape[0], c.ctypes.data, ctypes.byref(opts), None)
    return rc, h


def test_validation_without_gpu(lib):
    lat, mil, coef = inputs.random_cell(1, (8, 8, 8), 2, 4.0, 4.0, np.eye(3) * 6.0)
    # bad grid
    rc, h = _create(lib, lat, (3, 8, 8), mil, coef)
    assert rc == _lib.ERR_ARG and h.value is None
    # singular lattice
    rc, _ = _create(lib, np.zeros((3, 3)), (8, 8, 8), mil, coef)
    assert rc == _lib.ERR_ARG and b"singular" in lib.qmcspl_last_error()
    # unknown method / storage
    assert _create(lib, lat, (8, 8, 8), mil, coef, method=9)[0] == _lib.ERR_ARG
    assert _create(lib, lat, (8, 8, 8), mil, coef, storage=7)[0] == _lib.ERR_ARG
    # non-Hermitian: break c_{-G} = conj(c_G)
    bad = coef.copy()
    k = int(np.nonzero(np.any(mil != 0, axis=1))[0][0])
    bad[0, k] += 0.1
    rc, _ = _create(lib, lat, (8, 8, 8), mil, bad)
    assert rc == _lib.ERR_NOT_HERMITIAN
    # a planewave without its -G partner
    k = int(np.nonzero(np.any(mil != 0, axis=1))[0][0])
    keep = np.arange(mil.shape[0]) != k
    rc, _ = _create(lib, lat, (8, 8, 8), mil[keep], coef[:, keep])
    assert rc == _lib.ERR_NOT_HERMITIAN and b"partner" in lib.qmcspl_last_error()
    # duplicated G
    rc, _ = _create(lib, lat, (8, 8, 8), np.vstack([mil, mil[:1]]), np.hstack([coef, coef[:, :1]]))
    assert rc == _lib.ERR_ARG and b"duplicate" in lib.qmcspl_last_error()
    # Bloch options: flag must be 0/1, k finite; duplicates are still rejected
    assert _create(lib, lat, (8, 8, 8), mil, coef, bloch=2)[0] == _lib.ERR_ARG
    rc, _ = _create(lib, lat, (8, 8, 8), mil, coef, bloch=1, kpoint=(0.5, float("nan"), 0.0))
    assert rc == _lib.ERR_ARG and b"kpoint" in lib.qmcspl_last_error()
    rc, _ = _create(lib, lat, (8, 8, 8), np.vstack([mil, mil[:1]]), np.hstack([coef, coef[:, :1]]),
                    bloch=1, kpoint=(0.5, 0.0, 0.0))
    assert rc == _lib.ERR_ARG and b"duplicate" in lib.qmcspl_last_error()
    nonfinite = coef.copy()
    nonfinite[0, 0] = np.nan
    rc, _ = _create(lib, lat, (8, 8, 8), mil, nonfinite, bloch=1, kpoint=(0.5, 0.0, 0.0))
    assert rc == _lib.ERR_ARG and b"non-finite" in lib.qmcspl_last_error()
    # separate gradient tables need the Laplacian table
    rc, _ = _create(lib, lat, (8, 8, 8), mil, coef, sep=0, sep_grad=1)
    assert rc == _lib.ERR_ARG and b"separate_lap" in lib.qmcspl_last_error()
    # NULL handle calls
    assert lib.qmcspl_eval_vgl(None, None, 0, None, None, None, None) == _lib.ERR_ARG
    assert lib.qmcspl_sync(None, None) == _lib.ERR_ARG
    assert lib.qmcspl_set_table(None, 0, None, _lib.F64, None) == _lib.ERR_ARG
    assert lib.qmcspl_set_block(None, 512) == _lib.ERR_ARG
    assert lib.qmcspl_probe_cache(3, None, None, None, None) == _lib.ERR_ARG
    assert lib.qmcspl_probe_fma(2, None, None, None, None) == _lib.ERR_ARG
    order = ctypes.c_int(-1)
    assert lib.qmcspl_get_order(None, 100, ctypes.byref(order)) == _lib.ERR_ARG and order.value == -1
    assert lib.qmcspl_eval_vgl_host_ex(None, None, 0, None, None, None, ctypes.byref(_lib.HostOpts(1)), None) == _lib.ERR_ARG
    bad_plan = _lib.BatchOpts(7, 0)
    assert lib.qmcspl_eval_batched_ex(1, None, None, None, None, None, None, ctypes.byref(bad_plan), None) == _lib.ERR_ARG
    assert b"plan" in lib.qmcspl_last_error()
    assert lib.qmcspl_eval_vgl_noalloc(None, None, 0, None, None, None, None) == _lib.ERR_ARG
    assert lib.qmcspl_destroy(None) == _lib.OK


def test_grid_options_validated_without_gpu(lib):
    """qmcspl_create_grid checks degree, method and grid points before touching the device."""
    lat, mil, coef = inputs.random_cell(2, (8, 8, 8), 2, 4.0, 4.0, np.eye(3) * 6.0)

    def create(degree, knots, method=1, storage=0):
        h = ctypes.c_void_p()
        latc = np.ascontiguousarray(lat)
        dm = np.array([8, 8, 8], dtype=np.int32)
        c = np.ascontiguousarray(coef.astype(np.complex128)).view(np.float64)
        opts = _lib.Opts(method, storage, 0, 0)
        ks = [None if k is None else np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        g = _lib.GridOpts(degree, (ctypes.c_void_p * 3)(*[None if k is None else k.ctypes.data for k in ks]))
        return lib.qmcspl_create_grid(ctypes.byref(h), latc.ctypes.data, dm.ctypes.data, mil.shape[0],
                                      mil.ctypes.data, coef.shape[0], c.ctypes.data, ctypes.byref(opts),
                                      ctypes.byref(g), None)

    u = np.arange(8) / 8.0
    assert create(4, (None,) * 3) == _lib.ERR_ARG                       # even degree
    assert create(5, (None,) * 3, method=2) == _lib.ERR_UNSUPPORTED     # Lagrange, degree 5
    assert create(3, (u, u, u), method=0) == _lib.ERR_UNSUPPORTED       # smoothing, non-uniform
    assert create(5, (None,) * 3, storage=3) == _lib.ERR_UNSUPPORTED    # double-float
    assert create(3, (u, None, u)) == _lib.ERR_ARG                      # one axis missing
    assert create(7, (None, u, u)) == _lib.ERR_ARG                      # the same, degree 7
    bad = u.copy()
    bad[3] = bad[2]
    assert create(3, (u, bad, u)) == _lib.ERR_ARG and b"increasing" in lib.qmcspl_last_error()
    out = u.copy()
    out[7] = 1.0
    assert create(3, (u, u, out)) == _lib.ERR_ARG


def test_load_rejects_bad_files_without_gpu(lib, tmp_path):
    """qmcspl_load validates the file before touching the device."""
    h = ctypes.c_void_p()
    missing = str(tmp_path / "none.qmcspl").encode()
    assert lib.qmcspl_load(ctypes.byref(h), missing, None) == _lib.ERR_ARG
    bad = tmp_path / "bad.qmcspl"
    bad.write_bytes(b"NOTQMCSP" + b"\0" * 4096)
    assert lib.qmcspl_load(ctypes.byref(h), str(bad).encode(), None) == _lib.ERR_ARG
    assert b"not a qmcspl table file" in lib.qmcspl_last_error()
    short = tmp_path / "short.qmcspl"
    short.write_bytes(b"QMCSPLTB")
    assert lib.qmcspl_load(ctypes.byref(h), str(short).encode(), None) == _lib.ERR_ARG
    assert h.value is None
    assert lib.qmcspl_save(None, b"/tmp/x") == _lib.ERR_ARG
