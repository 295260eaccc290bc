"""Failure detection without a GPU fault: the allocator hook (qmcspl_debug_fail_alloc) makes
one device allocation fail as if the device were full.  Every entry point must report
QMCSPL_ERR_OOM, release what it had allocated and leave the library (and an existing
handle) fully usable; device memory must not drift over repeated failures."""
import numpy as np
import pytest

from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, dev, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture
def lib():
    from paper_1309_6250_gb300 import _lib
    L = _lib.load()
    yield L
    L.qmcspl_debug_fail_alloc(-1)


def scenario(kind, tmp_path):
    """Creation, a cell-ordered evaluation (scratch), a host-buffer evaluation (staging) and a
    save/load round trip; returns the outputs of the loaded handle."""
    from paper_1309_6250_gb300.api import OrbitalSplines
    dims = (12, 12, 12)
    kw = {}
    if kind == "bloch":
        lat, mil, coef = inputs.random_bloch_cell(1600, 4, 5.0, 4.0, inputs.KPOINTS["X"], NONORTHO)
        kw["kpoint"] = inputs.KPOINTS["X"]
    else:
        lat, mil, coef = inputs.random_cell(1601, dims, 6, 5.0, 4.0, NONORTHO)
        if kind == "graded":
            kw["knots"] = tuple(inputs.graded_knots(d, 0.4, 0.1 * a) for a, d in enumerate(dims))
    method = "interp" if kind == "graded" else "smooth"
    spl = splines(lat, dims, mil, coef, method=method, storage="f32", separate_lap=True, **kw)
    pos = torch.from_numpy(inputs.positions(lat, 9000, 1602, -1, 2)).to(dev())
    spl.set_order("cell")
    spl.eval_vgl(pos)
    spl.sync()
    spl.eval_vgl_host(pos[:700].cpu())
    path = tmp_path / ("%s.qmcspl" % kind)
    spl.save(str(path))
    spl.close()
    back = OrbitalSplines.load(str(path), device=dev())
    out = [o.clone() for o in back.eval_vgl(pos[:500])]
    back.sync()
    back.close()
    return out


def failure_pass(lib, kind, tmp_path, ref):
    """Make allocation n fail for n = 0, 1, ... until the scenario completes; every failure
    must be ERR_OOM and a clean run right after it must reproduce `ref`.  Returns the number
    of failures."""
    from paper_1309_6250_gb300 import _lib
    failures = 0
    for n in range(64):
        lib.qmcspl_debug_fail_alloc(n)
        try:
            scenario(kind, tmp_path)
            completed = True
        except _lib.QmcsplError as e:
            assert e.code == _lib.ERR_OOM, (n, e)
            completed = False
            failures += 1
        lib.qmcspl_debug_fail_alloc(-1)
        got = scenario(kind, tmp_path)
        assert all(torch.equal(a, b) for a, b in zip(got, ref)), n
        if completed:
            return failures
    raise AssertionError("the scenario never completed")


def free_device_memory():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("kind", ["real", "bloch", "graded"])
def test_every_allocation_failure_is_reported_and_recovered(lib, kind, tmp_path):
    ref = scenario(kind, tmp_path)
    # construction, cell-order scratch, host staging and load allocations are all hit
    assert failure_pass(lib, kind, tmp_path, ref) >= 5


def test_failures_leak_no_device_memory(lib, tmp_path):
    """Two identical passes of injected failures: a leak would lower the free device memory
    by the same amount each pass; caches do not grow the second time."""
    ref = scenario("graded", tmp_path)
    failure_pass(lib, "graded", tmp_path, ref)
    free_a = free_device_memory()
    failure_pass(lib, "graded", tmp_path, ref)
    free_b = free_device_memory()
    assert free_a - free_b < (8 << 20), (free_a, free_b)


def test_failed_growth_leaves_the_handle_usable(lib):
    """An evaluation whose scratch growth fails reports ERR_OOM; the handle then evaluates
    normally (smaller and larger calls)."""
    from paper_1309_6250_gb300 import _lib
    dims = (10, 10, 10)
    lat, mil, coef = inputs.random_cell(1603, dims, 5, 5.0, 4.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=False)
    small = torch.from_numpy(inputs.positions(lat, 100, 1604)).to(dev())
    big = torch.from_numpy(inputs.positions(lat, 20000, 1605)).to(dev())
    ref_small = [o.clone() for o in spl.eval_vgl(small)]
    spl.sync()
    lib.qmcspl_debug_fail_alloc(0)
    with pytest.raises(_lib.QmcsplError) as ei:
        spl.eval_vgl(big)              # first call of this size: the scratch must grow
    assert ei.value.code == _lib.ERR_OOM
    lib.qmcspl_debug_fail_alloc(-1)
    spl.sync()
    assert all(torch.equal(a, b) for a, b in zip(spl.eval_vgl(small), ref_small))
    v, g, l = spl.eval_vgl(big)
    spl.sync()
    assert torch.isfinite(v).all() and torch.equal(v[:0], v[:0])
    spl.close()
