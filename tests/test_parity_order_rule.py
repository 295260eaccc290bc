"""The automatic visiting order (QMCSPL_ORDER_AUTO, reported by qmcspl_get_order): cell order from
8192 positions for tables larger than L2; for tables that fit, once the positions per bin of
4 x 4 x 4 cells reach 8, 32 or 192 (tables filling more than 60 %, more than 30 %, at most 30 %
of L2).  Whatever the order, the outputs are the same bytes as those of the order it resolves to."""
import numpy as np
import pytest

from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, dev, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _expected(spl, n_pos):
    if n_pos < 8192:
        return "input"
    info = spl.info()
    share = info["table_bytes"] / torch.cuda.get_device_properties(dev()).L2_cache_size
    if share > 1.0:
        return "cell"
    bins = int(np.prod([(d + 3) // 4 for d in info["dims"]]))
    need = 8.0 if share > 0.6 else 32.0 if share > 0.3 else 192.0
    return "cell" if n_pos / bins >= need else "input"


@pytest.mark.parametrize("dims,n_orb", [((48, 48, 48), 16), ((40, 40, 40), 96), ((64, 64, 64), 160)])
def test_automatic_order_follows_the_rule(dims, n_orb):
    lat, mil, coef = inputs.random_cell(2440 + n_orb, dims, n_orb, 3.0, 4.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True)
    seen = set()
    for n in (1000, 8192, 32768, 131072, 524288):
        got = spl.resolved_order(n)
        assert got == _expected(spl, n), (dims, n_orb, n)
        seen.add(got)
    assert "input" in seen    # below 8192 positions
    # an explicit order is reported as it is
    for mode in ("input", "cell"):
        spl.set_order(mode)
        assert spl.resolved_order(524288) == mode
    # auto gives exactly the bytes of the order it resolves to
    n = 40000
    pos = torch.from_numpy(inputs.positions(lat, n, 2441, -1, 2)).to(dev())
    spl.set_order("auto")
    resolved = spl.resolved_order(n)
    a = spl.eval_vgl(pos)
    spl.set_order(resolved)
    b = spl.eval_vgl(pos)
    spl.sync()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    spl.close()


@pytest.mark.parametrize("n_orb,staged", [(32, True), (16, False)])
def test_pencil_order_is_reported_where_the_staged_kernel_applies(n_orb, staged):
    """Pencil order takes the shared-memory-staged kernel only for cubic B-splines whose rows
    are 128, 256 or 512 bytes (32 FP32 orbitals here); other handles evaluate in cell order,
    and qmcspl_get_order says which."""
    dims = (16, 16, 16)
    lat, mil, coef = inputs.random_cell(2480 + n_orb, dims, n_orb, 3.0, 4.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=True)
    assert bool(spl.info()["staged"]) == staged
    spl.set_order("pencil")
    assert spl.resolved_order(20000) == ("pencil" if staged else "cell")
    assert spl.resolved_order(0) == "input"
    spl.close()
