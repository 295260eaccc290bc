"""qmcspl_eval_vgl_host_ex: 16-bit outputs for the host-buffer evaluation.  Each value must be the
round-to-nearest-even bfloat16 / half of the float output qmcspl_eval_vgl gives (bit for bit), the
outputs a caller skips must stay untouched, and handles whose outputs are double or complex are
refused."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, dev, oracle_tables, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("out_dtype", ["bf16", "f16"])
def test_16_bit_host_outputs_are_the_rounded_device_outputs(storage, out_dtype):
    dt = {"bf16": torch.bfloat16, "f16": torch.float16}[out_dtype]
    dims = (12, 13, 14)
    lat, mil, coef = inputs.random_cell(2400, dims, 37, 6.0, 5.0, NONORTHO)   # ragged: 37 orbitals
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    # more positions than one staging chunk (65,536), so both staging buffers take turns
    pos = inputs.positions(lat, 150_001, 2401, -1, 2)
    dv, dg, dl = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    spl.sync()
    hv, hg, hl = spl.eval_vgl_host(torch.from_numpy(pos).pin_memory(), out_dtype=dt)
    for h, d in ((hv, dv), (hg, dg), (hl, dl)):
        assert h.dtype == dt and h.shape == d.shape
        assert torch.equal(h, d.to(dt).cpu())
    # a subset (value and Laplacian, no gradient buffer at all): the same values
    v2, g2, l2 = spl.eval_vgl_host(torch.from_numpy(pos), out=(torch.empty_like(hv), None, torch.empty_like(hl)),
                                   out_dtype=dt)
    assert g2 is None and torch.equal(v2, hv) and torch.equal(l2, hl)
    # against the oracle: within the 16-bit rounding of the largest output of each kind
    s = np.arange(0, pos.shape[0], 997)
    beta, blap = oracle_tables(lat, mil, coef, dims, "smooth", storage, True)
    ref = oracle.bspline_eval(beta, lat, pos[s], beta_lap=blap)
    rel = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}[out_dtype]
    for h, r in zip((hv, hg, hl), ref):
        assert oracle.relative_error(h[s].double().numpy(), r) <= rel
    spl.close()


def test_16_bit_host_outputs_are_refused_for_double_and_complex_outputs():
    from paper_1309_6250_gb300 import _lib
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_cell(2410, dims, 3, 5.0, 4.0, np.eye(3) * 6.0)
    pos = torch.from_numpy(inputs.positions(lat, 100, 2411))
    for kw in (dict(storage="f64"), dict(storage="df64")):
        spl = splines(lat, dims, mil, coef, method="smooth", separate_lap=False, **kw)
        with pytest.raises(_lib.QmcsplError) as ei:
            spl.eval_vgl_host(pos, out_dtype=torch.bfloat16)
        assert ei.value.code == _lib.ERR_UNSUPPORTED
        spl.close()
    k = inputs.KPOINTS["X"]
    bl, bm, bc = inputs.random_bloch_cell(2412, 3, 5.0, 4.0, k, np.eye(3) * 6.0)
    spl = splines(bl, dims, bm, bc, method="smooth", storage="f32", separate_lap=False, kpoint=k)
    with pytest.raises(_lib.QmcsplError) as ei:
        spl.eval_vgl_host(pos, out_dtype=torch.float16)
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    spl.close()
