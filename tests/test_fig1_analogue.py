"""The Fig. 1 analogue (Sec. III A) through the GPU library: its error table equals the
oracle's, so the paper's accuracy conclusions hold for the CUDA path as well."""
import pytest

import fig1_analogue as f1
from gpu_helpers import dev

pytestmark = pytest.mark.gpu

ECUTS = (10.0, 20.0, 40.0)


@pytest.mark.parametrize("storage,rel", [("f64", 1e-9), ("f32", 1e-4)])
def test_fig1_table_matches_the_oracle(storage, rel):
    got = f1.run(ECUTS, storage=storage, n_orb=8, n_pos=800, device=dev())
    ref = f1.run(ECUTS, use_oracle=True, n_orb=8, n_pos=800)
    for g, r in zip(got, ref):
        assert (g["ecut"], g["row"]) == (r["ecut"], r["row"])
        for what in ("value", "grad", "lap"):
            assert g[what] == pytest.approx(r[what], rel=rel), (g["ecut"], g["row"], what)
    for ecut in ECUTS:
        r = {x["row"]: x for x in got if x["ecut"] == ecut}
        assert r["smooth"]["value"] < r["interp"]["value"] < r["lagrange"]["value"]
        assert r["smooth_sep"]["lap"] < r["smooth"]["lap"]


def test_higher_degree_is_more_accurate_at_natural_spacing():
    """Interpolating B-splines of higher odd degree approximate the planewave value better at
    the same (natural) grid spacing: degree 1 > 3 > 5 > 7 in relative MAE."""
    rows = f1.run_degrees((10.0, 20.0), storage="f64", n_orb=8, n_pos=400, device=dev())
    for ecut in (10.0, 20.0):
        v = [r["value"] for r in rows if r["ecut"] == ecut]
        assert v[0] > v[1] > v[2] > v[3]
