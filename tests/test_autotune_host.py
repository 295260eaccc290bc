"""Host-side logic of the autotuner: candidate tile shapes, cache keys, cache file."""
import os

from paper_1309_6250_gb300 import autotune


def test_candidate_lanes_keep_padding_small():
    assert autotune.candidate_lanes(128, "f32") == [32, 16, 8, 4, 2]
    assert autotune.candidate_lanes(128, "bf16") == [16, 8, 4, 2]
    # 48 float orbitals = 12 chunks: 16 lanes would pad to 16 chunks (33%), 8 lanes to 16 too
    assert autotune.candidate_lanes(48, "f32") == [4, 2]
    assert autotune.candidate_lanes(3, "f64") == [2]
    assert autotune.candidate_lanes(1, "f32") == [1]
    for n in range(1, 200, 7):
        for st in ("f64", "f32", "bf16"):
            assert autotune.candidate_lanes(n, st)


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    k1 = autotune.cache_key("GB300", "smooth", "f32", True, 128, (96, 96, 96), 524288)
    k2 = autotune.cache_key("GB300", "smooth", "f32", True, 128, (96, 96, 96), 1000)
    assert k1 != k2 and "96x96x96" in k1
    autotune.store_cache(k1, {"lanes": 32, "order": "cell", "ms": 1.0}, path)
    autotune.store_cache(k2, {"lanes": 16, "order": "input", "ms": 0.1}, path)
    d = autotune.load_cache(path)
    assert d[k1]["lanes"] == 32 and d[k2]["order"] == "input"
    with open(path, "w") as f:
        f.write("not json")
    assert autotune.load_cache(path) == {}
    assert os.path.exists(path)


def test_block_shapes_and_batch_plans():
    assert autotune.candidate_threads("f32") == [512, 640]
    assert autotune.candidate_threads("bf16") == [512, 640]
    assert autotune.candidate_threads("f64") == [512] and autotune.candidate_threads("df64") == [512]
    plans = autotune.batch_plans("f32")
    assert {"launch": "split", "threads": 0} in plans
    assert {"launch": "single", "threads": 640} in plans and {"launch": "single", "threads": 512} in plans
    assert all(p["launch"] != "single" or p["threads"] == 512 for p in autotune.batch_plans("f64"))
    # entries of the tuner without the block shape are not read back
    assert autotune.cache_key("GB300", "smooth", "f32", True, 128, (96, 96, 96), 1).startswith(autotune.CACHE_VERSION)
