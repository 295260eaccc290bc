"""Autotuner for the evaluation launch shape.

Per handle, three choices set how the evaluation kernels map work onto the GPU:
  * lanes   -- threads that share one position (each owns one 16-byte chunk of every
               stored row, i.e. 2, 4 or 8 orbitals for f64, f32, bf16 tables), so that
               positions per warp = 32 / lanes and orbital tiles = row chunks / lanes;
  * threads -- the block shape of the B-spline kernel (512, or 640 for float and bfloat16
               tables): positions per CTA = threads / lanes, one CTA per SM;
  * order   -- input order, or positions sorted into spatial cell bins first.
tune() builds the tables once per candidate `lanes`, times the evaluation of a sample of
positions for every (threads, order) with the library's CUDA-event timing (qmcspl_profile),
and returns the fastest.  For a batch of cells, tune_batch() times the whole batched call,
replayed from a CUDA graph, under each launch plan (one launch per cell, or every cell in the
one persistent batched launch with 512 or 640 threads per block) and returns the fastest.
Results are cached in a JSON file keyed by GPU name and workload.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

_lock = threading.Lock()

ELEM_BYTES = {"f64": 8, "df64": 8, "f32": 4, "bf16": 2}
CACHE_VERSION = "v2"     # entries carry lanes, threads and order


def default_cache_path() -> str:
    return os.environ.get("QMCSPL_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "qmcspl", "autotune.json"))


def candidate_lanes(n_orb: int, storage: str, max_padding: float = 0.25) -> List[int]:
    """Lane counts whose row padding stays within `max_padding` of the row."""
    per_chunk = 16 // ELEM_BYTES[storage]
    chunks = -(-n_orb // per_chunk)
    out = [L for L in (32, 16, 8, 4, 2) if -(-chunks // L) * L <= (1 + max_padding) * chunks]
    return out or [1]


def candidate_threads(storage: str) -> List[int]:
    """Block shapes the B-spline kernel is compiled for with this table type."""
    return [512, 640] if storage in ("f32", "bf16") else [512]


def cache_key(gpu: str, method: str, storage: str, separate_lap: bool, n_orb: int,
              dims: Sequence[int], n_pos: int) -> str:
    bucket = int(math.log2(max(1, n_pos)))
    return "%s|%s|%s|%s|%d|%d|%s|p2^%d" % (CACHE_VERSION, gpu, method, storage, int(bool(separate_lap)), n_orb,
                                            "x".join(str(int(d)) for d in dims), bucket)


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(key: str, value: dict, path: Optional[str] = None) -> None:
    path = path or default_cache_path()
    with _lock:
        d = load_cache(path)
        d[key] = value
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = "%s.%d.tmp" % (path, os.getpid())
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time_eval(spl, pos, repeats: int) -> float:
    import torch
    out = spl.alloc_outputs(pos.shape[0])
    for _ in range(2):
        spl.eval_vgl(pos, out=out)
    torch.cuda.synchronize()
    spl.profile(True)
    for _ in range(repeats):
        spl.eval_vgl(pos, out=out)
    prof = spl.profile_read()
    spl.profile(False)
    spl.sync()
    return (prof["eval_ms"] + prof["order_ms"]) / max(1, prof["launches"])


def tune(lattice, dims, miller, coef, positions, method: str = "smooth", storage: str = "f32",
         separate_lap: bool = True, device=None, repeats: int = 10,
         lanes: Optional[Iterable[int]] = None, orders: Sequence[str] = ("input", "cell"),
         threads: Optional[Iterable[int]] = None, cache_path: Optional[str] = None,
         force: bool = False) -> dict:
    """Fastest {'lanes', 'threads', 'order', 'ms'} for this table and position sample."""
    import torch
    from .api import OrbitalSplines
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    pos = positions if isinstance(positions, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(positions))
    pos = pos.to(device=dev, dtype=torch.float64).reshape(-1, 3).contiguous()
    n_orb = np.asarray(coef).reshape(-1, np.asarray(miller).reshape(-1, 3).shape[0]).shape[0]
    key = cache_key(torch.cuda.get_device_name(dev), method, storage, separate_lap, n_orb, dims, pos.shape[0])
    if not force:
        hit = load_cache(cache_path).get(key)
        if hit is not None:
            return hit
    bspline = method in ("smooth", "interp")
    shapes = list(threads) if threads is not None else (candidate_threads(storage) if bspline else [0])
    trials = []
    for L in (list(lanes) if lanes is not None else candidate_lanes(n_orb, storage)):
        spl = OrbitalSplines(lattice, dims, miller, coef, method=method, storage=storage,
                             separate_lap=separate_lap, device=dev, lanes=L)
        for th in shapes:
            if bspline:
                spl.set_block(th)
            for order in orders:
                spl.set_order(order)
                trials.append({"lanes": L, "threads": th, "order": order, "ms": _time_eval(spl, pos, repeats)})
        spl.close()
        torch.cuda.empty_cache()
    best = min(trials, key=lambda t: t["ms"])
    result = {"lanes": best["lanes"], "threads": best["threads"], "order": best["order"], "ms": best["ms"],
              "trials": trials}
    store_cache(key, result, cache_path)
    return result


def tuned_splines(lattice, dims, miller, coef, positions, method: str = "smooth", storage: str = "f32",
                  separate_lap: bool = True, device=None, cache_path: Optional[str] = None, **kw):
    """OrbitalSplines built and set up with the tuned launch shape (tuning on a miss)."""
    from .api import OrbitalSplines
    t = tune(lattice, dims, miller, coef, positions, method=method, storage=storage,
             separate_lap=separate_lap, device=device, cache_path=cache_path, **kw)
    spl = OrbitalSplines(lattice, dims, miller, coef, method=method, storage=storage,
                         separate_lap=separate_lap, device=device, lanes=t["lanes"])
    if method in ("smooth", "interp"):
        spl.set_block(t.get("threads", 0))
    spl.set_order(t["order"])
    return spl, t


def batch_plans(storage: str) -> List[dict]:
    """Launch plans of qmcspl_eval_batched_ex worth trying for this table type."""
    plans = [{"launch": "split", "threads": 0}]
    plans += [{"launch": "single", "threads": th} for th in candidate_threads(storage)]
    return plans


def time_batch_graph(splines, positions, outs, plan, repeats: int = 20) -> float:
    """Mean ms of one batched call (sorting kernels and evaluation launches of every cell) replayed
    from a CUDA graph on the current stream."""
    import torch
    from .api import eval_batched
    stream = torch.cuda.current_stream()
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        eval_batched(splines, positions, outs=outs, stream=cap, plan=plan)   # sizes the scratch
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=cap):
            eval_batched(splines, positions, outs=outs, stream=cap, plan=plan)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(repeats)]
    for a, b in ev:
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / repeats


def tune_batch(splines, positions, outs=None, storage: str = "f32", key: Optional[str] = None,
               repeats: int = 20, cache_path: Optional[str] = None, force: bool = False) -> dict:
    """Fastest launch plan {'launch', 'threads', 'ms'} for this batch of cells (each already set
    up with its own tuned shape), timed as CUDA-graph replays of the whole call."""
    import torch
    if key is not None:
        key = "%s|batch|%s|%s|%s" % (CACHE_VERSION, torch.cuda.get_device_name(splines[0].device), storage, key)
        if not force:
            hit = load_cache(cache_path).get(key)
            if hit is not None:
                return hit
    if outs is None:
        outs = [s.alloc_outputs(p.reshape(-1, 3).shape[0]) for s, p in zip(splines, positions)]
    trials = []
    for plan in batch_plans(storage):
        trials.append(dict(plan, ms=time_batch_graph(splines, positions, outs, plan, repeats)))
    best = min(trials, key=lambda t: t["ms"])
    result = {"launch": best["launch"], "threads": best["threads"], "ms": best["ms"], "trials": trials}
    if key is not None:
        store_cache(key, result, cache_path)
    return result
