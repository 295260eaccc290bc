"""Benchmark: orbital x position evaluations per second (value + gradient + Laplacian).

Workload (default): the MgO-like 64-atom cell -- cubic a = 15.9 bohr, 128 real
orbitals with |G|^2/2 <= 40 Ha and coefficient envelope exp(-|G|^2/8), smoothing
B-spline on a 96^3 grid with the separate Laplacian table, 2048 walkers x 256
electrons (524,288 positions) uniform in the cell.  A step is one evaluation of every
orbital at every position (table construction is setup, reported separately).

`value` is timed with CUDA events on the launching stream with positions already in
HBM; `e2e` goes through the host-buffer entry point (pinned host positions in,
host outputs back) every step.  The table (934 MB for FP32) and the outputs
(1.34 GB) are both far larger than the 129 MB L2, so no extra flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1309_6250_gb300 import inputs  # noqa: E402

METRIC = "orbital x position evals/s (val+grad+lap)"
UNIT = "evals/s"
KERNEL_SOURCES = ["paper_1309_6250_gb300/csrc/eval_bspline.cu", "paper_1309_6250_gb300/csrc/eval_common.cuh"]
# the 128-orbital method legs run kernels of both evaluation files
METHOD_SOURCES = KERNEL_SOURCES + ["paper_1309_6250_gb300/csrc/eval_variants.cu"]


def out_bytes(storage):
    return 8 if storage in ("f64", "df64") else 4


def elem_bytes(storage):
    return {"f64": 8, "df64": 8, "f32": 4, "bf16": 2}[storage]


def algorithmic_bytes_per_eval(storage, n_tables, n_orb):
    """Gathered table bytes (64 coefficients per table) + 5 outputs per orbital-eval
    + the position (24 B) shared by the orbitals."""
    return n_tables * 64 * elem_bytes(storage) + 5 * out_bytes(storage) + 24.0 / n_orb


def kernel_source_hash(sources=None):
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(key, sources=None):
    """Bytes per launch from the committed ncu capture, if it was taken on the current kernel
    source: {'dram': DRAM read + write bytes, 'l2': L2 bytes or None}; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(key)
    if not e or e.get("kernel_source_sha") != kernel_source_hash(sources):
        return None
    return {"dram": e.get("dram_bytes_per_launch"), "l2": e.get("l2_bytes_per_launch")}


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None
        self.first = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample (it takes a while to start)."""
        if self.proc is not None:
            self.first.wait(timeout)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    from paper_1309_6250_gb300.replicas import env_rank_world
    rank, ws, local = env_rank_world()
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    import torch
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, ws, dist


def time_steps(fn, steps, warmup, torch, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def rounded_table(t, storage):
    """A table as the GPU stores it (FP32 or BF16 rounding), back in float64."""
    import oracle
    return oracle.round_to_storage(t, storage)


TOLERANCE = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "bf16": 1e-2}


def precision_report(storage, got, ref_fp64, ref_stored, sample_desc):
    """Error of sampled GPU outputs per output (value, gradient, Laplacian), as
    max |gpu - oracle| / max |oracle|:
      max_rel_err_vs_fp64 -- against the oracle on the unrounded FP64 tables: what the storage
                             type costs, plus the kernel's arithmetic;
      max_rel_err_arith   -- against the oracle on the tables rounded the way the GPU stores
                             them: the kernel's arithmetic alone (the parity tests' tolerance);
      dT_mHa              -- the largest change of the kinetic-energy estimate
                             T_n = -1/2 sum_p phi_n lap phi_n / sum_p phi_n^2 (Sec. I local energy,
                             Sec. III A on the Laplacian) over the sampled positions, in mHa,
                             against the unrounded FP64 oracle."""
    import oracle
    names = ("val", "grad", "lap")
    vs64 = {k: float(oracle.relative_error(g, r)) for k, g, r in zip(names, got, ref_fp64)}
    arith = {k: float(oracle.relative_error(g, r)) for k, g, r in zip(names, got, ref_stored)}
    if np.iscomplexobj(got[0]):
        # Bloch outputs: T_n from Re(conj(phi) lap phi) / |phi|^2
        t_gpu = -0.5 * np.sum((np.conj(got[0]) * got[2]).real, 0) / np.sum(np.abs(got[0]) ** 2, 0)
        t_ref = -0.5 * np.sum((np.conj(ref_fp64[0]) * ref_fp64[2]).real, 0) / np.sum(np.abs(ref_fp64[0]) ** 2, 0)
    else:
        t_gpu = oracle.kinetic_energy(got[0], got[2])
        t_ref = oracle.kinetic_energy(ref_fp64[0], ref_fp64[2])
    tol = TOLERANCE[storage]
    return {"max_rel_err_vs_fp64": vs64, "max_rel_err_arith": arith,
            "dT_mHa": float(1e3 * np.max(np.abs(t_gpu - t_ref))), "T_max_Ha": float(np.max(np.abs(t_ref))),
            "tolerance": tol, "ok": all(e <= tol for e in arith.values()), "sample": sample_desc,
            "reference": "FP64 oracle (oracle/), tables built by the oracle from the same planewaves"}


def bspline_precision(w, storage, sample, got, tables):
    """precision_report of B-spline outputs (value table + Laplacian table) at w.pos[sample]."""
    import oracle
    beta, blap = tables
    ref64 = oracle.bspline_eval(beta, w.lattice, w.pos[sample], beta_lap=blap)
    refst = oracle.bspline_eval(rounded_table(beta, storage), w.lattice, w.pos[sample],
                                beta_lap=rounded_table(blap, storage))
    desc = "%d positions (every %d-th of the step) x %d orbitals" % (
        len(sample), int(sample[1] - sample[0]) if len(sample) > 1 else 1, got[0].shape[-1])
    return precision_report(storage, got, ref64, refst, desc)


def cpu_baseline(w, storage, sep, budget_s=12.0, tables=None):
    """The FP64 oracle's evaluation, as it stands, on the host cores: sized to about
    `budget_s` seconds of work on a prefix of the positions."""
    import oracle
    n_orb = w.coef.shape[0]
    beta, blap = tables if tables is not None else \
        oracle.smoothing_tables(w.lattice, w.miller, w.coef, w.cell.grid, laplacian=sep)
    n = 256
    t0 = time.perf_counter()
    oracle.bspline_eval(beta, w.lattice, w.pos[:n], beta_lap=blap)
    dt = time.perf_counter() - t0
    n2 = int(min(w.pos.shape[0], max(n, n * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.bspline_eval(beta, w.lattice, w.pos[:n2], beta_lap=blap)
    dt2 = time.perf_counter() - t0
    cores = oracle.set_threads(0)
    # the same oracle on one thread, on a proportionally smaller sample
    n1 = max(64, n2 // max(1, cores))
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.bspline_eval(beta, w.lattice, w.pos[:n1], beta_lap=blap)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": n2 * n_orb / dt2, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d positions x %d orbitals, FP64 oracle evaluation (tables prebuilt)"
                      % (n2, w.pos.shape[0], n_orb), "seconds": dt2,
            "single_thread": {"value": n1 * n_orb / dt1, "sample": "%d positions" % n1, "seconds": dt1}}


def method_label(method="smooth", sep=True):
    return "%s B-spline%s" % ({"smooth": "smoothing", "interp": "interpolating"}[method],
                              " + separate Laplacian table" if sep else " (Laplacian from the Hessian)")


def workload_config(w, ws=1, method="smooth", sep=True):
    """The benchmark's workload, the same dict for both arms (no launch details)."""
    return {"workload": w.cell.name, "method": method_label(method, sep),
            "n_orb": int(w.coef.shape[0]), "grid": list(w.cell.grid), "walkers": w.cell.n_walkers,
            "electrons": w.cell.n_elec, "positions": int(w.pos.shape[0]),
            "l2": "table and outputs larger than L2 (no flush needed)",
            "parallelism": "replicas" if ws > 1 else "single"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = inputs.make_workload(args.workload)
    import oracle
    n_orb = w.coef.shape[0]
    beta, blap = oracle.smoothing_tables(w.lattice, w.miller, w.coef, w.cell.grid, laplacian=True)
    n = args.ref_sample
    for i in range(args.warmup):
        oracle.bspline_eval(beta, w.lattice, w.pos[:min(n, 64)], beta_lap=blap)
    times = []
    for i in range(args.steps):
        s0 = (i * n) % max(1, w.pos.shape[0] - n)
        t0 = time.perf_counter()
        oracle.bspline_eval(beta, w.lattice, w.pos[s0:s0 + n], beta_lap=blap)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = n * n_orb * args.steps / t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d positions x %d orbitals per step (a bounded sample of the "
                                       "workload's %d positions), FP64 tables prebuilt"
                                       % (n, n_orb, w.pos.shape[0])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def probe_cache(dev, level):
    """The SMs' L1 (level 1) or L2 (level 2) data-path rate for 16-byte loads, measured on this
    GPU by the library's probe (qmcspl_probe_cache): GB/s over all SMs, bytes per SM clock, and
    the SM clock it ran at."""
    import ctypes
    import torch
    from paper_1309_6250_gb300 import _lib
    lib = _lib.load()
    g, b, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        _lib.check(lib.qmcspl_probe_cache(int(level), ctypes.byref(g), ctypes.byref(b), ctypes.byref(m),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    how = {1: "16-byte ld.global.nc over a 64 KB buffer resident in every L1",
           2: "16-byte ld.global.cg (L2 only) over a 32 MB buffer resident in L2"}[level]
    return {"gbs": g.value, "bytes_per_clk_per_sm": b.value, "sm_mhz": m.value,
            "how": "qmcspl_probe_cache(%d): 2 x 1024 threads per SM, %s, 8 loads in flight per thread, "
                   "best of 5 CUDA-event-timed launches" % (level, how)}


def probe_fma(dev, packed=1):
    """The SMs' FP32 multiply-add rate, measured on this GPU by the library's probe
    (qmcspl_probe_fma): TFLOP/s over all SMs (2 FLOPs per multiply-add), FLOPs per SM clock, the
    SM clock it ran at."""
    import ctypes
    import torch
    from paper_1309_6250_gb300 import _lib
    lib = _lib.load()
    t, f, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        _lib.check(lib.qmcspl_probe_fma(int(packed), ctypes.byref(t), ctypes.byref(f), ctypes.byref(m),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return {"tflops": t.value, "flops_per_clk_per_sm": f.value, "sm_mhz": m.value,
            "how": "qmcspl_probe_fma(%d): 2 x 1024 threads per SM, 8 independent chains of %s per thread, "
                   "best of 5 CUDA-event-timed launches" % (packed, "fma.rn.f32x2" if packed else "fma.rn.f32")}


# FP32 multiply-adds per orbital-evaluation as the kernels form them (z sums of the 4 rows of each
# stencil column or pp unit, the column's weighted accumulations, then the 3 x 3 chain rule of
# the gradient): interpolating/smoothing B-spline with the Laplacian table 16 x (2 x 4 + 4 + 5) + 9;
# with the Laplacian from the Hessian 16 x (3 x 4 + 7) + 9, and the same for the pp-spline's 16
# units (2 x 2 corner columns x 4 labels); five tables (Lagrange, separate gradient tables)
# 80 x (4 + 1) + 9.
FMA_PER_EVAL = {"interp_lap": 281, "smooth_lap": 281, "smooth": 313, "pp": 313, "lagrange": 409,
                "smooth_sep_grad": 409}


def alu_roofline(fma_per_eval, evals, launch_s, fma):
    """Multiply-add FLOPs of one launch against the probe's packed FP32 rate."""
    achieved = 2.0 * fma_per_eval * evals / launch_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": fma["tflops"], "unit": "TFLOP/s",
            "frac": achieved / fma["tflops"], "fma_per_eval": fma_per_eval,
            "peak_kind": "measured in this run (qmcspl_probe_fma, packed fma.rn.f32x2)"}


def l1_roofline(gather_bytes, launch_s, l1):
    """Every gathered stencil byte is requested from the SM's L1 data path (hits there, misses
    continue to L2).  Peak: the probe's measured L1 rate."""
    achieved = gather_bytes / launch_s / 1e9
    return {"bound": "l1", "achieved": achieved, "peak": l1["gbs"], "unit": "GB/s",
            "frac": achieved / l1["gbs"], "peak_kind": "measured in this run (qmcspl_probe_cache level 1)"}


def cache_rooflines(gather_bytes, l2_bytes, dram_bytes, launch_s, l1, l2, hbm, hbm_kind):
    """The kernel's bytes at each level of the memory hierarchy against that level's measured
    rate: gathered (algorithmic) bytes through L1, the L2 bytes ncu counted (L1 misses), the DRAM
    bytes ncu counted.  Levels without a byte count are left out.  The binding level is the one
    with the highest fraction."""
    lv = {"l1": l1_roofline(gather_bytes, launch_s, l1)}
    if l2_bytes:
        a = l2_bytes / launch_s / 1e9
        lv["l2"] = {"bound": "l2", "achieved": a, "peak": l2["gbs"], "unit": "GB/s", "frac": a / l2["gbs"],
                    "bytes_per_launch": l2_bytes, "peak_kind": "measured in this run (qmcspl_probe_cache level 2)"}
    if dram_bytes:
        a = dram_bytes / launch_s / 1e9
        lv["hbm"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                     "bytes_per_launch": dram_bytes, "peak_kind": hbm_kind}
    top = max(lv.values(), key=lambda r: r["frac"])
    return dict(top), lv


def _time_handle(spl, pos, torch, stream, steps, graph=True):
    """Mean ms per qmcspl_eval_vgl call (records, sort and evaluation), as CUDA-graph replays
    like the main step (small cells are otherwise dominated by the launch gaps of the call's
    four kernels), or eager calls."""
    out = spl.alloc_outputs(pos.shape[0])
    step = lambda: spl.eval_vgl(pos, out=out)
    if graph:
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            spl.eval_vgl(pos, out=out, stream=cap)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=cap):
                spl.eval_vgl(pos, out=out, stream=cap)
        torch.cuda.synchronize()
        step = g.replay
    ms = time_steps(step, steps, 3, torch, stream)
    spl.sync()
    return sum(ms) / len(ms)


def bench_methods(args, dev, stream):
    """The four bases of the paper on the Si-like 8-atom cell (16 orbitals, 48^3 grid,
    1024 walkers x 32 electrons, same planewaves), FP32 tables: evaluations per second."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    w = inputs.make_workload("c2")
    pos = torch.from_numpy(w.pos).to(dev)
    evals = w.pos.shape[0] * w.coef.shape[0]
    out = {}
    for name, method, sep in (("smooth_lap", "smooth", True), ("smooth", "smooth", False),
                              ("interp_lap", "interp", True), ("interp", "interp", False),
                              ("lagrange", "lagrange", True), ("pp", "pp", False)):
        spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method=method, storage="f32",
                             separate_lap=sep, device=dev)
        t = _time_handle(spl, pos, torch, stream, max(10, args.steps // 4))
        te = _time_handle(spl, pos, torch, stream, max(10, args.steps // 4), graph=False)
        out[name] = {"value": evals / (t * 1e-3), "ms_per_step": t, "eager_ms_per_step": te,
                     "table_bytes": spl.info()["table_bytes"]}
        spl.close()
    return {"workload": "c2 Si-like 8-atom, 16 orbitals, 48^3, 32768 positions, f32 tables, CUDA-graph replays",
            "unit": UNIT, "results": out}


METHOD_LEGS_C3 = (("smooth", dict(method="smooth", separate_lap=False)),
                  ("interp_lap", dict(method="interp", separate_lap=True)),
                  ("lagrange", dict(method="lagrange", separate_lap=True)),
                  ("smooth_sep_grad", dict(method="smooth", separate_lap=True, separate_grad=True)),
                  ("pp", dict(method="pp", separate_lap=False)))


def method_oracle(name, lat, mil, coef, dims, pos, storage):
    """Oracle outputs of one basis of METHOD_LEGS_C3 at pos: (on the unrounded FP64 tables,
    on the tables rounded as `storage` stores them)."""
    import oracle
    if name == "smooth":
        t = oracle.smoothing_tables(lat, mil, coef, dims)
        ev = lambda tt: oracle.bspline_eval(tt[0], lat, pos)
    elif name == "interp_lap":
        t = oracle.interpolating_tables(lat, mil, coef, dims, laplacian=True)
        ev = lambda tt: oracle.bspline_eval(tt[0], lat, pos, beta_lap=tt[1])
    elif name == "lagrange":
        t = (oracle.lagrange_tables(lat, mil, coef, dims),)
        ev = lambda tt: oracle.lagrange_eval(tt[0], lat, pos)
    elif name == "smooth_sep_grad":
        t = (oracle.derivative_tables("smooth", lat, mil, coef, dims),)
        ev = lambda tt: oracle.bspline_eval_separate(tt[0], lat, pos)
    else:
        t = (oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims)),)
        ev = lambda tt: oracle.pp_eval(tt[0], lat, pos)
    return ev(t), ev(tuple(rounded_table(x, storage) for x in t))


def bench_methods_c3(args, dev, stream, l1, fma=None):
    """The paper's bases at the 128-orbital scale: MgO-like 64-atom cell, 96^3, 2048 walkers x
    256 electrons, FP32 tables, cell order.  Per method the evaluation kernel's own time
    (library CUDA events), its gathered bytes against the measured L1 data-path peak and its
    multiply-adds against the measured FP32 multiply-add rate:
    smoothing without the Laplacian table (Hessian Laplacian, 1 table), interpolating with it
    (2 tables), Lagrange and B-splines with separate gradient tables (5 tables each), pp (8
    points x 8 entries = 64 values, as one table).  Per method also the error of the first 16
    orbitals at every 512th position against the FP64 oracle (unrounded and FP32-rounded
    tables) and the kinetic-energy change it causes."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    w = inputs.make_workload("c3")
    pos = torch.from_numpy(w.pos).to(dev)
    n_pos, n_orb = w.pos.shape[0], w.coef.shape[0]
    evals = n_pos * n_orb
    sample = np.arange(0, n_pos, 512)
    n_chk = 16
    sidx = torch.from_numpy(sample).to(dev)
    out, samples = {}, {}
    for name, kw in METHOD_LEGS_C3:
        spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, storage="f32", device=dev, **kw)
        o = spl.alloc_outputs(n_pos)
        step = lambda: spl.eval_vgl(pos, out=o)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        spl.profile(True)
        ms = time_steps(step, max(5, args.steps // 40), 0, torch, stream)
        prof = spl.profile_read()
        spl.profile(False)
        spl.sync()
        samples[name] = tuple(t[sidx][..., :n_chk].double().cpu().numpy() for t in o)
        k_s = prof["eval_ms"] * 1e-3 / max(1, prof["launches"])
        n_tab = spl.info()["n_tables"]
        bpe = algorithmic_bytes_per_eval("f32", n_tab, n_orb)
        out[name] = {"value": evals / (sum(ms) / len(ms) * 1e-3), "ms_per_step": sum(ms) / len(ms),
                     "eval_kernel_ms": k_s * 1e3, "tables": n_tab, "bytes_per_eval": bpe,
                     "table_bytes": spl.info()["table_bytes"],
                     "roofline_l1": l1_roofline(bpe * evals, k_s, l1)}
        if fma is not None:
            out[name]["roofline_alu"] = alu_roofline(FMA_PER_EVAL[name], evals, k_s, fma)
        # DRAM bytes of the launch from the stored ncu capture of this source, against HBM
        tr = load_traffic("methods_c3/" + name, METHOD_SOURCES)
        if tr and tr["dram"]:
            hbm, hbm_kind = load_peaks()
            a = tr["dram"] / k_s / 1e9
            out[name]["roofline_hbm"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                                         "frac": a / hbm, "bytes_per_launch": tr["dram"], "peak_kind": hbm_kind,
                                         "traffic_source": "stored: ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                                           "of this kernel source, profiles/traffic.json"}
        del o
        spl.close()
        torch.cuda.empty_cache()
    desc = "%d positions (every 512-th) x the first %d orbitals" % (len(sample), n_chk)
    for name, _ in METHOD_LEGS_C3:
        r64, rst = method_oracle(name, w.lattice, w.miller, w.coef[:n_chk], w.cell.grid, w.pos[sample], "f32")
        out[name]["precision"] = precision_report("f32", samples[name], r64, rst, desc)
    return {"workload": "c3 MgO-like 64-atom, 128 orbitals, 96^3, 2048 x 256 positions, f32 tables, cell order",
            "unit": UNIT, "results": out}


def bench_backward(args, dev, stream):
    """Adjoint pass on the Si-like 64-atom cell (128 orbitals, 72^3, FP32 tables with the
    Laplacian table, 4096 positions, N(0,1) upstream weights): coefficient scatter and
    position gradient together, per second of positions x orbitals."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    w = inputs.make_workload("c5")
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev)
    n, o = w.pos.shape[0], w.coef.shape[0]
    gv, gg, gl = (torch.from_numpy(x).to(device=dev, dtype=torch.float32)
                  for x in inputs.upstream_weights(n, o, 3005))
    pos = torch.from_numpy(w.pos).to(dev)
    dc = torch.zeros(spl.coef_shape(), dtype=torch.float32, device=dev)
    dcl = torch.zeros_like(dc)
    step = lambda: spl.backward(pos, gv, gg, gl, dcoef=dc, dcoef_lap=dcl)
    ms = time_steps(step, max(10, args.steps // 4), 3, torch, stream)
    spl.sync()
    t = sum(ms) / len(ms)
    spl.close()
    return {"workload": "c5 Si-like 64-atom, 128 orbitals, 72^3, 4096 positions, f32", "unit": UNIT,
            "value": n * o / (t * 1e-3), "ms_per_step": t}


def bench_backward_c3(args, dev, stream, l1=None):
    """Both adjoints (coefficient scatter and position gradient) at the many-walker scale: the
    MgO-like 64-atom cell, 128 orbitals on 96^3, FP32 smoothing + Laplacian tables, 2048 walkers x
    256 electrons, upstream weights N(0,1) on value, gradient and Laplacian (seeded device
    generator).  Cell order (the automatic choice here) against input order; dL/dr of every
    512th position against the oracle adjoint."""
    import torch
    import oracle
    from paper_1309_6250_gb300.api import OrbitalSplines
    w = inputs.make_workload("c3", n_pos=args.n_pos)
    n, o = w.pos.shape[0], w.coef.shape[0]
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3006)
    gv = torch.randn((n, o), generator=gen, device=dev, dtype=torch.float32)
    gg = torch.randn((n, 3, o), generator=gen, device=dev, dtype=torch.float32)
    gl = torch.randn((n, o), generator=gen, device=dev, dtype=torch.float32)
    pos = torch.from_numpy(w.pos).to(dev)
    dc = torch.zeros(spl.coef_shape(), dtype=torch.float32, device=dev)
    dcl = torch.zeros_like(dc)
    res = {"workload": "c3 MgO-like 64-atom, 128 orbitals, 96^3, 2048 x 256 positions, f32 smoothing + Laplacian "
                       "tables, upstream N(0,1) (seed 3006)", "unit": UNIT, "orders": {}}
    # table rows read (64 per table) + their 64 dbeta rows updated (atomic adds) per orbital-evaluation,
    # the five upstream values and the position
    bpe = 2 * 64 * 4 + 2 * 64 * 4 + 5 * 4 + 48.0 / o
    for order in ("cell", "input"):
        spl.set_order(order)
        step = lambda: spl.backward(pos, gv, gg, gl, dcoef=dc, dcoef_lap=dcl)
        ms = time_steps(step, max(5, args.steps // 40), 2, torch, stream)
        spl.sync()
        t = sum(ms) / len(ms)
        r = {"value": n * o / (t * 1e-3), "ms_per_step": t, "bytes_per_eval": bpe}
        if l1 is not None:
            r["roofline_l1"] = l1_roofline(bpe * n * o, t * 1e-3, l1)
        res["orders"][order] = r
    # the two passes alone, in cell order: the coefficient adjoint (dL/dbeta only, gathered per
    # bin of cells) and the position adjoint (dL/dr only).  The first is held to its compulsory
    # DRAM bytes (both dbeta tables read and written once, the upstream weights and positions
    # read once) against the HBM copy rate, the second to its gathered bytes (64 rows of both
    # tables, the upstream weights and the position per orbital-evaluation) against the L1 rate.
    hbm, hbm_kind = load_peaks()
    coef_bytes = 2 * 2 * dc.numel() * 4 + n * o * 5 * 4 + n * 24
    pos_bpe = 2 * 64 * 4 + 5 * 4 + 48.0 / o
    spl.set_order("cell")
    for name, kw in (("cell_coef_only", dict(dcoef=dc, dcoef_lap=dcl, want_dpos=False)),
                     ("cell_pos_only", dict(want_dpos=True))):
        step = lambda: spl.backward(pos, gv, gg, gl, **kw)
        ms = time_steps(step, max(5, args.steps // 40), 2, torch, stream)
        spl.sync()
        t = sum(ms) / len(ms)
        r = {"ms_per_step": t}
        if name == "cell_coef_only":
            a = coef_bytes / (t * 1e-3) / 1e9
            r["roofline_hbm"] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                                 "compulsory_bytes": coef_bytes, "peak_kind": hbm_kind}
        elif l1 is not None:
            r["bytes_per_eval"] = pos_bpe
            r["roofline_l1"] = l1_roofline(pos_bpe * n * o, t * 1e-3, l1)
        res["orders"][name] = r
    res["value"] = res["orders"]["cell"]["value"]
    res["ms_per_step"] = res["orders"]["cell"]["ms_per_step"]
    # dL/dr of sampled positions against the oracle adjoint (FP64, on the oracle's FP32-rounded tables)
    spl.set_order("cell")
    dpos = spl.backward(pos, gv, gg, gl)
    spl.sync()
    sample = np.arange(0, n, 512)
    sidx = torch.from_numpy(sample).to(dev)
    up = [x[sidx].double().cpu().numpy() for x in (gv, gg, gl)]
    beta, blap = oracle.smoothing_tables(w.lattice, w.miller, w.coef, w.cell.grid, laplacian=True)
    _, _, rdpos = oracle.bspline_adjoint(rounded_table(beta, "f32"), w.lattice, w.pos[sample], *up,
                                         beta_lap=rounded_table(blap, "f32"))
    err = float(oracle.relative_error(dpos[sidx].cpu().numpy(), rdpos))
    res["dpos_parity"] = {"max_rel_err": err, "tolerance": TOLERANCE["f32"], "ok": err <= TOLERANCE["f32"],
                          "sample": "%d positions (every 512-th)" % len(sample),
                          "reference": "FP64 oracle adjoint on the oracle's tables rounded to FP32"}
    spl.close()
    return res


def bench_bloch(args, dev, stream):
    """Complex Bloch orbitals at k != 0 (Sec. II) on the MgO-like 64-atom cell: 64 bands at
    the zone corner R = (1/2, 1/2, 1/2) on 96^3 (the same table bytes as the 128 real
    orbitals), 2048 walkers x 256 electrons, FP32 smoothing + Laplacian tables, cell order.
    value = complex orbital evaluations (value, gradient, Laplacian) per second.  The outputs
    then feed the complex Slater consumer (4096 walkers x (64 + 64) electrons)."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    kp = inputs.KPOINTS["R"]
    w = inputs.make_bloch_workload("c3", kp)
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev, kpoint=kp)
    pos = torch.from_numpy(w.pos).to(dev)
    out = spl.alloc_outputs(pos.shape[0])
    step = lambda: spl.eval_vgl(pos, out=out)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    spl.profile(True)
    ms = time_steps(step, max(10, args.steps // 4), 0, torch, stream)
    prof = spl.profile_read()
    spl.profile(False)
    spl.sync()
    t = sum(ms) / len(ms) * 1e-3
    k_s = prof["eval_ms"] * 1e-3 / max(1, prof["launches"])
    n_pos, n_band = w.pos.shape[0], w.coef.shape[0]
    n_fun = 2 * n_band
    bpe = algorithmic_bytes_per_eval("f32", spl.info()["n_tables"], n_fun)
    res = {"workload": "MgO-like 64-atom cell, 64 complex bands at k = R (1/2,1/2,1/2), 96^3, "
                       "2048 x 256 positions, f32 smoothing + Laplacian tables",
           "unit": "complex orbital evaluations/s", "value": n_pos * n_band / t, "ms_per_step": t * 1e3,
           "eval_kernel_ms": k_s * 1e3, "order_kernels_ms": prof["order_ms"] / max(1, prof["launches"]),
           "real_function_evals_per_s": n_pos * n_fun / t,
           "algorithmic_gbs": bpe * n_pos * n_fun / k_s / 1e9}
    # the same outputs as complex Slater matrices: 4096 walkers x (64 + 64) electrons, 64 bands
    from paper_1309_6250_gb300.api import slater_kinetic
    v, g, l = out
    ne = 2 * n_band
    W = n_pos // ne
    cres = {}
    for arith in ("df64", "f64"):
        cstep = lambda: slater_kinetic(v, g, l, W, ne, n_band, arith=arith)
        cms = time_steps(cstep, max(5, args.steps // 40), 2, torch, stream)
        ct = sum(cms) / len(cms) * 1e-3
        cres[arith] = {"value": W / ct, "ms_per_step": ct * 1e3, "gflops_equiv": W * 2 * 8.0 * n_band ** 3 / ct / 1e9}
    res["consumer"] = {"workload": f"{W} walkers x ({n_band} + {n_band}) electrons, {n_band} complex bands, "
                                   "complex Gauss-Jordan", "unit": "walkers/s", "value": cres["df64"]["value"],
                       "ms_per_step": cres["df64"]["ms_per_step"], "arith": cres}
    # error of the first 8 bands at every 512th position against the FP64 oracle (Bloch tables of
    # u, then the phase and the product rule), unrounded and FP32-rounded tables
    import oracle
    sample = np.arange(0, n_pos, 512)
    sidx = torch.from_numpy(sample).to(dev)
    got = tuple(t[sidx][..., :8].cpu().numpy().astype(np.complex128) for t in out)
    beta, blap = oracle.bloch_tables("smooth", w.lattice, w.miller, w.coef[:8], kp, w.cell.grid, laplacian=True)
    r64 = oracle.bloch_eval("smooth", beta, w.lattice, kp, w.pos[sample], tables_lap=blap)
    rst = oracle.bloch_eval("smooth", rounded_table(beta, "f32"), w.lattice, kp, w.pos[sample],
                            tables_lap=rounded_table(blap, "f32"))
    res["precision"] = precision_report("f32", got, r64, rst,
                                        "%d positions (every 512-th) x the first 8 bands" % len(sample))
    spl.close()
    return res


def bench_consumer(args, dev, stream):
    """The Slater-determinant consumer (qmcspl_slater_kinetic) on the MgO-like 64-atom
    walker batch: 2048 walkers x (128 up + 128 down electrons), 128 x 128 Gauss-Jordan
    inversions (double-float and FP64) from the FP32 spline outputs, log-determinant, local
    kinetic energy and drift.  value = walkers per second (double-float)."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines, slater_kinetic
    w = inputs.make_workload("c3")
    spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="smooth", storage="f32",
                         separate_lap=True, device=dev)
    v, g, l = spl.eval_vgl(torch.from_numpy(w.pos).to(dev))
    spl.sync()
    W, ne = w.cell.n_walkers, w.cell.n_elec
    n = ne // 2
    flops = W * 2 * (2.0 * n ** 3)          # Gauss-Jordan: n^3 multiply-adds per block
    res = {}
    for arith in ("df64", "f64"):
        step = lambda: slater_kinetic(v, g, l, W, ne, ne // 2, arith=arith)
        ms = time_steps(step, max(5, args.steps // 40), 2, torch, stream)
        t = sum(ms) / len(ms) * 1e-3
        res[arith] = {"value": W / t, "ms_per_step": t * 1e3, "gflops_equiv": flops / t / 1e9}
    spl.close()
    return {"workload": "MgO-like 64-atom batch: 2048 walkers x (128 + 128) electrons, 128 orbitals, "
                        "FP32 spline outputs", "unit": "walkers/s", "value": res["df64"]["value"],
            "ms_per_step": res["df64"]["ms_per_step"], "arith": res}


def bench_general(args, dev, stream):
    """Interpolating B-splines of degree 1, 3, 5, 7 on the uniform grid and of degree 3, 5, 7 on a
    graded (non-uniform) grid of the same size, on the Si-like 8-atom cell (16 orbitals, 48^3, 1024 walkers x 32 electrons, FP32 tables
    with the Laplacian table): orbital evaluations per second.  Degree 3 on the uniform grid
    is the tuned cubic kernel, the others the general kernel ((n+1)^3-point stencils)."""
    import torch
    from paper_1309_6250_gb300.api import OrbitalSplines
    w = inputs.make_workload("c2")
    pos = torch.from_numpy(w.pos).to(dev)
    evals = w.pos.shape[0] * w.coef.shape[0]
    out = {}
    graded = tuple(inputs.graded_knots(d, 0.5, 0.17 * a) for a, d in enumerate(w.cell.grid))
    for name, kw in (("degree1", dict(degree=1)), ("degree3", dict(degree=3)), ("degree5", dict(degree=5)),
                     ("degree7", dict(degree=7)), ("graded_cubic", dict(knots=graded)),
                     ("graded_degree5", dict(degree=5, knots=graded)), ("graded_degree7", dict(degree=7, knots=graded))):
        spl = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method="interp", storage="f32",
                             separate_lap=True, device=dev, **kw)
        t = _time_handle(spl, pos, torch, stream, max(10, args.steps // 4))
        out[name] = {"value": evals / (t * 1e-3), "ms_per_step": t}
        spl.close()
    return {"workload": "c2 Si-like 8-atom, 16 orbitals, 48^3, 32768 positions, f32 interpolating + Lap, "
                        "CUDA-graph replays", "unit": UNIT, "results": out}


def bench_batched(args, dev, stream, l1=None):
    """The uneven three-cell workload (Al-like 32-atom: 48 orbitals, 64^3, 512 x 96 e;
    Si-like 64-atom: 128 orbitals, 80^3, 1024 x 256 e; MgO-like 16-atom: 32 orbitals,
    64^3, 2048 x 64 e; FP32 smoothing + Laplacian tables) through one qmcspl_eval_batched_ex
    call per step, replayed from a CUDA graph.  Each cell has the autotuner's lanes, block shape
    and order; the launch plan of the call (one launch per cell, or all cells in the one
    persistent batched launch of 512 or 640 threads per block) is the autotuner's too, and every
    plan's time is reported.  Sampled outputs of each cell are checked against the oracle."""
    import torch
    import oracle
    from paper_1309_6250_gb300 import autotune
    import tempfile
    cache = os.path.join(tempfile.gettempdir(), "qmcspl_autotune.json")   # tuned shapes, reused within a machine
    cells, shapes, evals, gathered, works = [], {}, 0, 0.0, []
    for key in ("c4-al32", "c4-si64", "c4-mgo16"):
        w = inputs.make_workload(key)
        spl, t = autotune.tuned_splines(w.lattice, w.cell.grid, w.miller, w.coef, w.pos, storage="f32",
                                        separate_lap=True, device=dev, cache_path=cache, repeats=5)
        shapes[w.cell.name] = {"lanes": t["lanes"], "threads": t.get("threads", 0), "order": t["order"]}
        p = torch.from_numpy(w.pos).to(dev)
        cells.append((spl, p, spl.alloc_outputs(p.shape[0])))
        n = w.pos.shape[0] * w.coef.shape[0]
        evals += n
        gathered += n * algorithmic_bytes_per_eval("f32", 2, w.coef.shape[0])
        works.append(w)
    spls = [c[0] for c in cells]
    pos = [c[1] for c in cells]
    outs = [c[2] for c in cells]
    plan = autotune.tune_batch(spls, pos, outs, storage="f32", key="c4-al32+si64+mgo16", cache_path=cache,
                               repeats=max(10, args.steps // 2))
    chosen = {"launch": plan["launch"], "threads": plan["threads"]}
    # the chosen plan, measured again as graph replays of the whole call
    t = autotune.time_batch_graph(spls, pos, outs, chosen, repeats=max(10, args.steps // 2))
    res = {"workload": "c4 uneven batch (Al-32 48 orb 64^3, Si-64 128 orb 80^3, MgO-16 32 orb 64^3)",
           "value": evals / (t * 1e-3), "unit": UNIT, "ms_per_step": t, "evals_per_step": evals,
           "storage": "f32", "cuda_graph": True, "shapes": shapes, "launch_plan": chosen,
           "plans_tried": plan["trials"]}
    if l1 is not None:
        res["roofline_l1"] = l1_roofline(gathered, t * 1e-3, l1)
        res["roofline_l1"]["note"] = "gathered bytes of all cells over the whole call (sorting kernels included)"
    # sampled outputs of every cell against the oracle (first 8 orbitals)
    prec = {}
    for w, (spl, p, o) in zip(works, cells):
        sample = np.arange(0, w.pos.shape[0], max(1, w.pos.shape[0] // 512))
        sidx = torch.from_numpy(sample).to(dev)
        got = tuple(x[sidx][..., :8].double().cpu().numpy() for x in o)
        beta, blap = oracle.smoothing_tables(w.lattice, w.miller, w.coef[:8], w.cell.grid, laplacian=True)
        r64 = oracle.bspline_eval(beta, w.lattice, w.pos[sample], beta_lap=blap)
        rst = oracle.bspline_eval(rounded_table(beta, "f32"), w.lattice, w.pos[sample],
                                  beta_lap=rounded_table(blap, "f32"))
        prec[w.cell.name] = precision_report("f32", got, r64, rst, "%d positions x the first 8 orbitals" % len(sample))
    res["precision"] = prec
    for s_ in spls:
        s_.sync()
        s_.close()
    return res


def run_ours(args):
    import torch
    rank, ws, dist = dist_setup()
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1309_6250_gb300.api import OrbitalSplines

    from paper_1309_6250_gb300 import replicas
    w = inputs.make_workload(args.workload, n_pos=args.n_pos)
    if rank > 0:   # weak scaling: every rank its own walkers
        w.pos[:] = replicas.rank_positions(w.lattice, w.pos.shape[0], w.cell.pos_seed, rank)
    n_pos, n_orb = w.pos.shape[0], w.coef.shape[0]
    stream = torch.cuda.current_stream()

    def build(storage, order):
        t0 = time.perf_counter()
        s = OrbitalSplines(w.lattice, w.cell.grid, w.miller, w.coef, method=args.method,
                           storage=storage, separate_lap=bool(args.separate_lap), device=dev)
        s.set_order(order)
        return s, time.perf_counter() - t0

    spl, setup_s = build(args.storage, args.order)
    info = spl.info()
    pos_d = torch.from_numpy(w.pos).to(dev)
    outs = spl.alloc_outputs(n_pos)
    eager = lambda: spl.eval_vgl(pos_d, out=outs)
    step = eager
    graph = None
    if not args.no_graph:
        # one step (records + sort + evaluation) captured once and replayed: no launch gaps
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            spl.eval_vgl(pos_d, out=outs, stream=cap)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=cap):
                spl.eval_vgl(pos_d, out=outs, stream=cap)
        torch.cuda.synchronize()
        step = graph.replay    # replays on the current (timed) stream
    # the path qmcspl_eval_vgl takes (the rule of qmcspl_set_order)
    order_name = spl.resolved_order(n_pos)     # the library's rule (qmcspl_get_order)
    staged = order_name == "pencil"
    kernel_name = "bspline_vgl_staged_kernel" if staged else "bspline_vgl_kernel"
    # sorted: records/bins, scan, place + evaluation; input order: a records pass from 8192
    # positions on (Bloch handles: always, for the phases) + evaluation
    kernels_per_step = 4 if order_name != "input" else (2 if n_pos >= 8192 or info["bloch"] else 1)

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    sampler.wait_first()
    ms = time_steps(step, args.steps, 0, torch, stream)
    # a short timed region holds few samples: keep the same step running, untimed, for another
    # half second before the sampler stops
    t_tail = time.perf_counter()
    while time.perf_counter() - t_tail < 0.5:
        for _ in range(8):
            step()
        torch.cuda.synchronize()
    clocks = sampler.stop()
    if clocks is not None:
        clocks["window"] = "timed region + 0.5 s of the same step, untimed"
    spl.sync()
    # the evaluation kernel's own launch time, from the library's CUDA events (eager calls)
    spl.profile(True)
    time_steps(eager, max(10, args.steps // 4), 0, torch, stream)
    prof = spl.profile_read()
    spl.profile(False)
    spl.sync()
    total_ms = replicas.max_over_ranks(sum(ms), dist, dev)
    evals_per_step = n_pos * n_orb
    # outputs of every 64th position, for the parity check against the oracle below
    par_sample = np.arange(0, n_pos, 64)
    par_idx = torch.from_numpy(par_sample).to(dev)
    par_got = [t[par_idx].double().cpu().numpy() for t in outs]
    value = replicas.job_throughput(evals_per_step * args.steps, ws, total_ms * 1e-3)

    # end to end through the host-buffer entry point: pinned positions in, outputs back; the same
    # through qmcspl_eval_vgl_host_ex with bfloat16 outputs (converted on the device: half the
    # bytes over the link) is reported beside the full-precision e2e, which stays the headline
    pos_h = torch.from_numpy(w.pos).pin_memory()
    e2e_steps = max(10, args.steps // 2)   # host-side outliers (a call in ~15 runs ~15% slower) average out

    def time_e2e(fn):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fn()
        torch.cuda.synchronize()
        return replicas.job_throughput(evals_per_step * e2e_steps, ws,
                                       replicas.max_over_ranks(time.perf_counter() - t0, dist, dev))

    host_out = tuple(torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs)
    e2e_value = time_e2e(lambda: spl.eval_vgl_host(pos_h, out=host_out))
    d2h = sum(o.numel() * o.element_size() for o in host_out)
    # the link's own rate for the same bytes: device outputs copied into the pinned host tensors
    # (cudaMemcpyAsync on one stream), the bound of the end-to-end number; CUDA events around
    # each copy, the best of five after one warm-up
    def copy_out():
        for h_, o_ in zip(host_out, outs):
            h_.copy_(o_, non_blocking=True)
    copy_out()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        copy_out()
        e1.record(cur)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1)
        best = ms_c if best is None else min(best, ms_c)
    link_gbs = d2h / (best * 1e-3) / 1e9
    e2e_gbs = d2h * e2e_value / evals_per_step / 1e9 / ws
    e2e_16 = None
    if args.storage in ("f32", "bf16"):
        host16 = tuple(torch.empty(o.shape, dtype=torch.bfloat16).pin_memory() for o in outs)
        e2e_16 = {"value": time_e2e(lambda: spl.eval_vgl_host(pos_h, out=host16, out_dtype=torch.bfloat16)),
                  "unit": UNIT, "out_dtype": "bf16", "h2d_bytes_per_step": int(pos_h.numel() * 8),
                  "d2h_bytes_per_step": int(sum(o.numel() * o.element_size() for o in host16)),
                  "api": "qmcspl_eval_vgl_host_ex (QMCSPL_OUT_BF16)"}
        del host16

    # roofline of the dominant kernel, from its own CUDA-event launch times
    hbm, peak_kind = load_peaks()
    l1, l2 = probe_cache(dev, 1), probe_cache(dev, 2)
    fma = probe_fma(dev, 1)
    bpe = algorithmic_bytes_per_eval(args.storage, info["n_tables"], n_orb)
    launch_s = prof["eval_ms"] * 1e-3 / max(1, prof["launches"])
    achieved = bpe * evals_per_step / launch_s / 1e9
    key = "%s/%s/%s/%s" % (kernel_name.replace("_kernel", ""), w.cell.name, args.storage, order_name)
    if args.method != "smooth" or not args.separate_lap:
        key += "/%s%s" % (args.method, "+lap" if args.separate_lap else "")
    traffic = load_traffic(key)

    variants, var_got = {}, {}
    if not args.no_variants and rank == 0:
        for st, order in (("f32", "input"), ("f32", "pencil"), ("bf16", "auto"), ("bf16", "pencil"),
                          ("f64", "auto"), ("df64", "auto"), ("bf16", "input")):
            if st == args.storage and order == args.order:
                continue
            del outs
            spl.close()
            torch.cuda.empty_cache()
            spl, _ = build(st, order)
            outs = spl.alloc_outputs(n_pos)
            vstep = lambda: spl.eval_vgl(pos_d, out=outs)
            for _ in range(3):
                vstep()
            torch.cuda.synchronize()
            spl.profile(True)
            vms = time_steps(vstep, max(5, args.steps // 4), 0, torch, stream)
            vp = spl.profile_read()
            spl.profile(False)
            spl.sync()
            vt = sum(vms) / len(vms) * 1e-3
            vk = vp["eval_ms"] * 1e-3 / max(1, vp["launches"])
            vb = algorithmic_bytes_per_eval(st, spl.info()["n_tables"], n_orb)
            variants["%s_%s" % (st, order)] = {
                "value": evals_per_step / vt, "ms_per_step": vt * 1e3, "eval_kernel_ms": vk * 1e3,
                "order_kernels_ms": vp["order_ms"] / max(1, vp["launches"]),
                "algorithmic_gbs": vb * evals_per_step / vk / 1e9,
                "frac_of_hbm": vb * evals_per_step / vk / 1e9 / hbm}
            if order == "auto" and st not in var_got:
                var_got[st] = [t[par_idx].double().cpu().numpy() for t in outs]

    batched = methods = methods_c3 = backward = backward_c3 = bloch = consumer = general = None
    if not args.no_variants and rank == 0:
        del outs
        spl.close()
        torch.cuda.empty_cache()
        batched = bench_batched(args, dev, stream, l1)
        methods = bench_methods(args, dev, stream)
        methods_c3 = bench_methods_c3(args, dev, stream, l1, fma)
        backward = bench_backward(args, dev, stream)
        backward_c3 = bench_backward_c3(args, dev, stream, l1)
        bloch = bench_bloch(args, dev, stream)
        consumer = bench_consumer(args, dev, stream)
        general = bench_general(args, dev, stream)

    cpu = parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        build_tables = oracle.smoothing_tables if args.method == "smooth" else oracle.interpolating_tables
        tables = build_tables(w.lattice, w.miller, w.coef, w.cell.grid, laplacian=bool(args.separate_lap))
        cpu = cpu_baseline(w, args.storage, bool(args.separate_lap), tables=tables)
        parity = {args.storage: bspline_precision(w, args.storage, par_sample, par_got, tables)}
        for st, got in var_got.items():
            parity[st] = bspline_precision(w, st, par_sample, got, tables)
        parity["headline"] = args.storage

    # the launch against each level's measured rate (DRAM and L2 bytes: the stored ncu counts)
    dram_b = traffic["dram"] if traffic else None
    l2_b = traffic["l2"] if traffic else None
    inorder = variants.get("%s_input" % args.storage)
    roofline, levels = cache_rooflines(bpe * evals_per_step, l2_b, dram_b, launch_s, l1, l2, hbm, peak_kind)
    if args.storage in ("f32", "bf16"):   # the packed FP32 arithmetic of the float and bfloat16 kernels
        levels["alu"] = alu_roofline(FMA_PER_EVAL["smooth_lap" if args.separate_lap else "smooth"],
                                     evals_per_step, launch_s, fma)
        roofline = dict(max(levels.values(), key=lambda r: r["frac"]))
    roofline.update({
        "traffic": dram_b,
        "traffic_source": ("stored: ncu dram__bytes_read.sum + dram__bytes_write.sum (and lts__t_bytes.sum) "
                           "of this kernel source, profiles/traffic.json (source hash matches)") if traffic else None,
        "kernel": kernel_name, "bytes_per_eval": bpe, "kernel_ms": launch_s * 1e3,
        "order_kernels_ms": prof["order_ms"] / max(1, prof["launches"]),
        "levels": levels,
        "probes": {"l1": l1, "l2": l2, "fma": fma},
        "reuse_factor": (bpe * evals_per_step / dram_b) if dram_b else None,
        "reuse_factor_note": "algorithmic (gathered) bytes per DRAM byte: stencil rows shared by neighbouring "
                             "positions in cell order are read from HBM about once",
        "input_order_hbm": None if inorder is None else {
            "kernel_ms": inorder["eval_kernel_ms"], "achieved": inorder["algorithmic_gbs"], "peak": hbm,
            "unit": "GB/s", "frac": inorder["frac_of_hbm"], "peak_kind": peak_kind,
            "note": "the same kernel without cell order: every gathered row comes from HBM or L2"},
    })
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": workload_config(w, ws, args.method, bool(args.separate_lap)),
        "launch": {"storage": args.storage,
                   "accumulate": {"f64": "f64", "df64": "double-float (f32 pairs)"}.get(args.storage, "f32"),
                   "order": order_name, "table_bytes": info["table_bytes"], "lanes": info["lanes"],
                   "tiles": info["tiles"], "cuda_graph": graph is not None},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "parity": parity,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(pos_h.numel() * 8),
                "d2h_bytes_per_step": int(d2h), "api": "qmcspl_eval_vgl_host",
                "link": {"bound": "d2h", "achieved": e2e_gbs, "peak": link_gbs, "unit": "GB/s",
                         "frac": e2e_gbs / link_gbs,
                         "peak_kind": "measured in this run: the same output bytes copied device to pinned host "
                                      "(cudaMemcpyAsync, CUDA events, best of 5)"}},
        "e2e_bf16_outputs": e2e_16,
        "gpu_launches": args.steps * kernels_per_step,
        "clocks": clocks,
        "setup_s": setup_s,
        "variants": variants,
        "batched": batched,
        "methods_si8_48": methods,
        "methods_mgo64_96": methods_c3,
        "backward_si64_72": backward,
        "backward_mgo64_96": backward_c3,
        "bloch_mgo64_96": bloch,
        "slater_consumer_mgo64": consumer,
        "general_degree_si8_48": general,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--storage", default="f32", choices=["f64", "df64", "f32", "bf16"])
    ap.add_argument("--order", default="auto", choices=["auto", "input", "cell", "pencil"])
    ap.add_argument("--method", default="smooth", choices=["smooth", "interp"],
                    help="B-spline of the main leg (profiling other kernels)")
    ap.add_argument("--separate-lap", type=int, default=1, choices=[0, 1],
                    help="0: the Laplacian of the spline itself (one table)")
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager calls instead of CUDA-graph replays")
    ap.add_argument("--n-pos", type=int, default=None, help="use only the first N positions (profiling)")
    ap.add_argument("--only", default="all",
                    choices=["all", "bloch", "consumer", "general", "methods", "methods_c3", "batched",
                             "backward", "backward_c3", "probes"],
                    help="run one secondary leg alone and print its JSON (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only != "all":
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        leg = {"bloch": bench_bloch, "consumer": bench_consumer, "general": bench_general,
               "methods": bench_methods, "methods_c3": lambda a, d, s: bench_methods_c3(a, d, s, probe_cache(d, 1), probe_fma(d, 1)),
               "batched": lambda a, d, s: bench_batched(a, d, s, probe_cache(d, 1)), "backward": bench_backward,
               "backward_c3": lambda a, d, s: bench_backward_c3(a, d, s, probe_cache(d, 1)),
               "probes": lambda a, d, s: {"l1": probe_cache(d, 1), "l2": probe_cache(d, 2),
                                           "fma": probe_fma(d, 1), "fma_scalar": probe_fma(d, 0)}}[args.only]
        print(json.dumps({"leg": args.only, **leg(args, dev, torch.cuda.current_stream())}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
