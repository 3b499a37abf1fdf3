#!/usr/bin/env python
"""Benchmark: set elements sketched per second (ProbMinHash, all six variants, m = 1024).

Workload (default): 20,000 weighted sets, n log-uniform on [1, 1e5]
(floor(10^(5U))), weights Uniform(0,1], distinct uniform-looking 64-bit ids,
m = 1024, variants 1, 1a, 2, 3, 3a, 4 in one persistent launch.  One step =
one pmh_sketch_batch call over the whole batch (every item is sketched; 1/1a
and 3/3a are separate items).  The metric counts elements x variants per
second.  The headline path is FP32 candidates + FP64 recheck; the plain FP64
path is timed beside it and its ids are compared with the headline's.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pmh|reference]

Under torchrun (N > 1) every rank sketches its own batch (seed + rank):
weak scaling, no collective on the data path; rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (the plain FP64 C restatement of the
paper) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "set elements sketched/sec at m=1024 on 1 GB300 (FP32+recheck vs plain FP64), % roofline"
UNIT = "elements/s"
VARIANTS = ["1", "1a", "2", "3", "3a", "4"]

# Algorithmic integer/FP32 operations per unit of work, counted from the method's arithmetic.
# SplitMix64 word: three 64-bit xor-shifts (4 each), two 64-bit multiplies by a constant (3 each) and the
# 64-bit counter add (2) = 20.
OPS_ELEMENT = 55        # every element-variant: key = mix(id ^ mix(seed)) (22), weight check (2), scaled w
                        # from the exponent and mantissa (5), value word of point 1 (20), 23-bit uniform
                        # lower bound (3), the products bound * w and U * (1 - e^-lambda)/lambda and compare (3)
OPS_POINT = 70          # every generated point: value word (20), label word (20), label from the word (3;
                        # the lazy permutation's bookkeeping is not counted), logarithm (20), point value and
                        # stop compare (4), offer to the component (3)
OPS_SURVIVOR = -10      # per survivor: its point-1 value word was counted with its element (-20), and its
                        # scaled 1/w is one reciprocal (+10)
OPS_LISTED = 30         # every prefilter list entry a variant visits: the key and scaled w come with the entry
                        # (decode 4), value word of point 1 (20), 23-bit uniform (3), products and compare (3);
                        # the elements the prefilter pass hashed count OPS_ELEMENT once for all variants
LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes issue one instruction per clock
OPS_PAIR_COMPONENT = 3  # equal-component count: two 32-bit compares and one add per component pair
# 8-bit codes, per pair of 64-bit words (8 fields): xor (2), per 32-bit half three fold steps of
# shift + or (6) and and-not + popcount (2), two adds (2)
OPS_BBIT_WORD = 2 + 2 * (6 + 2) + 2
# DRAM bytes (read + write) of the prefilter pass, the four family sketch kernels and their redo
# kernels per element-variant, from the ncu capture summarised in
# profiles/sketch_kernel_fp32_c2_2000sets.md (888.2 MB for 99,379,884 element-variants); the
# traffic grows in proportion to the elements (one pass over the ids and weights of a listed set,
# one per family over the others).
TRAFFIC_BYTES_PER_ELEMENT_VARIANT = 8.94
# Pipe use of the same four family kernels in that capture (per kernel, min-max over the families):
# what binds them beside the op model above.
NCU_SKETCH = {"issue_active_pct": [60.6, 65.9], "alu_pipe_pct": [44.9, 51.9], "fma_pipe_pct": [18.3, 19.5],
              "dram_throughput_pct": [1.0, 2.3], "active_lanes_per_inst": [24.9, 27.9],
              "warp_inst_per_element_variant": 17.8, "prefilter_issue_active_pct": 59.5,
              "prefilter_alu_pipe_pct": 56.4, "source": "profiles/sketch_kernel_fp32_c2_2000sets.md, "
                                                        "profiles/list_kernel_c2_2000sets.md"}
TRAFFIC_BASIS = ("ncu dram bytes per element-variant on a 2,000-set c2-shaped batch (sketch kernel source of "
                 "commit d70b279 and later, first-round constant 4) x this step's work")


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pmh", "reference"], default="pmh")
    ap.add_argument("--num-sets", type=int, default=20000, help="sets in the batch (20,000 = the benchmark config)")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="wall budget of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--team-shape", type=str, default="-1",
                    help="pin the sketch kernels' team shape (0 warp, 1 cta8, 2 quad, 3 pair, 4 quad8, 5 quad8l), "
                         "one value for every family or four comma-separated values for ProbMinHash1..4; "
                         "-1 = autotuned")
    ap.add_argument("--prefilter", type=float, default=None,
                    help="prefilter list factor of the library (pmh_set_prefilter; 0 = off; default: the library's)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the per-kernel measurements beside the headline (huge set, all-pairs counts)")
    return ap.parse_args()


# ------------------------------------------------------------------ CPU oracle
def _oracle_task(args):
    """Worker: oracle signature of one (set, variant); returns (variant, set, elements, points)."""
    variant, s, ids, w, m = args
    import oracle
    _, _, st = oracle.sketch(variant, ids, w, m, seed=0)
    return variant, s, len(ids), st["points"]


def _oracle_pool(cores):
    """A spawn pool (never fork after CUDA is initialised), warmed up so that process start-up and
    the oracle's import are not timed."""
    import multiprocessing as mp

    import numpy as np
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores)
    pool.map(_oracle_task, [("1", 0, np.array([1], dtype=np.uint64), np.ones(1), 8)] * cores)
    return pool


def oracle_throughput(batch, seconds, cores, rng_seed=1, done=None):
    """Elements x variants per second of the oracle on a random sample of (set, variant) tasks,
    run on `cores` processes for about `seconds` of wall time.  `done` (optional list) receives
    (variant, set, points) of every finished task."""
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(rng_seed)
    tasks = [(v, s) for s in rng.permutation(batch.num_sets) for v in VARIANTS]
    pool = _oracle_pool(cores)
    done_elems, done_tasks = 0, 0
    t0 = time.perf_counter()
    it = pool.imap_unordered(_oracle_task, ((v, int(s), *batch.set(s), batch.m) for v, s in tasks), chunksize=1)
    try:
        for v, s, n, pts in it:
            done_elems += n
            done_tasks += 1
            if done is not None:
                done.append((v, s, pts))
            if time.perf_counter() - t0 > seconds:
                break
    finally:
        el = time.perf_counter() - t0
        pool.terminate()
    return done_elems / el, done_elems, done_tasks, el


def parallel_overhead(h, batch, done, dev):
    """GPU point evaluations against the oracle's sequential point count on the same (set, variant)
    tasks: the oracle generates each element's points in order and stops at the running q_max, the
    GPU runs threshold rounds over elements in parallel.  The GPU side runs one call per variant
    over the sets the oracle finished with that variant."""
    import numpy as np
    import torch
    from paper_1911_00675_gb300 import pmh
    from paper_1911_00675_gb300 import workloads as W
    by_v = {}
    for v, s, pts in done:
        by_v.setdefault(v, []).append((s, pts))
    gpu = {"points32": 0, "prefiltered": 0, "elements": 0, "deep": 0}
    oracle_pts = 0
    for v, lst in by_v.items():
        sets = np.array(sorted(s for s, _ in lst), dtype=np.int64)
        oracle_pts += sum(p for _, p in lst)
        sizes = batch.offsets[sets + 1] - batch.offsets[sets]
        idx = np.concatenate([np.arange(batch.offsets[s], batch.offsets[s + 1]) for s in sets])
        off = np.zeros(len(sets) + 1, dtype=np.int64)
        np.cumsum(sizes, out=off[1:])
        sub = W.Batch(batch.ids[idx], batch.weights[idx], off, batch.m)
        cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device=dev)
        h.sketch_batch(torch.from_numpy(sub.ids.view(np.int64)).to(dev), torch.from_numpy(sub.weights).to(dev),
                       torch.from_numpy(sub.offsets).to(dev), batch.m, [v], pmh.FP32_RECHECK, 0, counters=cnt)
        c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
        for k in gpu:
            gpu[k] += c[k]
    tasks = sum(len(x) for x in by_v.values())
    return {"tasks": tasks, "oracle_points": oracle_pts, "gpu_points32": gpu["points32"],
            "gpu_prefiltered": gpu["prefiltered"], "gpu_elements": gpu["elements"], "gpu_deep_elements": gpu["deep"],
            "factor_points": gpu["points32"] / max(1, oracle_pts),
            "factor_points_and_prefiltered": (gpu["points32"] + gpu["prefiltered"]) / max(1, oracle_pts),
            "note": "factor_points = FP32 point evaluations on the GPU / points the oracle generated on the same "
                    "(set, variant) tasks; the second factor also counts each element the GPU rejected by its "
                    "first point's lower bound (no logarithm) as one point"}


# ------------------------------------------------------------------ host placement
def bind_gpu_local_cpus(gpu_index):
    """Restricts this process to the CPU cores attached to the GPU (its PCI device's local_cpulist),
    so that pinned host buffers are first touched on the memory next to it.  Returns the core list
    string, or None when the topology is not readable."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(gpu_index)],
                             capture_output=True, text=True, timeout=30).stdout.strip()
        dom, rest = out.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest.lower()}/local_cpulist"
        with open(path) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        if cpus and cpus != set(range(os.cpu_count() or 0)):
            os.sched_setaffinity(0, cpus)
        return spec
    except Exception:
        return None


# ------------------------------------------------------------------ peaks
def measured_peaks():
    """HBM GB/s measured on this GPU type (MEASURED_PEAKS.json, a STREAM-style copy), else the value
    that file held on the GB300s when it was last present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "basis": "measured (MEASURED_PEAKS.json)"}
    except Exception:
        return {"hbm_gbs": 6780.0, "basis": "measured copy bandwidth of this pool's GB300s (MEASURED_PEAKS.json "
                                            "absent in this run: its earlier value)"}


def alu_peak(n_sms, sm_mhz):
    return n_sms * LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ secondary kernels
def te_sampler_comparison(h, ids, w, off, m, work_per_variant, steps=5):
    """ProbMinHash3/3a/4 on the headline batch with Exp(lambda;0,1) by inversion (the default) and by
    the paper's rejection sampler (Sec. Truncated Exponential Sampling): device time of the sketch
    kernels from the library's events, FP32 candidates + FP64 recheck."""
    import statistics

    from paper_1911_00675_gb300 import pmh
    vs = ["3", "3a", "4"]
    out = {"workload": "the headline batch, variants 3, 3a, 4 (FP32 + recheck)"}
    h.set_profiling(True)
    try:
        for name, mode in (("inversion", pmh.TE_INVERSION), ("rejection", pmh.TE_REJECTION)):
            h.set_te_sampler(mode)
            for _ in range(2):
                _, _, st = h.sketch_batch(ids, w, off, m, vs, pmh.FP32_RECHECK, 0)
            for _ in range(steps):
                _, _, st = h.sketch_batch(ids, w, off, m, vs, pmh.FP32_RECHECK, 0)
            k = h.kernel_ms_history(steps)[1]
            ms = statistics.mean(k)
            out[name] = {"sketch_kernel_ms": ms, "elements_per_s": 3 * work_per_variant / (ms * 1e-3),
                         "status_ok": bool((st == 0).all().item())}
    finally:
        h.set_te_sampler(pmh.TE_INVERSION)
        h.set_profiling(False)
    out["speedup_rejection_vs_inversion"] = out["inversion"]["sketch_kernel_ms"] / out["rejection"]["sketch_kernel_ms"]
    return out


def pminhash_comparison(h, dev, m=1024, steps=3):
    """Time per signature of Algorithm P-MinHash (n m hash values per set) against ProbMinHash1 and 3
    (FP32 + recheck) over set sizes n = 1 .. 1e5 at m = 1024, Uniform(0,1] weights: the comparison of
    the paper's experiments (fig:speed), on the GPU.  Device time by CUDA events around each call."""
    import numpy as np
    import torch
    from paper_1911_00675_gb300 import pmh
    from paper_1911_00675_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    rows = []
    for n in (1, 10, 100, 1000, 10000, 100000):
        S = int(min(100000, max(100, 2e10 / (n * m))))
        b = W.random_batch(9000 + n, [n] * S, m, "uniform")
        ids = torch.from_numpy(b.ids.view(np.int64)).to(dev)
        w = torch.from_numpy(b.weights).to(dev)
        off = torch.from_numpy(b.offsets).to(dev)
        zp = torch.empty((S, m), dtype=torch.int64, device=dev)
        stp = torch.empty(S, dtype=torch.int32, device=dev)
        z1 = torch.empty((1, S, m), dtype=torch.int64, device=dev)
        st1 = torch.empty((1, S), dtype=torch.int32, device=dev)
        ms_p = timed(lambda: h.pminhash_batch(ids, w, off, m, 0, out_ids=zp, status=stp))
        ms_1 = timed(lambda: h.sketch_batch(ids, w, off, m, ["1"], pmh.FP32_RECHECK, 0, out_ids=z1, status=st1))
        ms_3 = timed(lambda: h.sketch_batch(ids, w, off, m, ["3"], pmh.FP32_RECHECK, 0, out_ids=z1, status=st1))
        rows.append({"n": n, "sets": S, "pminhash_us_per_sig": ms_p * 1e3 / S, "pmh1_us_per_sig": ms_1 * 1e3 / S,
                     "pmh3_us_per_sig": ms_3 * 1e3 / S, "speedup_pmh1_vs_pminhash": ms_p / ms_1,
                     "speedup_pmh3_vs_pminhash": ms_p / ms_3,
                     "status_ok": bool((stp == 0).all().item() and (st1 == 0).all().item())})
        del ids, w, off, zp, z1
    return {"workload": f"sets of n elements (Uniform(0,1] weights), m={m}; per n about 2e10 / (n m) sets "
                        "(at least 100, at most 100,000)", "rows": rows}


def secondary(h, dev, n_sms, sm_mhz, peaks, steps=3):
    """Per-kernel measurements beside the headline: the precision config (FP32 + recheck against FP64
    at m = 4096), grid mode on one huge set (HBM-bound) and the all-pairs equal-component count
    (integer-ALU-bound).  Device time by CUDA events on the stream."""
    import numpy as np
    import torch
    from paper_1911_00675_gb300 import pmh
    from paper_1911_00675_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    # precision config: 10,000 sets x n = 10,000, Pareto(1.5) weights, m = 4096, ProbMinHash2 and 4,
    # FP32 candidates + FP64 recheck against the all-FP64 path on identical inputs
    b3 = W.batch_c3()
    ids3 = torch.from_numpy(b3.ids.view(np.int64)).to(dev)
    w3 = torch.from_numpy(b3.weights).to(dev)
    off3 = torch.from_numpy(b3.offsets).to(dev)
    n3 = b3.num_elements
    S3 = b3.num_sets
    del b3
    v3 = ["2", "4"]
    z3 = {p: torch.empty((2, S3, 4096), dtype=torch.int64, device=dev) for p in (0, 1)}
    st3 = {p: torch.empty((2, S3), dtype=torch.int32, device=dev) for p in (0, 1)}
    res = {}
    for prec, name, k in ((pmh.FP32_RECHECK, "fp32", steps), (pmh.FP64, "fp64", 1)):
        ms = timed(lambda: h.sketch_batch(ids3, w3, off3, 4096, v3, prec, 0, out_ids=z3[prec], status=st3[prec]), k)
        res[name] = {"ms": ms, "elements_per_s": 2 * n3 / (ms * 1e-3),
                     "status_ok": bool((st3[prec] == 0).all().item())}
    cnt3 = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device=dev)
    h.sketch_batch(ids3, w3, off3, 4096, v3, pmh.FP32_RECHECK, 0, out_ids=z3[1], status=st3[1], counters=cnt3)
    torch.cuda.synchronize()
    c3 = dict(zip(pmh.COUNTERS, cnt3.cpu().tolist()))
    out["precision_c3"] = {
        "workload": "10,000 sets x n=10,000, Pareto(x_m=1, tail 1.5) weights, m=4096, ProbMinHash2 and 4",
        **res, "speedup_fp32_vs_fp64": res["fp64"]["ms"] / res["fp32"]["ms"],
        "identical_output": bool(torch.equal(z3[0], z3[1])),
        "near_margin_events": c3["contenders"], "exact_fp64_evaluations": c3["resolved"],
        "items_redone_in_fp64": c3["redo"], "components": 2 * S3 * 4096,
        "points32": c3["points32"], "points64": c3["points64"],
        "note": "near_margin_events: pairs of FP32 candidates of one component within the FP32 error bound "
                "(2^-18 relative), each resolved by exact FP64 evaluation; the oracle's own near ties "
                "(< 1e-12 relative) are counted by the GPU parity tests"}
    del ids3, w3, off3, z3, st3

    # huge set: 1e8 elements, lognormal(0, 2) weights, m = 4096, ProbMinHash3a, every SM on the one set
    b5 = W.batch_c5()
    ids5 = torch.from_numpy(b5.ids.view(np.int64)).to(dev)
    w5 = torch.from_numpy(b5.weights).to(dev)
    off5 = torch.from_numpy(b5.offsets).to(dev)
    del b5
    z5 = torch.empty((1, 1, 4096), dtype=torch.int64, device=dev)
    st5 = torch.empty((1, 1), dtype=torch.int32, device=dev)
    n5 = ids5.numel()
    res = {}
    for prec, name, k in ((pmh.FP32_RECHECK, "fp32", steps), (pmh.FP64, "fp64", 1)):
        ms = timed(lambda: h.sketch_batch(ids5, w5, off5, 4096, ["3a"], prec, 0, out_ids=z5, status=st5), k)
        res[name] = {"ms": ms, "elements_per_s": n5 / (ms * 1e-3), "status_ok": bool((st5 == 0).all().item())}
    byt = 16 * n5 + 8 * 4096
    a = byt / (res["fp32"]["ms"] * 1e-3) / 1e9
    out["huge_set"] = {"workload": "one set, n=1e8, lognormal(0,2) weights, m=4096, ProbMinHash3a, grid mode",
                       **res, "roofline": {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                           "frac": a / peaks["hbm_gbs"], "algorithmic_bytes": byt,
                                           "peak_basis": peaks["basis"]}}
    del ids5, w5, off5

    # all-pairs counts over 16,384 ProbMinHash3a signatures (m = 1024) of 512 perturbed families
    b4 = W.batch_c4_sets()
    ids4 = torch.from_numpy(b4.ids.view(np.int64)).to(dev)
    w4 = torch.from_numpy(b4.weights).to(dev)
    off4 = torch.from_numpy(b4.offsets).to(dev)
    z4, _, st4 = h.sketch_batch(ids4, w4, off4, 1024, ["3a"], pmh.FP32_RECHECK, 0)
    z4 = z4[0].contiguous()
    del ids4, w4, off4
    S4 = z4.shape[0]
    counts = torch.empty((S4, S4), dtype=torch.int16, device=dev)
    ms = timed(lambda: h.estimate_jp(z4, upper_only=True, counts=counts), steps)
    pairs = S4 * (S4 + 1) // 2
    ops = pairs * 1024 * OPS_PAIR_COMPONENT
    a = ops / (ms * 1e-3) / 1e12
    pk = alu_peak(n_sms, sm_mhz)
    out["allpairs"] = {"workload": "16,384 ProbMinHash3a signatures, m=1024, upper triangle with diagonal",
                       "ms": ms, "pairs_per_s": pairs / (ms * 1e-3),
                       "roofline": {"bound": "alu", "achieved": a, "peak": pk, "unit": "Tops/s (32-bit lane ops)",
                                    "frac": a / pk, "ops_per_launch": ops}}

    # the same signatures reduced to 8-bit codes, and their all-pairs equal-field counts
    bb = 8
    packed = h.bbit_reduce(z4, bb, seed=1)
    ms_red = timed(lambda: h.bbit_reduce(z4, bb, seed=1, packed=packed), steps)
    ms_bb = timed(lambda: h.bbit_allpairs(packed, 1024, bb, upper_only=True, counts=counts), steps)
    words = packed.shape[1]
    ops_bb = pairs * words * OPS_BBIT_WORD
    a_bb = ops_bb / (ms_bb * 1e-3) / 1e12
    red_bytes = S4 * 1024 * 8 + packed.numel() * 8
    out["bbit8"] = {"workload": "the same 16,384 signatures reduced to 8-bit codes (Algorithm b-bit), all pairs",
                    "reduce_ms": ms_red, "allpairs_ms": ms_bb, "pairs_per_s": pairs / (ms_bb * 1e-3),
                    "reduce_roofline": {"bound": "hbm", "achieved": red_bytes / (ms_red * 1e-3) / 1e9,
                                        "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                        "frac": red_bytes / (ms_red * 1e-3) / 1e9 / peaks["hbm_gbs"]},
                    "roofline": {"bound": "alu", "achieved": a_bb, "peak": pk, "unit": "Tops/s (32-bit lane ops)",
                                 "frac": a_bb / pk, "ops_per_launch": ops_bb}}
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"pmh_clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm
def workload_config(batch, world):
    """The workload both arms run: the same keys and values in the GPU line and the reference line."""
    n_elem, S = batch.num_elements, batch.num_sets
    return {"workload": f"c2: {S} sets, n log-uniform [1,1e5], Uniform(0,1] weights, m=1024, "
                        "variants 1,1a,2,3,3a,4 in one persistent launch",
            "m": batch.m, "num_sets": S, "elements_per_rank": n_elem, "variants": VARIANTS,
            "parallelism": f"weak x{world}",
            "l2": f"inputs {(16 * n_elem + 8 * S) / 1e9:.2f} GB per step > 129 MB L2"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    from paper_1911_00675_gb300 import workloads as W
    batch = W.batch_c2(num_sets=args.num_sets)
    cores = len(os.sched_getaffinity(0)) or 1
    per_step = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    for step in range(args.warmup + args.steps):
        v, el, tasks, sec = oracle_throughput(batch, per_step, cores, rng_seed=step + 1)
        if step >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(batch, world),
        "precision": "fp64 (the oracle)",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"random (set, variant) tasks of the workload for {per_step:.0f} s per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    from paper_1911_00675_gb300 import build, pmh
    from paper_1911_00675_gb300 import workloads as W

    local_cpus = bind_gpu_local_cpus(local)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    build.build()

    batch = W.batch_c2(seed=0xC0FFEE02 + rank, num_sets=args.num_sets)
    n_elem = batch.num_elements
    work = n_elem * len(VARIANTS)
    m = batch.m
    ids_h = torch.from_numpy(batch.ids.view(np.int64)).pin_memory()
    w_h = torch.from_numpy(batch.weights).pin_memory()
    off_h = torch.from_numpy(batch.offsets).pin_memory()
    ids = ids_h.to(dev)
    w = w_h.to(dev)
    off = off_h.to(dev)
    S = batch.num_sets
    out32 = torch.empty((len(VARIANTS), S, m), dtype=torch.int64, device=dev)
    out64 = torch.empty_like(out32)
    st32 = torch.empty((len(VARIANTS), S), dtype=torch.int32, device=dev)
    st64 = torch.empty_like(st32)
    h = pmh.Handle(local)
    if args.prefilter is not None:
        h.set_prefilter(args.prefilter)
    shapes_pinned = [int(x) for x in args.team_shape.split(",")]
    if len(shapes_pinned) == 1 and shapes_pinned[0] >= 0:
        h.set_team_shape(0, shapes_pinned[0])
    elif len(shapes_pinned) == 4:
        for f, sh in enumerate(shapes_pinned):
            h.set_team_shape(f + 1, sh)
    stream = torch.cuda.current_stream()

    def step(prec, out, st):
        h.sketch_batch(ids, w, off, m, VARIANTS, prec, 0, out_ids=out, status=st)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # ---------------- headline: FP32 + recheck, as the library runs it: each call replays the cached CUDA
    # graph of the batch (the first call autotunes the team shapes and captures the graph)
    h.set_profiling(False)
    for _ in range(args.warmup):
        step(pmh.FP32_RECHECK, out32, st32)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):       # enqueued back to back: no host synchronisation inside the timed region
        step(pmh.FP32_RECHECK, out32, st32)
    e1.record(stream)
    barrier()
    t32 = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    launches_per_step = h.last_launches()
    shapes_headline = h.last_team_shapes()
    # the same steps again with the library's profiling events (direct launches, not graph replay): the
    # device time of the queue build and of the sketch kernels of each call
    h.set_profiling(True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step(pmh.FP32_RECHECK, out32, st32)
    e1.record(stream)
    barrier()
    t32_profiled = max_over_ranks(e0.elapsed_time(e1) / args.steps)
    queue_ms, kernel_ms = h.kernel_ms_history(args.steps)
    h.set_profiling(False)

    # ---------------- e2e: host buffers in, signatures back, every step, through the host-buffer C-ABI
    # call (pinned host memory; the library pipelines copy-in, sketch and copy-out over chunks of sets)
    e2e = None
    h.set_profiling(False)
    if not args.no_e2e:
        out_h = torch.empty(out32.shape, dtype=torch.int64).pin_memory()

        def e2e_step():
            h.sketch_batch_host(ids_h, w_h, off_h, m, VARIANTS, pmh.FP32_RECHECK, 0, out_ids=out_h, with_status=False)

        for _ in range(2):
            e2e_step()
        barrier()
        ksteps = max(3, args.steps)
        t0 = time.perf_counter()
        spans, walls = [], []
        for _ in range(ksteps):
            s0 = time.perf_counter()
            e2e_step()   # blocking: returns once the signatures are in host memory
            walls.append((time.perf_counter() - s0) * 1e3)
            spans.append(h.last_host_span_ms()[0])
        barrier()
        # the mean step (total wall time / steps) is the end-to-end rate; the median is reported beside
        # it (the host link is shared with the other GPU of the same CPU, which slows some steps)
        te_mean = max_over_ranks((time.perf_counter() - t0) * 1e3 / ksteps)
        te_median = max_over_ranks(statistics.median(walls))
        identical_e2e = bool(torch.equal(out_h, out32.cpu()))
        # the copies alone, for reference: inputs in, signatures out (pinned, one stream)
        barrier()
        c0 = time.perf_counter()
        ids.copy_(ids_h, non_blocking=True)
        w.copy_(w_h, non_blocking=True)
        torch.cuda.synchronize()
        c1 = time.perf_counter()
        out_h.copy_(out32, non_blocking=True)
        torch.cuda.synchronize()
        c2 = time.perf_counter()
        h2d = ids_h.numel() * 8 + w_h.numel() * 8 + off_h.numel() * 8
        d2h = out_h.numel() * 8
        e2e = {"value": work * world / (te_mean * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": te_mean, "ms_per_step_median": te_median,
               "value_median_step": work * world / (te_median * 1e-3),
               "timing": f"host wall clock over {ksteps} blocking calls / {ksteps} (median step beside it)",
               "step_ms": walls,
               "identical_output": identical_e2e,
               "host_cpus": local_cpus, "copy_in_ms": (c1 - c0) * 1e3, "copy_out_ms": (c2 - c1) * 1e3,
               "device_span_ms": statistics.mean(spans), "device_span_ms_min": min(spans),
               "device_span_ms_median": statistics.median(spans), "chunks": h.last_host_span_ms()[1]}

    # ---------------- comparator: plain FP64 (graph replay as well), then its kernel time from profiled calls
    for _ in range(min(args.warmup, 2)):
        step(pmh.FP64, out64, st64)
    barrier()
    e0.record(stream)
    for _ in range(args.fp64_steps):
        step(pmh.FP64, out64, st64)
    e1.record(stream)
    barrier()
    t64 = max_over_ranks(e0.elapsed_time(e1) / max(1, args.fp64_steps))
    h.set_profiling(True)
    step(pmh.FP64, out64, st64)
    k64 = h.kernel_ms_history(1)[1] or [float("nan")]
    clk = clocks.stop()
    h.set_profiling(False)

    identical = bool(torch.equal(out32, out64))
    statuses_ok = bool((st32 == 0).all().item() and (st64 == 0).all().item())

    # ---------------- counters of one (untimed) step
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device=dev)
    h.sketch_batch(ids, w, off, m, VARIANTS, pmh.FP32_RECHECK, 0, out_ids=out32, status=st32, counters=cnt)
    torch.cuda.synchronize()
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))

    # ---------------- roofline of the dominant kernel (the persistent sketch kernel)
    k_avg = statistics.mean(kernel_ms)
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    survivors = c["elements"] - c["prefiltered"]
    # algorithmic work: the per-unit figures x the units one step processes (every element-variant of
    # the batch, every point the kernels evaluated, every survivor)
    per_launch_ops = work * OPS_ELEMENT + c["points32"] * OPS_POINT + survivors * OPS_SURVIVOR
    # the operations this design executes for them: the prefilter pass hashes the elements of listed
    # sets once for all variants (c["list_hashed"]); the variants then filter only the list entries
    # (c["listed"]) and skip the rest (c["list_skipped"]); extra rounds revisit elements
    filtered_full = c["elements"] - c["list_skipped"] - c["listed"]
    executed_ops = (filtered_full * OPS_ELEMENT + c["listed"] * OPS_LISTED + c["list_hashed"] * OPS_ELEMENT
                    + c["points32"] * OPS_POINT + survivors * OPS_SURVIVOR)
    achieved = per_launch_ops / (k_avg * 1e-3) / 1e12
    peak = n_sms * LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (32-bit lane ops)",
                "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_ELEMENT_VARIANT * work,
                "traffic_basis": TRAFFIC_BASIS,
                "kernel": "pmh::list_kernel + pmh::sketch_kernel<FP32> (prefilter pass and four family launches per step)",
                "kernel_ms": k_avg, "kernel_ms_basis": "library CUDA events around the prefilter pass and the sketch "
                                                         "kernels of each profiled call (the second timed pass)",
                "ops_per_launch": per_launch_ops,
                "ops_basis": f"{OPS_ELEMENT} per element-variant x {work} + {OPS_POINT} per point x points32 "
                             f"{OPS_SURVIVOR:+d} per survivor",
                "executed_ops_per_launch": executed_ops,
                "frac_executed": executed_ops / (k_avg * 1e-3) / 1e12 / peak,
                "peak_basis": f"{n_sms} SMs x {LANES_PER_SM_CLK} lane-ops/clk x {sm_mhz:.0f} MHz (median under load)",
                "ncu": NCU_SKETCH}

    # ---------------- queue build + set statistics: one read of offsets (x3) and weights
    peaks = measured_peaks()
    q_avg = statistics.mean(queue_ms)
    q_bytes = 8 * n_elem + 3 * 8 * (S + 1) + 8 * S * len(VARIANTS)
    qa = q_bytes / (q_avg * 1e-3) / 1e9
    queue_roof = {"bound": "hbm", "achieved": qa, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": qa / peaks["hbm_gbs"],
                  "algorithmic_bytes": q_bytes, "ms": q_avg, "peak_basis": peaks["basis"]}

    sec_res = None
    if not args.no_secondary:
        sec_res = secondary(h, dev, n_sms, sm_mhz, peaks)
        sec_res["te_sampler"] = te_sampler_comparison(h, ids, w, off, m, n_elem)
        sec_res["pminhash_vs_probminhash"] = pminhash_comparison(h, dev)

    # ---------------- CPU baseline (rank 0, N=1 only), and the GPU's point work on the same tasks
    cpu = None
    overhead = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0)) or 1
        done = []
        v, el, tasks, sec = oracle_throughput(batch, args.cpu_seconds, cores, done=done)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{tasks} random (set, variant) tasks, {el} elements, {sec:.1f} s wall on {cores} processes"}
        overhead = parallel_overhead(h, batch, done, dev)

    if rank == 0:
        value = work * world / (t32 * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(batch, world),
            "precision": "fp32 candidates + fp64 recheck", "team_shapes": shapes_headline,
            "timing": "CUDA events around the timed steps on the launching stream; each step replays the "
                      "library's cached CUDA graph",
            "ms_per_step_profiled": t32_profiled,
            "fp64": {"value": work * world / (t64 * 1e-3), "ms_per_step": t64, "kernel_ms": statistics.mean(k64),
                     "speedup_fp32_vs_fp64": t64 / t32},
            "identical_output": identical, "status_ok": statuses_ok,
            # per-phase cycle counters are recorded only by a build with PMH_CYCLE_COUNTERS=1
            "counters": {k: v for k, v in c.items() if not (k.startswith("cyc_") and v == 0)},
            "queue_build_ms": statistics.mean(queue_ms),
            "roofline": roofline,
            "queue_build_roofline": queue_roof,
            "parallel_overhead": overhead,
            "secondary": sec_res,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,   # as reported by the library for each call
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
