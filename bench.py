#!/usr/bin/env python
"""Benchmark of the GB300 sparse TTV library.

One step = one complete TTV (stream, gather, scale, linearise, accumulate,
emit) of the chosen workload through the library's C ABI, computed from the
raw COO input every step.  Default workload: the largest single TTV, mode 2
of a 5-way 20000x5000x100000x2000x500 tensor with 1e8 distinct nonzeros whose
subscripts are Zipf(1.2) per mode, values N(0,1), vector U[-1,1], sparse
4-way result of about 6.1e7 rows; subscripts stored as d contiguous columns
(pyttb's column-major layout).  Inputs (4.8 GB) are larger than L2, so no
flush between steps.  The roofline of that workload is the whole step's:
algorithmic bytes (subs + vals once, the vector once, the result rows once)
over the step time.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import synthetic as S  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}

WORKLOADS = {
    "allbutone_4way_1000": dict(
        make=lambda dev, seed, nnz=None: S.allbutone_4way_1000(seed=seed, device=dev, nnz=nnz or 10_000_000), fmt="dense",
        desc="all-but-one TTV, modes 0,1,3 of a 1000^4 COO tensor, nnz 1e7 uniform distinct, U[-1,1], dense 1000 result"),
    "single_5way_zipf": dict(
        make=lambda dev, seed, nnz=None: S.single_5way_zipf(seed=seed, device=dev, nnz=nnz or 100_000_000), fmt="sparse",
        desc="single TTV mode 2 of a 20000x5000x100000x2000x500 COO tensor, nnz 1e8 Zipf(1.2) distinct, N(0,1), sparse 4-way result"),
    "batch_512": dict(make=None, fmt="sparse",
        desc="512 independent 3-to-5-way COO tensors, nnz log-uniform [1e3, 2e6], sizes U[50, 50000], own mode each, one graph launch"),
    "serve_64": dict(make=None, fmt="sparse",
        desc="Poisson TTV requests against 64 resident 4-way FP32 tensors (nnz log-uniform [1e4, 5e7]), random mode, fresh vectors"),
    "dot_1e8": dict(make=None, fmt=None,
        desc="dense dot product (Eq. 1) of two float64 vectors of 1e8 elements, U[0,1)"),
    "matvec_1e4": dict(make=None, fmt=None,
        desc="dense matrix-vector product (Eq. 2), float64 10000x10000 matrix (--order C or F), U[0,1)"),
    "paper_sweep": dict(make=None, fmt=None,
        desc="the paper's TTV experiment (Sec. 4.3): n^3 COO tensors, n = 100..1200, density 1 %, values and "
             "vector U[0,1], vector along the second mode; one line with every n"),
    "single_3way_100": dict(
        make=lambda dev, seed, nnz=None: S.single_3way_100(seed=seed, device=dev), fmt="sparse",
        desc="single TTV mode 0 of a 100^3 COO tensor, nnz 1e4 uniform distinct, sparse 100x100 result"),
}

# Nonzeros of the single-tensor workloads at full size.
WORKLOAD_NNZ = {"allbutone_4way_1000": 10_000_000, "single_5way_zipf": 100_000_000, "single_3way_100": 10_000}

# Kernel whose roofline is reported, per workload, and its algorithmic bytes
# per launch: every nonzero's d subscripts and value read once, plus the
# contracted vectors once.
# The kernel that dominates each workload, and the bytes one launch of it
# must move: the streaming kernels read the tensor and the vectors once
# (nnz*(8d + w) + vectors); one onesweep digit pass reads and writes every
# (key, term) pair once (32 bytes per nonzero).
def _stream_bytes(problem, ab):
    return ab["input"] + ab["vectors"]


def _pass_bytes(problem, ab):
    return 32 * problem.tensor.nnz


def _prepared_emit_bytes(problem, ab):
    # a prepared run's emit pass reads key, value and the contracted
    # subscripts (int32) of every nonzero and writes every result row
    t = problem.tensor
    w = t.vals.element_size()
    return t.nnz * (8 + w + 4 * len(problem.modes)) + ab["output"]


DOMINANT_PREPARED = [("rbk_emit", _prepared_emit_bytes)]

# Workloads whose step runs several kernels of comparable weight: their
# "roofline" is taken over the whole step (the algorithmic bytes of one TTV
# over the step time); the dominant kernel's own figure is reported beside it.
STEP_ROOFLINE = {"single_5way_zipf"}

DOMINANT = {"allbutone_4way_1000": [("dense_accum", _stream_bytes), ("dense_fx", _stream_bytes)],
            "single_5way_zipf": [("onesweep", _pass_bytes), ("keys_terms", _stream_bytes)],
            "single_3way_100": [("dense_accum", _stream_bytes), ("dense_fx", _stream_bytes)]}

# DRAM bytes of one whole step of the step-roofline workloads (the sum of
# dram__bytes_read.sum + dram__bytes_write.sum over the step's launches, from
# the ncu launch list under profiles/), with the sha1 of the sources those
# kernels are built from; reported as null once the sources differ.
STEP_TRAFFIC = {
    "batch_512": {
        "files": ["ttv_keys.cu", "ttv_sort.cu", "ttv_internal.cuh", "ttv_udiv.h"],
        "sha": "4c23fb15fea3",
        "bytes_per_step": 43772273664,   # the 19 stage-wise launches of one step; 4.14x the algorithmic bytes
    },
    "single_5way_zipf": {
        "files": ["ttv_keys.cu", "ttv_sort.cu", "ttv_internal.cuh", "ttv_udiv.h"],
        "sha": "4c23fb15fea3",
        "bytes_per_step": 31025177088,   # 12 launches of one (warm) TTV; 4.3x the algorithmic bytes
    },
}

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel from an ncu capture of this workload (summary under profiles/), with
# the sha1 of the sources that kernel is built from; reported as null once
# those sources differ from the ones the counters were taken on.
TRAFFIC = {
    "allbutone_4way_1000": {
        "kernel": "dense_accum",
        "files": ["ttv_dense_vec.cu", "ttv_internal.cuh", "ttv_udiv.h", "ttv_tma.cuh"],
        "sha": "cbcfd784a6c0",
        "bytes_per_launch": 400297495,   # 400.08 MB read + 0.21 MB written, mean of 45 launches
    },
}


def kernel_source_hash(files=None) -> str:
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2510_01495_gb300", "csrc")
    names = files if files else sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h")))
    for f in names:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:12]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(problem, nnz_out: int, w: int = 8) -> dict:
    """Bytes a TTV must move: subs + vals once, contracted vectors once, and
    the result (rows of order int64 subscripts plus a value; values only when
    dense)."""
    t = problem.tensor
    d = t.d
    vec = sum(t.shape[m] for m in problem.modes) * w
    order = d - len(problem.modes)
    inp = t.nnz * (8 * d + w)
    out = nnz_out * (8 * order + 8) if not problem.dense else nnz_out * 8
    return {"input": inp, "vectors": vec, "output": out, "total": inp + vec + out,
            "gathered_per_nonzero": t.nnz * len(problem.modes) * w}


# Per-kernel CUDA events bracket every launch of every PROFILE_EVERY-th timed
# step: the kernels' durations are measured inside the timed region, while
# the event records stay out of the other steps (recording around every
# launch added about 10 us to a 0.12 ms step).
PROFILE_EVERY = 8


def profiler_prewarm(ttv, step, steps: int):
    """Runs the sampled steps' worth of profiled steps before the timed region
    so that the library's pool already holds every CUDA event they need."""
    ttv.profile_enable(True)
    for _ in range(steps // PROFILE_EVERY + 1):
        step()
    torch.cuda.synchronize()
    ttv.profile_collect()
    ttv.profile_reset()
    ttv.profile_enable(False)


def profiled(ttv, i: int, fn):
    """fn(), with per-launch events when step i is a sampled one."""
    if i % PROFILE_EVERY:
        return fn()
    ttv.profile_enable(True)
    try:
        return fn()
    finally:
        ttv.profile_enable(False)


def cpu_parallel_sample(problem, target_s: float = 5.0, max_nnz: int = 20_000_000):
    """The same definition on all allowed host cores (the oracle's OpenMP
    statement, bit-identical to it) on the first m nonzeros; GNNZ/s, m,
    seconds, threads -- or None when it could not be built."""
    import oracle
    try:
        oracle.build_parallel()
        threads = oracle.parallel_threads()
    except Exception:   # noqa: BLE001
        return None
    t = problem.tensor
    subs = t.subs.cpu().numpy()
    vals = t.vals.cpu().numpy()
    vecs = [v.cpu().numpy() for v in problem.vecs]
    m = min(t.nnz, 500_000)
    t0 = time.perf_counter()
    oracle.ttv_parallel(subs[:m], vals[:m], t.shape, problem.modes, vecs, dense=problem.dense)
    dt = time.perf_counter() - t0
    m2 = int(min(t.nnz, max_nnz, max(m, m * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.ttv_parallel(subs[:m2], vals[:m2], t.shape, problem.modes, vecs, dense=problem.dense)
    dt2 = time.perf_counter() - t0
    return m2 / dt2 / 1e9, m2, dt2, threads


def cpu_oracle_sample(problem, target_s: float = 10.0, max_nnz: int = 20_000_000):
    """The CPU oracle on the first m nonzeros of the workload (m chosen so the
    call runs ~target_s seconds, at most max_nnz); returns GNNZ/s and what was run."""
    import oracle
    t = problem.tensor
    subs = t.subs.cpu().numpy() if t.subs.is_cuda else t.subs.numpy()
    vals = t.vals.cpu().numpy()
    vecs = [v.cpu().numpy() for v in problem.vecs]
    oracle.build()
    m = min(t.nnz, 200_000)
    t0 = time.perf_counter()
    oracle.ttv(subs[:m], vals[:m], t.shape, problem.modes, vecs, dense=problem.dense)
    dt = time.perf_counter() - t0
    m2 = int(min(t.nnz, max_nnz, max(m, m * target_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.ttv(subs[:m2], vals[:m2], t.shape, problem.modes, vecs, dense=problem.dense)
    dt2 = time.perf_counter() - t0
    return m2 / dt2 / 1e9, m2, dt2


# ---- ranks: independent replicas (no data-path collective) -------------------

def replica_seed(base: int, rank: int) -> int:
    """Each rank draws its own replica of the workload."""
    return base + 1000 * rank


def init_ranks(world: int, dev):
    """Process group for the barrier and the timing reduction (NCCL on the
    GPU); None with one rank."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        if dev is not None and dev.type == "cuda":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group("gloo")
    return dist


def sum_over_ranks(dist, value: float, dev) -> float:
    """The sum of every rank's value (work done by all replicas)."""
    if dist is None:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, dev) -> float:
    """The largest of every rank's value (timings: the slowest replica sets
    the job's time)."""
    if dist is None:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step a bounded sample."""
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    if wl["make"] is None:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm covers the single-tensor TTV "
                          f"workloads, not {args.workload}"}), flush=True)
        return
    # The generator keeps the first distinct rows in draw order, so the first
    # m nonzeros of a smaller draw are exactly the full workload's first m:
    # only the largest sample a step can use is drawn.
    problem = wl["make"]("cpu", args.seed, min(args.nnz or WORKLOAD_NNZ[args.workload], args.ref_sample))
    import oracle
    oracle.build()
    t = problem.tensor
    full = args.nnz or WORKLOAD_NNZ[args.workload]
    subs, vals = t.subs.numpy(), t.vals.numpy()
    vecs = [v.numpy() for v in problem.vecs]
    # per-step sample: the oracle's measured rate on a calibration call sets
    # it so that the whole --steps/--warmup run takes about ref_budget seconds
    mc = min(t.nnz, 200_000)
    t0 = time.perf_counter()
    oracle.ttv(subs[:mc], vals[:mc], t.shape, problem.modes, vecs, dense=problem.dense)
    rate = mc / max(time.perf_counter() - t0, 1e-6)
    m = int(rate * args.ref_budget / max(1, args.steps + args.warmup))
    m = max(1000, min(t.nnz, args.ref_sample, m))
    for _ in range(args.warmup):
        oracle.ttv(subs[:m], vals[:m], t.shape, problem.modes, vecs, dense=problem.dense)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.ttv(subs[:m], vals[:m], t.shape, problem.modes, vecs, dense=problem.dense)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": "TTV nonzeros/sec", "value": value, "unit": "GNNZ/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "layout": "aos", "sample_nnz": m},
        "cpu_baseline": {"value": value, "unit": "GNNZ/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {m} of {full} nonzeros per step"},
        "e2e": {"value": value, "unit": "GNNZ/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single_5way_zipf", choices=sorted(WORKLOADS))
    ap.add_argument("--path", default="auto")
    ap.add_argument("--accum", default="fp64", choices=["fp64", "compensated", "exact"])
    ap.add_argument("--layout", default="soa", choices=["soa", "aos"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--nnz", type=int, default=None, help="smaller case of the workload (profiling)")
    ap.add_argument("--no-tune", action="store_true", help="batch_512: skip the autotuner (planner rule only)")
    ap.add_argument("--prepared", action="store_true",
                    help="single workloads: prepare the tensor once (untimed), then time prepared runs")
    ap.add_argument("--order", default="F", choices=["C", "F"], help="matvec_1e4: matrix storage order")
    ap.add_argument("--mttkrp", type=int, default=0, metavar="R",
                    help="single workloads: time MTTKRP of rank R on the prepared tensor instead of the TTV")
    ap.add_argument("--ref-sample", type=int, default=1_000_000, help="largest per-step oracle sample")
    ap.add_argument("--ref-budget", type=float, default=90.0, help="seconds the reference arm's timed steps aim at")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--scale", type=float, default=1.0, help="nnz scale for batch_512 / serve_64")
    ap.add_argument("--requests", type=int, default=2000, help="serve_64: requests in the timed stream")
    ap.add_argument("--rate", type=float, default=20000.0, help="serve_64: Poisson arrival rate (req/s)")
    ap.add_argument("--light-rate", type=float, default=200.0, help="serve_64: arrival rate of the light-load leg")
    args = ap.parse_args()
    if args.seed == 0:
        args.seed = {"allbutone_4way_1000": 2, "single_5way_zipf": 3, "single_3way_100": 1, "batch_512": 5,
                     "serve_64": 6, "dot_1e8": 8, "matvec_1e4": 9, "paper_sweep": 4}[args.workload]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch_512":
        return run_batch(args, rank, world, local_rank)
    if args.workload == "serve_64":
        return run_serve(args, rank, world, local_rank)
    if args.mttkrp:
        return run_mttkrp(args, rank, world, local_rank)
    if args.workload in ("dot_1e8", "matvec_1e4"):
        return run_dense(args, rank, world, local_rank)
    if args.workload == "paper_sweep":
        return run_paper_sweep(args, rank, world, local_rank)

    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = init_ranks(world, dev)
    lib = ttv.load()

    wl = WORKLOADS[args.workload]
    # independent replica per rank: its own seed, no data-path collective
    problem = wl["make"](dev, replica_seed(args.seed, rank), args.nnz)
    t = problem.tensor
    if args.layout == "soa":
        subs = t.subs.t().contiguous().t()
    else:
        subs = t.subs.contiguous()
    vals = t.vals.contiguous()
    vecs = [v.contiguous() for v in problem.vecs]
    fmt = wl["fmt"]
    del t

    # preallocated workspace and result (the steady-state way to call the ABI)
    ws_bytes = ttv.workspace_size(subs, vals, problem.tensor.shape, problem.modes, fmt=fmt, path=args.path,
                                  accum=args.accum)
    workspace = torch.empty(max(1, ws_bytes), dtype=torch.uint8, device=dev)
    rows, nv = ttv.out_capacity(subs, vals, problem.tensor.shape, problem.modes, fmt=fmt, path=args.path)
    order = problem.tensor.d - len(problem.modes)
    out_vals = torch.empty(nv, dtype=torch.float64, device=dev)
    out_subs = torch.empty((max(1, rows), max(1, order)), dtype=torch.int64, device=dev) if fmt != "dense" else None

    stream = torch.cuda.current_stream(dev)
    tdesc = ttv.make_tensor(subs, vals, problem.tensor.shape)
    modes_c = (ctypes.c_int32 * len(problem.modes))(*problem.modes)
    vecp = (ctypes.c_void_p * len(vecs))(*[v.data_ptr() for v in vecs])
    lens = (ctypes.c_int64 * len(vecs))(*[v.numel() for v in vecs])
    opts = ttv.make_opts(fmt=fmt, path=args.path, accum=args.accum, workspace=workspace, async_=True)
    sh = ctypes.c_void_p(stream.cuda_stream)
    prepared = None
    if args.prepared:
        # the tensor is prepared once, outside the timed region (a resident
        # tensor queried repeatedly with fresh vectors)
        t_prep = time.perf_counter()
        prepared = ttv.Prepared(subs, vals, problem.tensor.shape, problem.modes, stream=stream)
        torch.cuda.synchronize(dev)
        t_prep = time.perf_counter() - t_prep
        workspace = torch.empty(max(1, prepared.workspace_bytes), dtype=torch.uint8, device=dev)
        opts = ttv.make_opts(fmt=fmt, workspace=workspace, async_=True)

    def submit():
        res = ttv.Out()
        res.vals = out_vals.data_ptr()
        res.vals_capacity = out_vals.numel()
        if out_subs is not None:
            res.subs = out_subs.data_ptr()
            res.subs_capacity = out_subs.shape[0]
        if prepared is not None:
            rc = lib.ttv_prepared_run(prepared._h, vecp, lens, 0, ctypes.byref(res), ctypes.byref(opts), sh)
        else:
            rc = lib.ttv_multi_checked(ctypes.byref(tdesc), modes_c, len(problem.modes), vecp, lens, 0,
                                       ctypes.byref(res), ctypes.byref(opts), sh)
        if rc != 0:
            raise ttv.TTVError(rc, lib.ttv_last_error().decode())
        return res

    def finish(results):
        nnz_out = None
        for r in results:
            rc = lib.ttv_out_sync(ctypes.byref(r))
            if rc != 0:
                raise ttv.TTVError(rc, lib.ttv_last_error().decode())
            nnz_out = int(r.nnz)
            lib.ttv_out_free(ctypes.byref(r))
        return nnz_out

    for _ in range(args.warmup):
        nnz_out = finish([submit()])
    torch.cuda.synchronize(dev)
    profiler_prewarm(ttv, lambda: finish([submit()]), args.steps)

    # ---- timed region: K steps, device resident inputs ----
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ttv.profile_reset()
    barrier(dist)
    torch.cuda.synchronize(dev)
    launches0 = ttv.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    pending = []
    for i in range(args.steps):
        pending.append(profiled(ttv, i, submit))
        if len(pending) >= 64:
            finish(pending[:-8])
            pending = pending[-8:]
    ev1.record(stream)
    nnz_out = finish(pending)
    torch.cuda.synchronize(dev)
    barrier(dist)
    launches = ttv.launch_count() - launches0
    ms = ev0.elapsed_time(ev1)
    ttv.profile_collect()
    clk = clocks.stop()
    ms = max_over_ranks(dist, ms, dev)
    nnz = problem.tensor.nnz
    prep_info = None
    if prepared is not None:
        prep_info = {"prepare_s": round(t_prep, 3), "device_bytes": prepared.device_bytes,
                     "note": "the tensor is sorted once by its result key outside the timed region"}
    value = nnz * args.steps * world / (ms * 1e-3) / 1e9
    ms_step = ms / args.steps

    # ---- per-kernel roofline of the dominant kernel ----
    peaks, peak_src = load_peaks()
    per_kernel = {}
    for name in ttv.profile_names():
        tot, n = ttv.profile_get(name)
        per_kernel[name] = {"ms_total": tot, "launches": n, "ms_avg": tot / max(1, n)}
    ab = algorithmic_bytes(problem, nnz_out if fmt != "dense" else int(np.prod([problem.tensor.shape[m] for m in range(problem.tensor.d) if m not in problem.modes])))
    dom_list = DOMINANT_PREPARED if args.prepared else DOMINANT[args.workload]
    dom, dom_bytes = next(((k, f(problem, ab)) for k, f in dom_list if k in per_kernel), (None, None))
    if dom is None and per_kernel:
        dom = max(per_kernel, key=lambda k: per_kernel[k]["ms_total"])
        dom_bytes = _stream_bytes(problem, ab)
    dom_ms = per_kernel.get(dom, {}).get("ms_avg", float("nan"))
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms and dom_ms == dom_ms else None
    peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    src_hash = kernel_source_hash()
    traffic = None
    tr = TRAFFIC.get(args.workload)
    default_cfg = (args.layout == "soa" and args.accum == "fp64" and args.path == "auto" and not args.nnz and
                   not args.prepared)
    if tr and default_cfg and tr.get("kernel") == dom and kernel_source_hash(tr["files"]) == tr["sha"]:
        traffic = tr["bytes_per_launch"]

    line = {
        "metric": "TTV nonzeros/sec", "value": value, "unit": "GNNZ/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "layout": args.layout,
                   "path": "prepared" if args.prepared else args.path,
                   "accum": args.accum,
                   "nnz": nnz, "nnz_out": nnz_out, "l2": "inputs larger than L2 (no flush)",
                   "kernel_timing": f"CUDA events around every launch of every {PROFILE_EVERY}th timed step",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_src} hbm_gbs", "alg_bytes_per_launch": dom_bytes},
        "step_roofline": {"alg_bytes_per_step": ab["total"], "achieved_gbs": ab["total"] / (ms_step * 1e-3) / 1e9,
                          "frac": ab["total"] / (ms_step * 1e-3) / 1e9 / peak,
                          "with_gathered_vectors_gbs": (ab["total"] + ab["gathered_per_nonzero"]) / (ms_step * 1e-3) / 1e9},
        "kernels": per_kernel,
        "gpu_launches": launches,
        "clocks": clk,
        "sources": src_hash,
    }
    if prep_info:
        line["prepared"] = prep_info
    if args.workload in STEP_ROOFLINE and not args.prepared:
        # several kernels of comparable weight: the roofline is the step's
        # (algorithmic bytes of one TTV over the step time); the dominant
        # kernel's own rate, on the bytes one launch of it moves, stays beside it
        line["dominant_kernel"] = dict(line["roofline"])
        line["dominant_kernel"]["bytes_basis"] = ("bytes one launch of this kernel moves (not the TTV's "
                                                  "algorithmic bytes)")
        step_gbs = ab["total"] / (ms_step * 1e-3) / 1e9
        st_tr = STEP_TRAFFIC.get(args.workload)
        step_traffic = None
        if st_tr and default_cfg and kernel_source_hash(st_tr["files"]) == st_tr["sha"]:
            step_traffic = st_tr["bytes_per_step"]
        line["roofline"] = {
            "bound": "hbm", "kernel": "whole step: " + " + ".join(sorted(per_kernel)), "achieved": step_gbs,
            "peak": peak, "unit": "GB/s", "frac": step_gbs / peak, "traffic": step_traffic,
            "peak_source": f"{peak_src} hbm_gbs",
            "alg_bytes_per_step": ab["total"],
            "alg_bytes_basis": "nnz*(8d+w) + vector once + nnz_out*(8*order+8)"}

    # ---- end to end: host buffers through the public call ----
    if rank == 0 or world > 1:
        e2e = run_e2e(ttv, problem, subs, vals, vecs, fmt, args, dev)
        if dist:
            # whole job: every replica's nonzeros over the slowest replica's time
            e2e["ms_per_step"] = max_over_ranks(dist, e2e["ms_per_step"], dev)
            e2e["value"] = nnz * world / (e2e["ms_per_step"] * 1e-3) / 1e9
        line["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, m, dt = cpu_oracle_sample(problem)
        line["cpu_baseline"] = {"value": v, "unit": "GNNZ/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {m} of {nnz} nonzeros, one call, {dt:.1f} s"}
        par = cpu_parallel_sample(problem)
        if par is not None:
            pv, pm, pdt, pth = par
            line["cpu_baseline_parallel"] = {
                "value": pv, "unit": "GNNZ/s", "cores": pth, "kind": "oracle-openmp",
                "sample": f"first {pm} of {nnz} nonzeros, one call, {pdt:.1f} s; per-thread sorts of contiguous "
                          f"ranges merged into the one-core oracle's order (bit-identical result)"}
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _clock_start(local_rank):
    c = ClockSampler(local_rank)
    c.start()
    time.sleep(0.3)
    return c


def run_batch(args, rank, world, local_rank):
    """512 independent TTVs per step: one graph launch (ttv_batch) against a
    loop of single asynchronous ttv_multi launches over the same problems."""
    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ttv.load()
    dist = init_ranks(world, dev)
    probs = S.batch_problems(seed=replica_seed(args.seed, rank), count=512, scale=args.scale, device=dev)
    items = []
    for p in probs:
        t = p.tensor
        items.append((t.subs.t().contiguous().t(), t.vals, t.shape, p.modes, p.vecs))
    total_nnz = sum(p.tensor.nnz for p in probs)
    # autotune: one record per problem class (untimed), consulted when the
    # graph is captured and by the loop of singles alike
    t_tune = time.perf_counter()
    tuned = 0
    if not args.no_tune:
        ttv.tune_clear()
        for it in items:
            if ttv.tune_lookup(it[0], it[1], it[2], it[3]) is None:
                ttv.autotune(it[0], it[1], it[2], it[3], it[4], trials=2)
                tuned += 1
    t_tune = time.perf_counter() - t_tune
    chosen = {}
    for it in items:
        rec = ttv.tune_lookup(it[0], it[1], it[2], it[3])
        key = rec[0] if rec else "untuned"
        chosen[key] = chosen.get(key, 0) + 1
    b = ttv.Batch(items)
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    clocks = _clock_start(local_rank)
    ttv.profile_reset()
    ttv.profile_enable(False)
    l0 = ttv.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        b.run()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1) / args.steps, dev)
    launches = ttv.launch_count() - l0
    clk = clocks.stop()
    # the plain form: one launch sequence per problem, same buffers
    outs = [(ttv.workspace_size(it[0], it[1], it[2], it[3]), ttv.out_capacity(it[0], it[1], it[2], it[3]))
            for it in items]
    wss = [torch.empty(max(1, w), dtype=torch.uint8, device=dev) for w, _ in outs]
    ovs = [torch.empty(max(1, c[1]), dtype=torch.float64, device=dev) for _, c in outs]
    oss = [torch.empty((max(1, c[0]), len(it[2]) - len(it[3])), dtype=torch.int64, device=dev)
           for (_, c), it in zip(outs, items)]

    def loop_once():
        for it, w, ov, os_ in zip(items, wss, ovs, oss):
            ttv.ttv_multi(it[0], it[1], it[2], it[3], it[4], workspace=w, out_vals=ov, out_subs=os_)

    for _ in range(max(1, args.warmup // 2)):
        loop_once()
    torch.cuda.synchronize(dev)
    k2 = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(k2):
        loop_once()
    torch.cuda.synchronize(dev)
    ms_loop = (time.perf_counter() - t0) * 1e3 / k2
    value = total_nnz * world / (ms * 1e-3) / 1e9
    line = {
        "metric": "TTV nonzeros/sec", "value": value, "unit": "GNNZ/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch_512", "desc": WORKLOADS["batch_512"]["desc"], "problems": len(probs),
                   "nnz_total": total_nnz, "scale": args.scale, "l2": "inputs larger than L2 (no flush)"},
        "loop_of_singles": {"value": total_nnz / (ms_loop * 1e-3) / 1e9, "unit": "GNNZ/s", "ms_per_step": ms_loop,
                            "note": "one synchronous ttv_multi per problem (host-timed)"},
        "graph_kernel_launches_per_step": b.graph_launches(), "gpu_launches": launches, "clocks": clk,
        "autotune": {"classes_tuned": tuned, "seconds": round(t_tune, 2), "problems_by_path": chosen},
    }
    # the step's roofline: every problem's algorithmic bytes over the step time
    res = b.run()
    torch.cuda.synchronize(dev)
    nnz_out = [int(res[i].vals.numel()) for i in range(len(probs))]
    alg = sum(algorithmic_bytes(p, n)["total"] for p, n in zip(probs, nnz_out))
    peaks, peak_src = load_peaks()
    peak = peaks["hbm_gbs"]
    step_gbs = alg / (ms * 1e-3) / 1e9
    st_tr = STEP_TRAFFIC.get("batch_512")
    traffic = None
    if st_tr and args.scale == 1.0 and world == 1 and kernel_source_hash(st_tr["files"]) == st_tr["sha"]:
        traffic = st_tr["bytes_per_step"]
    line["config"]["nnz_out_total"] = sum(nnz_out)
    line["roofline"] = {
        "bound": "hbm", "kernel": "whole step: the batch graph (stage-wise sort path)", "achieved": step_gbs,
        "peak": peak, "unit": "GB/s", "frac": step_gbs / peak, "traffic": traffic,
        "peak_source": f"{peak_src} hbm_gbs", "alg_bytes_per_step": alg,
        "alg_bytes_basis": "sum over problems of nnz*(8d+w) + vector once + nnz_out*(8*order+8)"}
    line["e2e"] = batch_e2e(ttv, b, items, probs, args, dev)
    if dist:
        line["e2e"]["ms_per_step"] = max_over_ranks(dist, line["e2e"]["ms_per_step"], dev)
        line["e2e"]["value"] = total_nnz * world / (line["e2e"]["ms_per_step"] * 1e-3) / 1e9
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(probs)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_e2e(ttv, b, items, probs, args, dev):
    """The batch through ttv_batch with HOST inputs: every problem's subs,
    vals and vector copied from pinned host memory into the buffers the
    batch was built on (so the cached graph replays), the launch, and every
    result read back, inside the timed region."""
    h_subs = [it[0].t().contiguous().cpu().pin_memory() for it in items]    # stored as d columns
    h_vals = [it[1].cpu().pin_memory() for it in items]
    h_vecs = [[v.cpu().pin_memory() for v in it[4]] for it in items]
    d_subs = [it[0].t() for it in items]             # the (d, nnz) column storage behind each view
    h2d = sum(x.numel() * 8 for x in h_subs) + sum(x.numel() * x.element_size() for x in h_vals) + \
        sum(v.numel() * v.element_size() for vs in h_vecs for v in vs)
    # pinned host buffers for the results, at the batch's output capacities
    res0 = b.run()
    h_out = [(torch.empty(tuple(m[1].shape) if m[1] is not None else (0,), dtype=torch.int64).pin_memory(),
              torch.empty(m[0].numel(), dtype=torch.float64).pin_memory()) for m in b.meta]
    del res0
    times, d2h = [], 0
    for i in range(max(1, args.e2e_steps) + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for ds, hs, it, hv, hvs in zip(d_subs, h_subs, items, h_vals, h_vecs):
            ds.copy_(hs, non_blocking=True)
            it[1].copy_(hv, non_blocking=True)
            for a, c in zip(it[4], hvs):
                a.copy_(c, non_blocking=True)
        res = b.run()
        d2h = 0
        for r, (hs_, hv_) in zip(res, h_out):
            n = r.vals.numel()
            hv_[:n].copy_(r.vals, non_blocking=True)
            d2h += n * 8
            if r.subs is not None and r.subs.numel():
                hs_[:n].copy_(r.subs, non_blocking=True)
                d2h += r.subs.numel() * 8
        torch.cuda.synchronize(dev)
        if i > 0:
            times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    total = sum(p.tensor.nnz for p in probs)
    return {"value": total / mean / 1e9, "unit": "GNNZ/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": mean * 1e3, "steps": len(times)}


def batch_cpu_baseline(probs, target_s: float = 10.0):
    """The oracle, as it stands, on whole problems of the batch taken in
    their order until about target_s seconds of one core have run."""
    import oracle
    oracle.build()
    done, nnz, t_all = 0, 0, 0.0
    for p in probs:
        t = p.tensor
        subs = t.subs.cpu().numpy()
        vals = t.vals.cpu().numpy()
        vecs = [v.cpu().numpy() for v in p.vecs]
        t0 = time.perf_counter()
        oracle.ttv(subs, vals, t.shape, p.modes, vecs, dense=p.dense)
        t_all += time.perf_counter() - t0
        done += 1
        nnz += t.nnz
        if t_all >= target_s:
            break
    return {"value": nnz / t_all / 1e9, "unit": "GNNZ/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {done} of {len(probs)} problems ({nnz} nonzeros), one call each, {t_all:.1f} s"}


def run_serve(args, rank, world, local_rank):
    """Poisson stream of TTV requests against resident FP32 tensors through
    the continuous-batching server (8 slots), against the plain
    one-request-at-a-time form (1 slot, submit then wait); p50/p99 latency
    beside throughput."""
    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ttv.load()
    dist = init_ranks(world, dev)
    seed = replica_seed(args.seed, rank)
    g = np.random.default_rng(seed)
    tensors = []
    acc_sample = []   # FP64 originals of a few small tensors, for the accuracy report
    for i in range(64):
        s = seed * 1000 + i
        r = S.uniform(s, 9, 2).numpy()
        nnz = max(1000, int(math.exp(math.log(1e4) + r[0] * (math.log(5e7) - math.log(1e4))) * args.scale))
        shp = None
        for tries in range(100):
            shp = tuple(int(x) for x in (S.uniform_int(s, 11 + tries, 4, 4901).numpy() + 100))
            if nnz <= 0.01 * float(np.prod([float(x) for x in shp])):
                break
        t = S.sptenrand(s, shp, nnz, vals="u11", device=dev)
        tensors.append((t.subs, t.vals.to(torch.float32), shp, nnz))
        if nnz <= 2_000_000 and len(acc_sample) < 8:
            acc_sample.append((t.subs, t.vals, shp, i))
    resident = sum(x[3] * (4 * 8 + 4) for x in tensors)
    srv = ttv.Server(budget_bytes=60 << 30, slots=8)
    plain = ttv.Server(budget_bytes=60 << 30, slots=1)
    ids = [srv.register(sb, vl, sh) for sb, vl, sh, _ in tensors]
    pids = [plain.register(sb, vl, sh) for sb, vl, sh, _ in tensors]
    nnzs = [x[3] for x in tensors]
    shapes = [x[2] for x in tensors]
    del tensors
    torch.cuda.empty_cache()
    reqs = []
    for _ in range(args.requests + 64):
        ti = int(g.integers(0, len(ids)))
        m = int(g.integers(0, 4))
        reqs.append((ti, m, g.uniform(-1, 1, shapes[ti][m]).astype(np.float32)))
    for ti, m, x in reqs[:64]:
        srv.wait(srv.submit(ids[ti], [m], [x], accum="compensated"), timeout_us=120_000_000)
        plain.wait(plain.submit(pids[ti], [m], [x], accum="compensated"), timeout_us=120_000_000)
    srv.reset_stats()
    clocks = _clock_start(local_rank)
    arrivals = np.cumsum(g.exponential(1.0 / args.rate, size=args.requests))

    rows = []   # result rows of each request of the last stream, in submission order

    def stream(accum, arr=None, items=None, server=None, tids=None):
        # the client takes every result as soon as it is ready (a waiter
        # thread, in submission order), so results do not pile up on the device
        import queue
        arr = arrivals if arr is None else arr
        items = reqs[64:] if items is None else items
        server = srv if server is None else server
        tids = ids if tids is None else tids
        pending = queue.Queue()
        errors = []
        rows.clear()
        rid_rows = {}
        rids = []

        def waiter():
            # results in completion order (a result left unclaimed behind a
            # slow request no longer counts against the server's budget)
            while True:
                rid = pending.get()
                if rid is None:
                    return
                try:
                    got, res = server.wait_any(timeout_us=120_000_000, copy=False)
                    rid_rows[got] = int(res.vals.numel())
                except Exception as e:   # noqa: BLE001 -- re-raised by the submitting thread
                    errors.append(e)

        th = threading.Thread(target=waiter)
        barrier(dist)
        t0 = time.perf_counter()
        th.start()
        for k, (ti, m, x) in enumerate(items):
            delay = arr[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            rid = server.submit(tids[ti], [m], [x], accum=accum)
            rids.append(rid)
            pending.put(rid)
        pending.put(None)
        th.join()
        if errors:
            raise errors[0]
        rows.extend(rid_rows[r] for r in rids)
        w = time.perf_counter() - t0
        barrier(dist)
        return max_over_ranks(dist, w, dev)

    wall = stream("compensated")
    st = srv.stats()
    # algorithmic bytes of the stream: FP32 values and vectors, int64
    # subscripts, result rows of 3 subscripts and a binary64 value
    served_bytes = sum(nnzs[ti] * (8 * 4 + 4) + shapes[ti][m] * 4 + nr * (8 * 3 + 8)
                       for (ti, m, _), nr in zip(reqs[64:], rows))
    served_rows = sum(rows)
    # light load: the same requests arriving at --light-rate, where a request
    # rarely waits for another; its latency against the one-at-a-time form
    n_light = min(300, args.requests)
    srv.reset_stats()
    light_arr = np.cumsum(g.exponential(1.0 / args.light_rate, size=n_light))
    stream("compensated", light_arr, reqs[64:64 + n_light])
    st_l = srv.stats()
    # the one-slot server on the same paced requests, right after: the same
    # client, the same state of the GPU and its memory pool
    plain.reset_stats()
    stream("compensated", light_arr, reqs[64:64 + n_light], server=plain, tids=pids)
    pst_l = plain.stats()
    # the plain form's throughput: one request at a time, submit then wait
    n_plain = min(300, args.requests)
    plain.reset_stats()
    t1 = time.perf_counter()
    for ti, m, x in reqs[64:64 + n_plain]:
        plain.wait(plain.submit(pids[ti], [m], [x], accum="compensated"), timeout_us=120_000_000)
    wall_plain = time.perf_counter() - t1
    pst = plain.stats()
    plain_nnz = sum(nnzs[ti] for ti, _, _ in reqs[64:64 + n_plain])
    # the same stream on prepared layouts (every mode of every tensor, as far
    # as the budget allows), the same compensated accumulation
    t_prep = time.perf_counter()
    n_prep = 0
    for tid in ids:
        for m in range(4):
            try:
                srv.prepare(tid, [m])
                n_prep += 1
            except ttv.TTVError:
                pass
    t_prep = time.perf_counter() - t_prep
    for ti, m, x in reqs[:64]:
        srv.wait(srv.submit(ids[ti], [m], [x], accum="compensated"), timeout_us=120_000_000)
    srv.reset_stats()
    wall_p = stream("compensated")
    st_p = srv.stats()
    clk = clocks.stop()
    served_nnz = sum_over_ranks(dist, sum(nnzs[ti] for ti, _, _ in reqs[64:]), dev)
    # accuracy of FP32 storage: the server's FP32 + compensated result against
    # the all-FP64 compensated result of the same request (values and vector
    # unrounded), per entry relative to A = TTV of |vals| with |x|
    acc = []
    for sb, v64, shp, ti in acc_sample:
        m = int(g.integers(0, 4))
        x64 = g.uniform(-1, 1, shp[m])
        r32 = srv.wait(srv.submit(ids[ti], [m], [x64.astype(np.float32)], accum="compensated"), timeout_us=120_000_000)
        xd = torch.from_numpy(x64).to(dev)
        r64 = ttv.ttv_multi(sb, v64, shp, [m], [xd], accum="compensated")
        ra = ttv.ttv_multi(sb, v64.abs(), shp, [m], [xd.abs()], accum="compensated")
        A = ra.vals.double()
        e = ((r32.vals.double() - r64.vals.double()).abs() / A.clamp_min(1e-300)).max().item()
        subs_equal = bool(torch.equal(r32.subs, r64.subs))
        acc.append({"nnz": int(v64.numel()), "mode": m, "max_err_over_A": e, "subs_equal": subs_equal})
    srv.close()
    plain.close()
    accuracy = {
        "reference": "all-FP64 compensated run of the same requests (parity tests pin it to the FP64 oracle)",
        "requests": len(acc), "max_err_over_A": max((a["max_err_over_A"] for a in acc), default=None),
        "bound_over_A": (1 + 2.0 ** -24) ** 2 - 1 + 5 * 2.0 ** -53,   # n_v = 1
        "subs_bit_exact": all(a["subs_equal"] for a in acc),
    }
    line = {
        "metric": "TTV nonzeros/sec", "value": served_nnz / wall / 1e9, "unit": "GNNZ/s", "n_gpus": world,
        "steps": args.requests, "warmup": 64, "ms_per_step": 1e3 * wall / args.requests, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 storage, f64 compensated accumulation",
        "data": "synthetic",
        "config": {"workload": "serve_64", "desc": WORKLOADS["serve_64"]["desc"], "rate_req_s": args.rate,
                   "requests": args.requests, "scale": args.scale, "resident_bytes": resident, "slots": 8,
                   "budget_bytes": 60 << 30},
        "serve": {"p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3, "max_ms": st["max_us"] / 1e3,
                  "throughput_rps": args.requests * world / wall, "completed": st["completed"]},
        "serve_light": {"rate_req_s": args.light_rate, "requests": n_light, "p50_ms": st_l["p50_us"] / 1e3,
                        "p99_ms": st_l["p99_us"] / 1e3},
        "serve_prepared": {"p50_ms": st_p["p50_us"] / 1e3, "p99_ms": st_p["p99_us"] / 1e3,
                           "throughput_rps": args.requests * world / wall_p,
                           "throughput_gnnz_s": sum_over_ranks(dist, sum(nnzs[ti] for ti, _, _ in reqs[64:]), dev)
                           / wall_p / 1e9,
                           "prepared_runs": st_p["prepared_runs"], "layouts": n_prep, "prepare_s": round(t_prep, 2),
                           "accum": "compensated (prepared runs)"},
        "plain": {"requests": n_plain, "throughput_rps": n_plain / wall_plain,
                  "throughput_gnnz_s": plain_nnz / wall_plain / 1e9, "p50_ms": pst["p50_us"] / 1e3,
                  "p99_ms": pst["p99_us"] / 1e3, "note": "one slot, submit then wait"},
        "plain_light": {"rate_req_s": args.light_rate, "requests": n_light, "p50_ms": pst_l["p50_us"] / 1e3,
                        "p99_ms": pst_l["p99_us"] / 1e3,
                        "note": "one-slot server, the light-load stream above (same arrivals, same client)"},
        "clocks": clk, "accuracy_fp32_storage": accuracy,
    }
    peaks, peak_src = load_peaks()
    served_gbs = sum_over_ranks(dist, served_bytes, dev) / wall / 1e9
    line["config"]["nnz_out_total"] = served_rows
    line["roofline"] = {
        "bound": "hbm", "kernel": "whole stream: every served request's kernels", "achieved": served_gbs,
        "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": served_gbs / peaks["hbm_gbs"], "traffic": None,
        "peak_source": f"{peak_src} hbm_gbs", "alg_bytes": served_bytes,
        "alg_bytes_basis": "per request nnz*(8*4+4) + vector once (FP32) + nnz_out*(8*3+8)",
        "note": "the offered arrival rate, not the GPU, bounds this stream's rate"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serve_cpu_baseline(acc_sample, g)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_cpu_baseline(sample, g, target_s: float = 10.0):
    """The oracle, as it stands, on requests against the sampled resident
    tensors (their FP32-rounded values), until about target_s seconds of one
    core have run."""
    import oracle
    oracle.build()
    nnz, t_all, calls = 0, 0.0, 0
    host = [(sb.cpu().numpy(), v64.float().double().cpu().numpy(), shp) for sb, v64, shp, _ in sample]
    while host and t_all < target_s:
        for subs, vals, shp in host:
            m = int(g.integers(0, 4))
            x = g.uniform(-1, 1, shp[m]).astype(np.float32).astype(np.float64)
            t0 = time.perf_counter()
            oracle.ttv(subs, vals, shp, [m], [x], dense=False)
            t_all += time.perf_counter() - t0
            nnz += vals.shape[0]
            calls += 1
            if t_all >= target_s:
                break
    return {"value": nnz / max(t_all, 1e-9) / 1e9, "unit": "GNNZ/s", "cores": 1, "kind": "oracle",
            "sample": f"{calls} requests against {len(host)} resident tensors of at most 2e6 nonzeros, "
                      f"{nnz} nonzeros, {t_all:.1f} s"}


# FP64 multiply rate used as the MTTKRP roofline: the nominal FP64 rate of
# 1.25 TFLOP/s counts a fused multiply-add as two flops, and a multiply
# issues at the fused multiply-add rate, so 625 G multiplies/s.
FP64_MUL_NOMINAL_G = 625.0


def mttkrp_workload(problem):
    """Output mode of the MTTKRP timed on a TTV workload: the surviving mode
    of the all-but-one TTV, the contracted mode of the single TTV."""
    d = problem.tensor.d
    surv = [m for m in range(d) if m not in problem.modes]
    mode = surv[0] if len(surv) == 1 else problem.modes[0]
    return mode, [m for m in range(d) if m != mode]


def run_mttkrp(args, rank, world, local_rank):
    """MTTKRP of rank R, M(i,:) = sum of vals[k] * Hadamard product of the
    factor rows A_m(subs[k,m], :) over the other modes, on the tensor prepared
    once (untimed) for every mode but the output one; factors U[0,1)."""
    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = init_ranks(world, dev)
    ttv.load()
    wl = WORKLOADS[args.workload]
    if wl["make"] is None:
        raise SystemExit("--mttkrp applies to the single-tensor workloads")
    R = int(args.mttkrp)
    problem = wl["make"](dev, replica_seed(args.seed, rank), args.nnz)
    t = problem.tensor
    mode, others = mttkrp_workload(problem)
    subs = t.subs.t().contiguous().t()
    t_prep = time.perf_counter()
    prep = ttv.Prepared(subs, t.vals, t.shape, others)
    torch.cuda.synchronize(dev)
    t_prep = time.perf_counter() - t_prep
    g = torch.Generator(device=dev).manual_seed(replica_seed(args.seed, rank) + 77)
    fd = [torch.rand((t.shape[m], R), dtype=torch.float64, device=dev, generator=g) for m in others]
    out = torch.empty((t.shape[mode], R), dtype=torch.float64, device=dev)
    nb = ctypes.c_size_t()
    prep._lib.ttv_mttkrp_workspace_size(prep._h, R, ctypes.byref(nb))
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    def step():
        prep.mttkrp(fd, out=out, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    profiler_prewarm(ttv, step, args.steps)

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ttv.profile_reset()
    barrier(dist)
    torch.cuda.synchronize(dev)
    launches0 = ttv.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        profiled(ttv, i, step)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    launches = ttv.launch_count() - launches0
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1), dev)
    ttv.profile_collect()
    clk = clocks.stop()
    nnz, n_v = t.nnz, len(others)
    per_kernel = {}
    for name in ttv.profile_names():
        tot, n = ttv.profile_get(name)
        per_kernel[name] = {"ms_total": tot, "launches": n, "ms_avg": tot / max(1, n)}
    dom_ms = per_kernel.get("mttkrp_chunks", {}).get("ms_avg")
    muls = float(nnz) * R * n_v                     # factor products: n_v multiplies per nonzero and rank
    achieved = muls / (dom_ms * 1e-3) / 1e9 if dom_ms else None
    ms_step = ms / args.steps
    line = {
        "metric": "MTTKRP nonzeros/sec", "value": nnz * args.steps * world / (ms * 1e-3) / 1e9, "unit": "GNNZ/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"mttkrp_{args.workload}", "desc": wl["desc"], "rank": R, "mode": mode,
                   "nnz": nnz, "rows": int(t.shape[mode]), "factors": "U[0,1) float64, row-major (shape[m], R)",
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "kernel": "mttkrp_chunks", "achieved": achieved, "peak": FP64_MUL_NOMINAL_G,
                     "unit": "G FP64 mul/s", "frac": achieved / FP64_MUL_NOMINAL_G if achieved else None,
                     "traffic": None, "peak_source": "nominal FP64 1.25 TFLOP/s, fused multiply-add = 2 flops",
                     "mul_per_launch": muls},
        "step": {"gflops_f64": 2.0 * nnz * R * n_v / (ms_step * 1e-3) / 1e9},
        "prepared": {"prepare_s": round(t_prep, 3), "device_bytes": prep.device_bytes},
        "kernels": per_kernel, "gpu_launches": launches, "clocks": clk,
    }
    # end to end: host factors in, host result out, on the resident tensor
    h_f = [f.cpu().pin_memory() for f in fd]
    h_out = torch.empty(out.shape, dtype=torch.float64).pin_memory()
    times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for a, b in zip(fd, h_f):
            a.copy_(b, non_blocking=True)
        prep.mttkrp(fd, out=out, workspace=ws, stream=stream)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
        if i > 0:
            times.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(dist, sum(times) / len(times) * 1e3, dev)
    line["e2e"] = {"value": nnz * world / (e2e_ms * 1e-3) / 1e9, "unit": "GNNZ/s",
                   "h2d_bytes_per_step": int(sum(f.numel() * 8 for f in h_f)),
                   "d2h_bytes_per_step": int(h_out.numel() * 8), "ms_per_step": e2e_ms,
                   "note": "resident prepared tensor; factors copied in and the result read back each step"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        hs, hv = t.subs.cpu().numpy(), t.vals.cpu().numpy()
        hfac = [None] * t.d
        for m, f in zip(others, h_f):
            hfac[m] = f.numpy()
        hfac[mode] = np.zeros((t.shape[mode], R))
        m = min(nnz, 100_000)
        t0 = time.perf_counter()
        oracle.mttkrp(hs[:m], hv[:m], t.shape, mode, hfac)
        dt = time.perf_counter() - t0
        m2 = int(min(nnz, max(m, m * 10.0 / max(dt, 1e-6))))
        t0 = time.perf_counter()
        oracle.mttkrp(hs[:m2], hv[:m2], t.shape, mode, hfac)
        dt2 = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m2 / dt2 / 1e9, "unit": "GNNZ/s", "cores": 1, "kind": "oracle",
                                "sample": f"first {m2} of {nnz} nonzeros, rank {R}, one call, {dt2:.1f} s"}
    prep.close()
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_dense(args, rank, world, local_rank):
    """The paper's two simple kernels: one ttv_dot (1e8 elements) or one
    ttv_matvec (10000 x 10000) per step through the C ABI, operands resident;
    elements/s with the HBM roofline of the kernel."""
    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = init_ranks(world, dev)
    lib = ttv._declare_dense(ttv.load())
    seed = replica_seed(args.seed, rank)
    stream = torch.cuda.current_stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    if args.workload == "dot_1e8":
        n = args.nnz or 100_000_000
        x = S.uniform(seed, 1, n, device=dev)
        y = S.uniform(seed, 2, n, device=dev)
        out = torch.empty(1, dtype=torch.float64, device=dev)
        ws = torch.empty(max(1, ttv.dot_workspace_size(n)), dtype=torch.uint8, device=dev)
        elems, alg_bytes = n, 16 * n + 8
        kernel = "dot"

        def call():
            rc = lib.ttv_dot(x.data_ptr(), y.data_ptr(), n, 0, out.data_ptr(), ws.data_ptr(), ws.numel(), sh)
            if rc:
                raise ttv.TTVError(rc, lib.ttv_last_error().decode())
        host_in = [x, y]
        res = out
        cfg = {"n": n}
    else:
        n1 = n2 = 10_000
        A = S.uniform(seed, 1, n1 * n2, device=dev).reshape(n1, n2)
        if args.order == "F":
            A = A.t().contiguous().t()
        x = S.uniform(seed, 2, n2, device=dev)
        out = torch.empty(n1, dtype=torch.float64, device=dev)
        ws = torch.empty(max(1, ttv.matvec_workspace_size(A)), dtype=torch.uint8, device=dev)
        elems, alg_bytes = n1 * n2, 8 * n1 * n2 + 8 * n2 + 8 * n1
        kernel = "matvec"
        sr, sc = A.stride(0), A.stride(1)

        def call():
            rc = lib.ttv_matvec(A.data_ptr(), n1, n2, sr, sc, 0, x.data_ptr(), out.data_ptr(), ws.data_ptr(),
                                ws.numel(), sh)
            if rc:
                raise ttv.TTVError(rc, lib.ttv_last_error().decode())
        host_in = [A, x]
        res = out
        cfg = {"n1": n1, "n2": n2, "order": args.order}
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize(dev)
    profiler_prewarm(ttv, call, args.steps)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    ttv.profile_reset()
    barrier(dist)
    torch.cuda.synchronize(dev)
    launches0 = ttv.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        profiled(ttv, i, call)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    launches = ttv.launch_count() - launches0
    ms = max_over_ranks(dist, ev0.elapsed_time(ev1), dev)
    ttv.profile_collect()
    clk = clocks.stop()
    per_kernel = {}
    for name in ttv.profile_names():
        tot, cnt = ttv.profile_get(name)
        per_kernel[name] = {"ms_total": tot, "launches": cnt, "ms_avg": tot / max(1, cnt)}
    peaks, peak_src = load_peaks()
    peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    dom_ms = per_kernel.get(kernel, {}).get("ms_avg")
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms else None
    ms_step = ms / args.steps
    line = {
        "metric": "dense elements/sec", "value": elems * args.steps * world / (ms * 1e-3) / 1e9, "unit": "Gelem/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload=args.workload, desc=WORKLOADS[args.workload]["desc"],
                       l2="inputs larger than L2 (no flush)",
                       parallelism=f"{world} independent replicas" if world > 1 else "1 GPU", **cfg),
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "peak_source": f"{peak_src} hbm_gbs", "alg_bytes_per_launch": alg_bytes,
                     "fp64_fma_cap_gbs": (16.0 if kernel == "dot" else 8.0) * FP64_MUL_NOMINAL_G},
        "kernels": per_kernel, "gpu_launches": launches, "clocks": clk,
    }
    # end to end: operands copied in from pinned host memory, the result read back
    h_in = [t.cpu().pin_memory() for t in host_in]
    d_in = [torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=dev) for t in host_in]
    h_out = torch.empty(res.shape, dtype=torch.float64).pin_memory()
    times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for a, b in zip(d_in, h_in):
            a.copy_(b, non_blocking=True)
        if kernel == "dot":
            ttv.dot(d_in[0], d_in[1], out=out, workspace=ws, stream=stream)
        else:
            ttv.matvec(d_in[0], d_in[1], out=out, workspace=ws, stream=stream)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.synchronize(dev)
        if i > 0:
            times.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(dist, sum(times) / len(times) * 1e3, dev)
    line["e2e"] = {"value": elems * world / (e2e_ms * 1e-3) / 1e9, "unit": "Gelem/s",
                   "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in h_in)),
                   "d2h_bytes_per_step": int(h_out.numel() * 8), "ms_per_step": e2e_ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        if kernel == "dot":
            m = min(n, 20_000_000)
            xs, ys = h_in[0][:m].numpy(), h_in[1][:m].numpy()
            t0 = time.perf_counter()
            oracle.dot(xs, ys)
            dt = time.perf_counter() - t0
            sample = f"first {m} of {n} elements, one call, {dt:.2f} s"
        else:
            rows = 2000
            Ah = h_in[0][:rows].numpy()
            t0 = time.perf_counter()
            oracle.matvec(Ah, h_in[1].numpy())
            dt = time.perf_counter() - t0
            m = rows * 10_000
            sample = f"first {rows} of 10000 rows ({args.order} order), one call, {dt:.2f} s"
        line["cpu_baseline"] = {"value": m / dt / 1e9, "unit": "Gelem/s", "cores": 1, "kind": "oracle",
                                "sample": sample}
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_paper_sweep(args, rank, world, local_rank):
    """The paper's own TTV experiment on the GPU: for n = 100..1200 one TTV of
    an n^3 tensor with 0.01 n^3 distinct nonzeros along the second mode
    (sparse n x n result), timed with CUDA events over --steps calls of the C
    ABI after --warmup; the line's value is the n = 1200 rate."""
    import paper_2510_01495_gb300 as ttv
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = init_ranks(world, dev)
    ttv.load()
    steps = min(args.steps, 200)
    rows = []
    clocks = ClockSampler(local_rank)
    clocks.start()
    for n in range(100, 1300, 100):
        p = S.paper_sweep(n, seed=replica_seed(args.seed, rank), device=dev)
        t = p.tensor
        subs = t.subs.t().contiguous().t()
        ws = torch.empty(max(1, ttv.workspace_size(subs, t.vals, t.shape, p.modes)), dtype=torch.uint8, device=dev)
        nrow, nval = ttv.out_capacity(subs, t.vals, t.shape, p.modes)
        ov = torch.empty(nval, dtype=torch.float64, device=dev)
        osb = torch.empty((max(1, nrow), 2), dtype=torch.int64, device=dev)

        def call():
            return ttv.ttv_multi(subs, t.vals, t.shape, p.modes, p.vecs, workspace=ws, out_vals=ov, out_subs=osb)
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize(dev)
        barrier(dist)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            r = call()
        ev1.record()
        torch.cuda.synchronize(dev)
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1) / steps, dev)
        rows.append({"n": n, "nnz": t.nnz, "nnz_out": int(r.vals.numel()), "ms": ms,
                     "gnnz_s": t.nnz * world / (ms * 1e-3) / 1e9})
        del p, t, subs, ws, ov, osb
    clk = clocks.stop()
    last = rows[-1]
    line = {
        "metric": "TTV nonzeros/sec", "value": last["gnnz_s"], "unit": "GNNZ/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": last["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "paper_sweep", "desc": WORKLOADS["paper_sweep"]["desc"],
                   "timing": "CUDA events around --steps synchronous ttv_multi calls (result size read each call)",
                   "l2": "inputs up to 553 MB; the small sizes are L2-resident"},
        "sweep": rows, "clocks": clk,
    }
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(ttv, problem, subs, vals, vecs, fmt, args, dev):
    """Same metric through ttv_multi with HOST inputs: pinned host -> device
    copies of subs, vals and vectors, the call, and the result read back, all
    inside the timed region."""
    store = subs.t().contiguous() if args.layout == "soa" else subs.contiguous()
    h_store = store.cpu().pin_memory()
    del store
    h_vals = vals.cpu().pin_memory()
    h_vecs = [v.cpu().pin_memory() for v in vecs]
    d_subs_store = torch.empty_like(h_store, device=dev)
    d_vals = torch.empty_like(h_vals, device=dev)
    d_vecs = [torch.empty_like(v, device=dev) for v in h_vecs]
    h2d = (d_subs_store.numel() * 8 + d_vals.numel() * d_vals.element_size() +
           sum(v.numel() * v.element_size() for v in h_vecs))
    d2h = 0
    times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        d_subs_store.copy_(h_store, non_blocking=True)
        d_vals.copy_(h_vals, non_blocking=True)
        for a, b in zip(d_vecs, h_vecs):
            a.copy_(b, non_blocking=True)
        ds = d_subs_store.t() if args.layout == "soa" else d_subs_store
        r = ttv.ttv_multi(ds, d_vals, problem.tensor.shape, problem.modes, d_vecs, fmt=fmt, path=args.path)
        hv = r.vals.cpu()
        hs = r.subs.cpu() if r.subs is not None else None
        torch.cuda.synchronize(dev)
        if i > 0:
            times.append(time.perf_counter() - t0)
        d2h = hv.numel() * 8 + (hs.numel() * 8 if hs is not None else 0)
    mean = sum(times) / len(times)
    return {"value": problem.tensor.nnz / mean / 1e9, "unit": "GNNZ/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": mean * 1e3, "steps": len(times)}


if __name__ == "__main__":
    main()
