"""Benchmark of one Lloyd pass of LBG on image-block data (one GB300 per rank).

Workload (default ``img2048x8_b8_n4096``): eight seeded synthetic 2048x2048
8-bit images cut into 8x8 blocks -> X [524288 x 64] float32, codebook grown by
splitting to N = 4096 (delta = 0.01, theta = 1e-3).

A *step* is one Lloyd pass through the C ABI (``lbg_lloyd_step``): cell
allocation of all M rows against the trained N = 4096 codebook, integration
of the distortion, cell table and centroid update -- every kernel of the hot
path.  ``value`` = M * N distance evaluations / device time per step, the
steps enqueued back to back (the call's asynchronous form: its graph is
replayed and D, n_exact and the status land in a device buffer).
``phase_ms`` and the roofline's kernel time come from as many directly
launched steps right after the timed ones (per-phase CUDA events).

Other legs in the same run:
* full LBG design time (``lbg_train`` from the centroid to N = 4096);
* ``e2e``: the same step through the C ABI with HOST buffers (pinned), the
  host->device copy of X and C and the device->host read of C, the cell
  table and D inside the timed region;
* ``roofline``: the nearest-codevector kernel of the timed precision,
  algorithmic work 2*L*M*N flop per launch over its CUDA-event time, against
  the measured BF16 tensor peak (burst) for the BF16 form (default) or, for
  the FP32 form, the FP32 FMA peak measured in this run by the library's
  FFMA kernel (``fp32_peak``, with the device's SM count); ``traffic`` = the
  ncu DRAM bytes per launch recorded under profiles/ while the kernel
  sources keep the digest recorded there;
* ``update_roofline``: cell table and update, algorithmic bytes over their
  time, against the measured HBM copy peak;
* ``other_precision`` (the other form's step and full LBG), ``step_after_split``
  (the step against the codebook right after the last split, the least
  converged one of the design), ``differentiation`` (with the FP64 oracle's
  full LBG on the same Gaussian-mixture data), ``batched``, ``small_full_lbg``
  (with the pass-by-pass comparison of each precision's design with the
  oracle) and ``large`` (64 images, 4x4 blocks: LBG on 16.8M vectors and
  encode of 16.8M more, with the oracle's sampled encode rate);
* ``cpu_baseline``: the FP64 oracle's Lloyd pass on a bounded row sample on
  the host cores.
``ms_per_step`` is the median of the timed steps; ``gpu_launches`` is the
library's own count of the kernels it launched in the timed region.
``--impl reference`` times only the oracle (the baseline arm).
With ``--gpus N`` (under torchrun) every rank runs an independent replica.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vector·codevector distance evals/s per Lloyd pass; full LBG time, bf16 vs fp32"
UNIT = "evals/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="img2048x8_b8_n4096")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"],
                    help="form timed for the headline value (the other is timed beside it)")
    ap.add_argument("--fp32-steps", type=int, default=3,
                    help="timed steps of the other form (0: skip it)")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the differentiation leg (GMM, M=262144, L=32, N=512)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched leg (64 ragged problems, L=16)")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the full-LBG timing of the 512x512 image workload")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 64-image leg: LBG to N=4096 on 16.7M vectors + encode of 16.7M more")
    ap.add_argument("--no-after-split", action="store_true",
                    help="skip the step against the codebook right after the last split")
    return ap.parse_args()


def workload_desc(name, X, N):
    w = {"img2048x8_b8_n4096": "8 synthetic 2048x2048 8-bit images, 8x8 blocks",
         "img512_b4_n256": "1 synthetic 512x512 8-bit image, 4x4 blocks",
         "img2048x64_b4_n4096": "64 synthetic 2048x2048 8-bit images, 4x4 blocks"}[name]
    return f"{name}: {w}, M={X.shape[0]}, L={X.shape[1]}, N={N}, delta=0.01, theta=1e-3"


# ------------------------------------------------------------------ measured traffic
# DRAM bytes per launch of the roofline kernel come from a committed ncu summary
# (profiles/), valid only while the kernel's sources are unchanged since that
# capture: the summary records a digest of them.
TRAFFIC = {("bf16", "img2048x8_b8_n4096"): ("k_assign_tc_img2048x8_b8_n4096_full.md",
                                             ("k_assign_tc.cu", "lbg_internal.cuh"))}


def source_digest(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_0910_4711_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(precision, workload):
    """(bytes per launch or None, summary file, current source digest)."""
    import re
    entry = TRAFFIC.get((precision, workload))
    if entry is None:
        return None, None, None
    summary, files = entry
    digest = source_digest(files)
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None, summary, digest
    m_d = re.search(r"source digest: `([0-9a-f]+)`", text)
    m_b = re.search(r"dram bytes per launch: `([0-9,]+)`", text)
    if m_d and m_b and m_d.group(1) == digest:
        return int(m_b.group(1).replace(",", "")), summary, digest
    return None, summary, digest


# ------------------------------------------------------------------ distributed
def dist_setup(n, backend="nccl"):
    """Join the process group torchrun set up (one replica per GPU); (0, 1, None) alone."""
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    if backend == "nccl":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    dist.init_process_group(backend)
    return rank, world, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job rate of `world` replicas that each process `units_per_rank` units, timed by the
    slowest rank (`seconds` is already the max over ranks)."""
    return world * units_per_rank / seconds


SLOWDOWNS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clocks):
    """True when the clock record of a timed region shows a hardware or thermal
    slowdown (a number taken then is re-measured once; sw_power_cap is kept)."""
    return any(r in SLOWDOWNS for r in (clocks or {}).get("reasons") or [])


def estimated_full_lbg_s(passes_per_stage, M, evals_per_s):
    """Estimated time of a whole LBG design on the CPU oracle: stage s (codebook
    size 2**s) ran passes_per_stage[s] passes, each costing M * 2**s distance
    evaluations at the oracle's measured rate.  An estimate (the oracle's full
    design at this size would take hours): the update's share, which does not
    grow with the codebook size, is not counted."""
    n, total = 1, 0.0
    for p in passes_per_stage:
        total += p * M * n / evals_per_s
        n *= 2
    return total


# ------------------------------------------------------------------ clocks
def gpu_uuid(dev):
    """nvidia-smi id of the CUDA device `dev` (its UUID; the box may list other GPUs)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


class NvmlClocks:
    """Reads SM clock, max SM clock, power and clock-event reasons of one GPU
    through NVML's public C API (libnvidia-ml, shipped with the driver).  Read
    only: nothing here changes a GPU setting."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, uuid):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle for " + uuid)
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        ct = self.ct
        sm, mx, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(sm))        # NVML_CLOCK_SM
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx))
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
        self.reasons_fn(self.h, ct.byref(rs))
        return sm.value, mx.value, mw.value / 1e3, rs.value

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """Samples the GPU's clocks while the timed region runs: NVML from a thread
    every ~2 ms (so a region of a few ms still gets samples), else nvidia-smi
    at its 200 ms minimum interval."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_uuid):
        self.gpu = gpu_uuid
        self.p = None
        self.nvml = None
        self.rows = []
        self.source = None

    def _loop(self):
        while not self.stop:
            try:
                self.rows.append(self.nvml.sample())
            except Exception:
                return
            time.sleep(0.002)

    def __enter__(self):
        import threading
        try:
            self.nvml = NvmlClocks(self.gpu)
            self.stop = False
            self.rows.append(self.nvml.sample())
            self.th = threading.Thread(target=self._loop, daemon=True)
            self.th.start()
            self.source = "nvml"
            return self
        except Exception:
            self.nvml = None
        self.path = tempfile.mktemp(suffix=".csv")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}",
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi"
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.nvml is not None:
            self.stop = True
            self.th.join(timeout=5)
            try:
                self.rows.append(self.nvml.sample())
                self.nvml.close()
            except Exception:
                pass
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.nvml is not None:
            if not self.rows:
                return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
            reasons = sorted({name for r in self.rows for bit, name in NvmlClocks.REASONS.items()
                              if r[3] & bit})
            return {"sm_mhz": statistics.median(r[0] for r in self.rows),
                    "sm_max_mhz": max(r[1] for r in self.rows),
                    "power_w_median": statistics.median(r[2] for r in self.rows),
                    "samples": len(self.rows), "source": "nvml", "reasons": reasons}
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1].split()[0]), float(parts[2].split()[0]),
                             parts[5], parts[6], parts[7], parts[8], parts[3]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "source": "nvidia-smi", "reasons": reasons}


# ------------------------------------------------------------------ cpu baseline
def cpu_baseline(X, C, seconds, seed=0):
    """FP64 oracle Lloyd pass (allocation + distortion + updation) on a row
    sample of X against C, on all host cores; sample grown to ~`seconds`."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    Cd = np.asarray(C, np.float64)
    # calibrate on 1024 rows, then time one sample sized to take ~`seconds`
    S = np.ascontiguousarray(X[np.sort(rng.choice(X.shape[0], min(1024, X.shape[0]), replace=False))])
    t0 = time.perf_counter()
    oracle.lloyd_step(S, Cd)
    t1 = time.perf_counter() - t0
    rows = int(min(X.shape[0], max(1024, 1024 * seconds / max(t1, 1e-4))))
    idx = np.sort(rng.choice(X.shape[0], rows, replace=False))
    S = np.ascontiguousarray(X[idx])
    t0 = time.perf_counter()
    oracle.lloyd_step(S, Cd)
    t = time.perf_counter() - t0
    evals = S.shape[0] * Cd.shape[0]
    # the same pass on one host thread, on 1/16 of that sample
    S1 = S[: max(256, S.shape[0] // 16)]
    t0 = time.perf_counter()
    oracle.lloyd_step(S1, Cd, nthreads=1)
    t_1 = time.perf_counter() - t0
    return {"value": evals / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "seconds": t, "value_1thread": S1.shape[0] * Cd.shape[0] / t_1,
            "sample": (f"one FP64 oracle Lloyd pass (allocation, distortion, updation) over "
                       f"{S.shape[0]} random rows of the same X against the same N={Cd.shape[0]} "
                       f"codebook on all host threads (OpenMP static row split); value_1thread: "
                       f"the first {S1.shape[0]} of those rows on one thread")}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_0910_4711_gb300 import synth
    import oracle
    oracle.build()
    X, N = synth.workload(args.workload)
    rng = np.random.default_rng(7)
    C = X[rng.choice(X.shape[0], N, replace=False)].astype(np.float64)
    # size each step's row sample so one step takes ~ a few seconds
    rows = 256
    while True:
        S = X[:rows]
        t0 = time.perf_counter()
        oracle.lloyd_step(S, C)
        t = time.perf_counter() - t0
        if t > 1.0 or rows >= 65536:
            break
        rows *= 2
    for _ in range(args.warmup):
        oracle.lloyd_step(X[:rows], C)
    times = []
    for k in range(args.steps):
        lo = (k * rows) % max(1, X.shape[0] - rows)
        S = np.ascontiguousarray(X[lo:lo + rows])
        t0 = time.perf_counter()
        oracle.lloyd_step(S, C)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = rows * N / (ms / 1e3)
    sample = (f"each step: one FP64 oracle Lloyd pass over {rows} consecutive rows of X against an "
              f"N={N} codebook of seeded rows of X (a trained codebook needs the GPU)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, X, N), "M": int(X.shape[0]),
                       "L": int(X.shape[1]), "N": int(N), "rows_per_step": rows,
                       "codebook": f"N={N} seeded rows of X (untrained: the trained codebook needs the GPU)",
                       "sample": "each step is one Lloyd pass over rows_per_step consecutive rows of X "
                                 "(a bounded sample of the workload; value scales it to M*N evals/s)"},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.max_threads(), "sample": sample,
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, world, dist = dist_setup(args.gpus)
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    dev = torch.cuda.current_device()
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4711_gb300 as lbg
    from paper_0910_4711_gb300 import synth

    X_np, N = synth.workload(args.workload)
    M, L = X_np.shape
    # inputs of the 64-image leg, generated on the host cores in worker processes started
    # now, before the first GPU call (their pool is spawned, never forked)
    large_future = None if args.no_large else start_large_inputs()
    X = torch.from_numpy(X_np).cuda()
    stream = torch.cuda.current_stream()
    # the FP32 FMA peak of this device, measured (the FP32 form's roofline denominator)
    fp32_tflops, n_sms = lbg.measure_fp32_peak(stream.cuda_stream)

    # full LBG design in both forms (the headline form's codebook is the one
    # the timed steps run against)
    other = "fp32" if args.precision == "bf16" else "bf16"
    precs = [other, args.precision] if args.fp32_steps > 0 else [args.precision]
    for prec in precs:   # untimed: workspace allocation and first launches
        lbg.lbg_train(X, N, delta=0.01, theta=1e-3, max_passes=1, precision=prec)
    trains = {}
    for prec in precs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr = lbg.lbg_train(X, N, delta=0.01, theta=1e-3, trace=100000, precision=prec)
        torch.cuda.synchronize()
        trains[prec] = (time.perf_counter() - t0, tr)
    full_lbg_s, tr = trains[args.precision]
    C = tr.C.clone()
    C_out = torch.empty_like(C)
    A = torch.empty(M, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def timed_steps(prec, steps, clocks=None):
        """`steps` passes enqueued back to back (replayed graphs, each reporting
        D / n_exact / status into a device buffer, no host wait in between), L2
        flushed before each; then as many directly launched passes with
        per-phase CUDA events (same inputs, same flush) for the phase breakdown
        and the nearest-codevector kernel's time."""
        buf = lbg.step_result_buffer()
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            lbg.lbg_lloyd_step(X, C, C_out=C_out, assign_out=A, precision=prec, result_out=buf)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier(dist)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_steps")
        l0 = lbg.launch_count()
        w0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            lbg.lbg_lloyd_step(X, C, C_out=C_out, assign_out=A, precision=prec, result_out=buf)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        launches = lbg.launch_count() - l0
        torch.cuda.nvtx.range_pop()
        barrier(dist)
        per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms = max_over_ranks(dist, statistics.median(per))
        ms_mean = max_over_ranks(dist, statistics.mean(per))
        _, n_exact, status = lbg.read_step_result(buf)
        if status != 0:
            raise RuntimeError(f"device status {status} in the timed passes")
        phases = []
        for _ in range(steps):
            flush.zero_()
            phases.append(lbg.lbg_lloyd_step(X, C, C_out=C_out, assign_out=A, phase_ms=True,
                                             precision=prec).phase_ms)
        ph = {k: statistics.median(p[k] for p in phases)
              for k in ("prep", "assign", "exact", "update", "total")}
        return {"ms": ms, "ms_mean": ms_mean, "ph": ph, "n_exact": n_exact, "wall": wall,
                "launches": launches, "per_step_ms": per}

    with ClockSampler(gpu_uuid(dev)) as clk:
        t = timed_steps(args.precision, args.steps)
    clocks = clk.summary()
    # a slowdown on any rank: every rank times the steps once more (same barriers)
    if max_over_ranks(dist, 1.0 if throttled(clocks) else 0.0) > 0:
        first = clocks
        with ClockSampler(gpu_uuid(dev)) as clk:
            t = timed_steps(args.precision, args.steps)
        clocks = clk.summary()
        clocks["remeasured_after"] = first.get("reasons")
    ms, ph, n_exact, wall = t["ms"], t["ph"], t["n_exact"], t["wall"]
    value = job_throughput(world, M * N, ms / 1e3)
    other_line = None
    if args.fp32_steps > 0:
        ot = timed_steps(other, args.fp32_steps)
        o_ms, o_ph, o_ex = ot["ms"], ot["ph"], ot["n_exact"]
        o_train_s, o_tr = trains[other]
        other_line = {"precision": other, "value": job_throughput(world, M * N, o_ms / 1e3), "unit": UNIT,
                      "ms_per_step": o_ms, "phase_ms": o_ph, "exact_rows_per_step": o_ex,
                      "full_lbg_s": o_train_s, "full_lbg_passes": o_tr.n_passes,
                      "full_lbg_D": o_tr.D}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    # without the measured file: the fallback peaks of an earlier GB300 measurement
    of = "of measured" if peaks else "of fallback (MEASURED_PEAKS.json absent)"
    fp32_peak = fp32_tflops                                   # measured in this run
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    flops = 2.0 * L * M * N          # algorithmic: L FMA per distance evaluation
    assign_ms = ph["assign"]
    achieved = flops / (assign_ms / 1e3) / 1e12
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    upd_bytes = M * L * 4 + M * 4 + N * L * 4 + N * 4
    upd_gbs = upd_bytes / (ph["update"] / 1e3) / 1e9
    traffic, t_summary, t_digest = measured_traffic(args.precision, args.workload)
    if args.precision == "bf16":
        Lk = (L + 15) // 16 * 16
        Nt = (N + 143) // 144 * 144      # whole 144-codevector tiles
        executed = 2.0 * M * Nt * (2 * Lk + 16) / (assign_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "kernel": "k_assign_tc", "achieved": achieved, "peak": bf16_peak,
                "unit": "TFLOP/s", "frac": achieved / bf16_peak, "traffic": traffic,
                "traffic_source": (f"profiles/{t_summary} (ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                   f"per launch; kernel source digest {t_digest})"
                                   if traffic is not None else
                                   f"null: no capture of the current kernel sources (digest {t_digest})"),
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops (burst), {of}",
                "work": "2*L*M*N flop per launch (algorithmic; the two-piece BF16 split of the codevectors, "
                        "the norm column and whole 144-codevector tiles make the tensor cores execute "
                        "2*M*ceil144(N)*(2*ceil16(L)+16))",
                "executed_tflops": executed, "executed_frac": executed / bf16_peak,
                "epilogue_bound": {"ops_per_distance": 5, "peak_tops": fp32_peak / 2,
                                   "bound_ms": 5.0 * M * N / (fp32_peak / 2 * 1e12) * 1e3}}
    else:
        roof = {"bound": "alu", "kernel": "k_assign_f32", "achieved": achieved, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                "peak_source": f"FP32 FMA peak measured in this run (lbg_measure_fp32_peak, {n_sms} SMs)",
                "work": "2*L*M*N flop per launch"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_mean": t["ms_mean"],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, X_np, N), "M": M, "L": L, "N": N,
                       "precision": args.precision + (" (BF16 tensor-core distances, FP32 accumulation, "
                                                      "certified or exact FP32 re-scoring)"
                                                      if args.precision == "bf16" else " (FFMA)"),
                       "step": "one Lloyd pass (lbg_lloyd_step) against the trained N-entry codebook",
                       "l2": f"flushed: {L2_FLUSH_BYTES >> 20} MiB device write between steps",
                       "full_lbg_s": full_lbg_s, "full_lbg_passes": tr.n_passes,
                       "full_lbg_passes_per_stage": tr.passes_per_stage(),
                       "full_lbg_D": tr.D, "exact_rows_per_step": n_exact,
                       "phase_ms": ph, "wall_s_timed_region": wall,
                       "timing": "median of the timed steps' CUDA-event times (ms_per_step_mean: their mean)",
                       "data_sha256": synth.digest(X_np)[:16],
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "update_roofline": {"bound": "hbm", "achieved": upd_gbs, "peak": hbm, "unit": "GB/s",
                                "frac": upd_gbs / hbm, "bytes": upd_bytes,
                                "work": "M*L*4 + M*4 + N*L*4 + N*4 bytes (read X, cell table; "
                                        "write codebook, counts)",
                                "peak_source": f"MEASURED_PEAKS.json hbm_gbs, {of}"},
            "clocks": clocks,
            "fp32_peak": {"tflops": fp32_tflops, "sms": n_sms,
                          "how": "lbg_measure_fp32_peak: independent FFMA chains on every SM, CUDA events"},
            "gpu_launches": t["launches"],
            "gpu_launches_source": "lbg_launch_count() difference over the timed region (kernels of "
                                   "replayed graphs included)"}
    if other_line is not None:
        line["other_precision"] = other_line
        if args.precision == "bf16":
            f_ach = flops / (o_ph["assign"] / 1e3) / 1e12
            other_line["roofline"] = {"bound": "alu", "kernel": "k_assign_f32", "achieved": f_ach,
                                      "peak": fp32_peak, "unit": "TFLOP/s", "frac": f_ach / fp32_peak,
                                      "peak_source": "FP32 FMA peak measured in this run"}
    if not args.no_after_split:
        try:
            line["step_after_split"] = after_split_leg(lbg, torch, X, N, args, flush, stream, dist)
        except Exception as exc:   # a report must never cost the measured line
            line["step_after_split"] = {"error": repr(exc)}

    # differentiation form: D(X, C) forward (nearest codevector) + backward at
    # the fixed cell table, on Gaussian-mixture vectors (M=262144, L=32, 512
    # components, sigma 0.1), codebook from LBG to N=512
    if not args.no_grad:
        line["differentiation"] = grad_leg(lbg, synth, torch, stream, flush, args, dist,
                                           with_oracle=not args.no_cpu_baseline)

    if not args.no_batched:
        line["batched"] = batched_leg(lbg, synth, torch)
    if not args.no_small:
        line["small_full_lbg"] = small_leg(lbg, synth, torch, with_oracle=not args.no_cpu_baseline)
    if large_future is not None:
        line["large"] = large_leg(lbg, synth, torch, large_future, with_oracle=not args.no_cpu_baseline)

    # end to end through the public API with host buffers
    if not args.no_e2e:
        Xh = torch.from_numpy(X_np).pin_memory()
        Ch = tr.C.cpu().pin_memory()
        Coh = torch.empty_like(Ch).pin_memory()
        Ah = torch.empty(M, dtype=torch.int32).pin_memory()
        for _ in range(2):
            lbg.lbg_lloyd_step(Xh, Ch, C_out=Coh, assign_out=Ah, precision=args.precision)
        times = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = lbg.lbg_lloyd_step(Xh, Ch, C_out=Coh, assign_out=Ah, precision=args.precision)
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(dist, statistics.mean(times))
        line["e2e"] = {"value": job_throughput(world, M * N, e2e_s), "unit": UNIT,
                       "h2d_bytes_per_step": M * L * 4 + N * L * 4,
                       "d2h_bytes_per_step": N * L * 4 + M * 4 + 8,
                       "ms_per_step": 1e3 * e2e_s}

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(X_np, tr.C.cpu().numpy(), args.cpu_seconds)
        try:
            cb = line["cpu_baseline"]
            cb["full_lbg_estimated_s"] = estimated_full_lbg_s(tr.passes_per_stage(), M, cb["value"])
            cb["full_lbg_estimate"] = ("estimated, not run: the GPU design's passes per stage x "
                                       "M x stage size evaluations at the oracle's measured rate")
        except Exception as exc:   # an estimate must never cost the measured line
            line["cpu_baseline"]["full_lbg_estimate"] = f"not computed: {exc!r}"
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def grad_leg(lbg, synth, torch, stream, flush, args, dist, with_oracle=True):
    Xg_np, _, _ = synth.gmm(4, 262144, L=32, K=512, sigma=0.1)
    Mg, Lg = Xg_np.shape
    Ng = 512
    Xg = torch.from_numpy(Xg_np).cuda()
    lbg.lbg_train(Xg, Ng, delta=0.01, theta=1e-3, max_passes=1)   # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr = lbg.lbg_train(Xg, Ng, delta=0.01, theta=1e-3)
    torch.cuda.synchronize()
    gpu_lbg_s = time.perf_counter() - t0
    Cg = tr.C
    idx = torch.empty(Mg, dtype=torch.int32, device="cuda")
    for _ in range(3):
        lbg.vq_encode(Xg, Cg, idx_out=idx)
        lbg.distortion_backward(Xg, Cg, idx)
    fw, bw, bwph = [], [], []
    for _ in range(max(3, args.steps)):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        lbg.vq_encode(Xg, Cg, idx_out=idx)
        e1.record(stream)
        D, dC, dX, ph = lbg.distortion_backward(Xg, Cg, idx, phase_ms=True)
        e2.record(stream)
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
        bw.append(e1.elapsed_time(e2))
    fwd = max_over_ranks(dist, statistics.median(fw))
    bwd = max_over_ranks(dist, statistics.median(bw))
    bytes_bwd = 3 * Mg * Lg * 4 + 2 * Mg * 4 + 2 * Ng * Lg * 4
    # the mixture's real values on the tensor cores (two BF16 pieces per x, L = 32) against
    # the FP32 form: enqueue-only encodes of the designed codebook, the same cells expected
    encode, ref_idx = {}, None
    buf = lbg.step_result_buffer()
    for prec in ("fp32", "bf16"):
        out_idx = torch.empty(Mg, dtype=torch.int32, device="cuda")
        for _ in range(3):
            lbg.vq_encode(Xg, Cg, idx_out=out_idx, precision=prec)
        ts = []
        for _ in range(max(3, args.steps)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lbg.vq_encode(Xg, Cg, idx_out=out_idx, precision=prec, result_out=buf)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        Dp, nex, status = lbg.read_step_result(buf)
        ms = max_over_ranks(dist, statistics.median(ts))
        encode[prec] = {"ms": ms, "evals_per_s": Mg * Ng / (ms / 1e3), "exact_rows": nex, "D": Dp,
                        "status": status}
        if ref_idx is None:
            ref_idx = out_idx.clone()
        else:
            encode[prec]["rows_differing_from_fp32"] = int((out_idx != ref_idx).sum().item())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trb = lbg.lbg_train(Xg, Ng, delta=0.01, theta=1e-3, precision="bf16")
    torch.cuda.synchronize()
    full = {"gpu_fp32_s": gpu_lbg_s, "gpu_passes": tr.n_passes, "gpu_D": tr.D,
            "gpu_bf16_s": time.perf_counter() - t0, "gpu_bf16_passes": trb.n_passes, "gpu_bf16_D": trb.D}
    if with_oracle:
        try:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            o = oracle.lbg_train(Xg_np, Ng, 0.01, 1e-3)
            full["oracle_s"] = time.perf_counter() - t0
            full["oracle_passes"] = int(len(o.trace_D))
            full["oracle_D"] = float(o.D)
            full["oracle_cores"] = oracle.max_threads()
            full["oracle_kind"] = "FP64 oracle LBG to N=512 on the same data, all host threads"
        except Exception as exc:   # a report must never cost the measured line
            full["oracle_error"] = repr(exc)
    return {"workload": "gmm262144_l32_n512: 262144 Gaussian-mixture vectors, L=32, 512 components "
                        "(sigma 0.1, means U[0,1]^32), codebook from LBG to N=512",
            "full_lbg": full,
            "encode": encode,
            "forward_ms": fwd, "backward_ms": bwd, "D": D,
            "backward_gbs": bytes_bwd / (bwd / 1e3) / 1e9,
            "backward_bytes": bytes_bwd,
            "backward_work": "read X twice (dX pass, cell sums), write dX, read the cell table twice, "
                             "read C, write dC: 3*M*L*4 + 2*M*4 + 2*N*L*4 bytes",
            "forward_evals_per_s": Mg * Ng / (fwd / 1e3)}


def small_leg(lbg, synth, torch, with_oracle=True):
    """Full LBG design on one 512x512 image, 4x4 blocks (M=16384, L=16, N=256)."""
    X_np, N = synth.workload("img512_b4_n256")
    X = torch.from_numpy(X_np).cuda()
    out = {"workload": workload_desc("img512_b4_n256", X_np, N)}
    runs = {}
    for prec in ("fp32", "bf16"):
        lbg.lbg_train(X, N, 0.01, 1e-3, precision=prec)   # warm
        ts = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = lbg.lbg_train(X, N, 0.01, 1e-3, precision=prec)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[prec] = {"full_lbg_ms": 1e3 * statistics.median(ts), "passes": r.n_passes, "D": r.D}
        runs[prec] = r
    if with_oracle:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        o = oracle.lbg_train(X_np, N, 0.01, 1e-3)
        out["oracle_full_lbg"] = {"seconds": time.perf_counter() - t0, "passes": int(len(o.trace_D)),
                                  "D": float(o.D), "cores": oracle.max_threads(),
                                  "kind": "FP64 oracle LBG on the host (same data, delta, theta)"}
        # whole-run comparison (meaningful when the oracle's run met no near-tie row), and
        # the pass-by-pass comparison: the oracle's step from every pass's own codebook
        try:
            from oracle import trajectory
            den = np.maximum(np.abs(o.C).max(1), 1.0)
            for prec, r in runs.items():
                Cg = r.C.cpu().numpy().astype(np.float64)
                out[prec]["vs_oracle"] = {
                    "near_tie_rows_in_oracle_run": o.near_ties(),
                    "same_passes_per_stage": r.passes_per_stage() == o.passes_per_stage(),
                    "D_rel_diff": abs(r.D - o.D) / o.D,
                    "codebook_max_rel_diff": float((np.abs(Cg - o.C).max(1) / den).max())}
                t = lbg.lbg_train(X, N, 0.01, 1e-3, precision=prec, trace=4096, trace_passes=4096)
                rep = trajectory.compare(X_np, N, 0.01, 1e-3, t.records, t.pass_C.cpu().numpy(),
                                         t.pass_assign.cpu().numpy(), t.C.cpu().numpy(),
                                         t.assign.cpu().numpy(), t.D)
                out[prec]["per_pass_vs_oracle"] = rep.summary()
                out[prec]["pass_ms_median"] = statistics.median(rec["ms"] for rec in t.records)
        except Exception as exc:   # a report must never cost the measured line
            out["vs_oracle_error"] = repr(exc)
    return out


def batched_leg(lbg, synth, torch):
    """64 ragged problems: M_s log-uniform in [4096, 262144], N_s in {64..1024}, L=16 (4x4
    blocks of each problem's own 2048x2048 image); the whole batched design vs one lbg_train
    per problem on the same GPU."""
    spec = synth.batched_sets(3000)
    parts = [synth.blocks(synth.make_image(seed, 2048, 2048), 4)[:M] for seed, M, _ in spec]
    Ns = [n for _, _, n in spec]
    row_off = np.concatenate([[0], np.cumsum([p.shape[0] for p in parts])])
    X = torch.from_numpy(np.concatenate(parts)).cuda()
    # warm: workspace, graph capture, and the tile autotuner's calibration of this bucket
    tune = lbg.lbg_train_batched(X, row_off, Ns, max_passes=1).tune
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lbg.lbg_train_batched(X, row_off, Ns)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    Xs = [X[row_off[s]:row_off[s + 1]] for s in range(len(Ns))]
    for s in range(len(Ns)):   # warm the single-problem path
        lbg.lbg_train(Xs[s], Ns[s], 0.01, 1e-3, max_passes=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_passes = 0
    for s in range(len(Ns)):
        seq_passes = max(seq_passes, lbg.lbg_train(Xs[s], Ns[s], 0.01, 1e-3).n_passes)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    bt = statistics.median(ts)
    # the same batch with one launch per phase of a pass (tuned tiles) instead of one
    # persistent launch per pass
    lbg.lbg_train_batched(X, row_off, Ns, max_passes=1, per_phase=True)
    tp = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp = lbg.lbg_train_batched(X, row_off, Ns, per_phase=True)
        torch.cuda.synchronize()
        tp.append(time.perf_counter() - t0)
    return {"workload": f"64 problems, sum M = {int(row_off[-1])}, L = 16, N in {{64..1024}}",
            "batched_s": bt, "sequential_s": seq, "speedup": seq / bt,
            "one_launch_per_pass": bool(r.tune.get("persistent")),
            "per_phase_launches_s": statistics.median(tp),
            "per_phase_tile": {"tile_rows": rp.tune["tile_rows"], "ctas_per_sm": rp.tune["ctas_per_sm"]},
            "max_passes": r.max_passes_run, "passes_per_s": r.max_passes_run / bt,
            "assign_tile": {"chosen": {"tile_rows": r.tune["tile_rows"], "ctas_per_sm": r.tune["ctas_per_sm"]},
                            "calibration": tune["candidates"]}}


def _large_part(seeds):
    from paper_0910_4711_gb300 import synth
    return synth.image_blocks(seeds, 2048, 2048, 4)


def start_large_inputs():
    """Start generating the 64-image leg's inputs (train seeds 5001..5064, encode seeds
    5101..5164) in spawned worker processes; returns a callable giving (X, Y)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    n = max(1, min(16, os.cpu_count() or 1))
    pool = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
    groups = [list(range(a, a + 4)) for a in range(5001, 5065, 4)] + \
             [list(range(a, a + 4)) for a in range(5101, 5165, 4)]
    futs = [pool.submit(_large_part, g) for g in groups]

    def result():
        parts = [f.result() for f in futs]
        pool.shutdown()
        return np.concatenate(parts[:16]), np.concatenate(parts[16:])
    return result


def large_leg(lbg, synth, torch, inputs, with_oracle=True):
    """64 2048x2048 images, 4x4 blocks: LBG to N=4096 on 16.7M vectors, then encode 16.7M more;
    BF16 vs FP32; beside it the FP64 oracle's encode rate on a row sample."""
    X_np, Y_np = inputs()
    N = 4096
    X = torch.from_numpy(X_np).cuda()
    Y = torch.from_numpy(Y_np).cuda()
    out = {"workload": "img2048x64_b4_n4096 train (M=16777216, L=16, N=4096, seeds 5001..5064) + "
                       "encode of 16777216 more vectors (seeds 5101..5164)",
           "data_sha256": {"train": synth.digest(X_np)[:16], "encode": synth.digest(Y_np)[:16]}}
    C_last = None
    for prec in ("bf16", "fp32"):
        lbg.lbg_train(X, N, 0.01, 1e-3, max_passes=1, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = lbg.lbg_train(X, N, 0.01, 1e-3, precision=prec)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        idx = torch.empty(Y.shape[0], dtype=torch.int32, device="cuda")
        lbg.vq_encode(Y, r.C, idx_out=idx, precision=prec)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            enc = lbg.vq_encode(Y, r.C, idx_out=idx, precision=prec, phase_ms=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        t_enc = statistics.median(ts)
        out[prec] = {"full_lbg_s": t_train, "passes": r.n_passes, "D": r.D, "encode_s": t_enc,
                     "encode_evals_per_s": Y.shape[0] * N / t_enc, "encode_phase_ms": enc.phase_ms,
                     "encode_exact_rows": enc.n_exact}
        C_last = r.C
    if with_oracle:
        try:
            import oracle
            oracle.build()
            rng = np.random.default_rng(5)
            C = C_last.cpu().numpy().astype(np.float64)
            rows = 4096
            while True:
                S = np.ascontiguousarray(Y_np[np.sort(rng.choice(Y_np.shape[0], rows, replace=False))])
                t0 = time.perf_counter()
                oracle.assign(S, C)
                t = time.perf_counter() - t0
                if t > 3.0 or rows >= 1 << 20:
                    break
                rows *= 4
            out["oracle_encode"] = {"evals_per_s": rows * N / t, "rows": rows, "seconds": t,
                                    "cores": oracle.max_threads(), "kind": "FP64 oracle nearest "
                                    "codevector of a random row sample of the encode set against the "
                                    "FP32 design's codebook, all host threads"}
        except Exception as exc:   # a report must never cost the measured line
            out["oracle_encode"] = {"error": repr(exc)}
    return out


def after_split_leg(lbg, torch, X, N, args, flush, stream, dist):
    """The step against the codebook right after the design's last split (pass 0 of the
    N-entry stage: every codevector has a twin at 2 delta, the least converged codebook and
    the one with the most near-ties), in both precisions."""
    half = lbg.lbg_train(X, N // 2, 0.01, 1e-3, precision=args.precision).C
    Cs = lbg.lbg_train(X, N, 0.01, 1e-3, C_init=half, max_passes=1, precision=args.precision).C
    C_out = torch.empty_like(Cs)
    A = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    out = {"codebook": f"N={N}: the N/2 design split once (pass 0 of the last stage)"}
    for prec in (args.precision, "fp32" if args.precision == "bf16" else "bf16"):
        for _ in range(3):
            flush.zero_()
            lbg.lbg_lloyd_step(X, Cs, C_out=C_out, assign_out=A, precision=prec)
        # enqueue-only calls (replayed graph, report in a device buffer) as in the headline
        # step; the phases from one directly launched call after them
        buf = lbg.step_result_buffer()
        per = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lbg.lbg_lloyd_step(X, Cs, C_out=C_out, assign_out=A, precision=prec, result_out=buf)
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1))
        _, nex, status = lbg.read_step_result(buf)
        if status != 0:
            raise RuntimeError(f"after-split step status {status}")
        flush.zero_()
        r = lbg.lbg_lloyd_step(X, Cs, C_out=C_out, assign_out=A, precision=prec, phase_ms=True)
        ms = max_over_ranks(dist, statistics.median(per))
        out[prec] = {"ms_per_step": ms, "value": X.shape[0] * N / (ms / 1e3), "unit": UNIT,
                     "exact_rows_per_step": nex, "phase_ms": r.phase_ms}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
