#!/usr/bin/env python
"""Benchmark of the compressed-multiplication hot path on one GB300 per rank.

Workload (one "step"): Compress (prep + fused sketch/FWHT/MAC + FP64 finish),
Decompress of every entry (median over d) and the heavy-hitter list, for
n = 8192 planted +-1 correlations (64 planted row pairs, rho = 0.9, B = A^T,
FP64 inputs), b = 2^16, d = 9, tau = n/2.  The metric is the step time in ms;
the JSON line also carries the HBM-roofline fraction of the step (bytes of A
and B read once), the roofline of the dominant kernel, the plain FP64 form's
step time on the same input (the FP32 path's R is compared against it), an
end-to-end time through the host-buffer C call, and the FP64 CPU oracle timed
on a bounded sample on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cmm|reference]
Multi-GPU: one process per GPU (torchrun), every rank runs its own independent
problem (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import contextlib
import gc
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sketch+FWHT+extract ms & % HBM roofline; speedup vs plain FP64 at equal error"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
def traffic_path(prec: str, n: int) -> str:
    """ncu DRAM traffic of one sketch launch, stored by the profiling summary."""
    return os.path.join(ROOT, "profiles", "sketch_%s_n%d_traffic.json" % (prec, n))


FALLBACK_HBM_GBS = 6800.0
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cmm", "reference"], default="cmm")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--log2b", type=int, default=16)
    ap.add_argument("--d", type=int, default=9)
    ap.add_argument("--prec", default="fx64",
                    choices=["f32", "f64", "fx64", "ternary", "bf16tc", "f16tc"],
                    help="arithmetic of the timed step (default: the exact fixed-point form, within the FP64 tolerance)")
    ap.add_argument("--compare-steps", type=int, default=3,
                    help="timed steps of each other form (FP32, plain FP64) on the same input")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-dgemm", action="store_true", help="skip the cuBLAS DGEMM comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--workload", default="planted",
                    choices=["planted", "batched", "precision", "diff", "cyclic", "paper",
                             "instances"],
                    help="planted (the headline line) or one of the other configurations")
    ap.add_argument("--tune-budget", type=float, default=120.0)
    ap.add_argument("--batch-count", type=int, default=256,
                    help="problems in the batched workload (256 = its configuration)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload: default tiles only (no autotuner pass)")
    return ap.parse_args()


L2_BYTES = 129e6   # L2 of one GB300


def l2_note(nbytes: float) -> str:
    """How the timed steps relate to the L2: inputs larger than it, or not."""
    if nbytes > L2_BYTES:
        return "inputs (%.0f MiB) larger than L2 (129 MB)" % (nbytes / 2**20)
    return "inputs (%.0f MiB) fit in L2 (129 MB); L2 not flushed between steps" % (nbytes / 2**20)


def workload_config(a):
    l2 = l2_note(2 * a.n * a.n * 8)
    return {
        "workload": "planted +-1 correlations n=%d (64 row pairs, rho=0.9, B=A^T, FP64 storage), "
                    "b=2^%d, d=%d, median, heavy hitters |C|>=n/2" % (a.n, a.log2b, a.d),
        "n": a.n, "m": a.n, "k": a.n, "p": a.n, "log2b": a.log2b, "d": a.d,
        "tau": a.n / 2, "input_dtype": "f64", "l2": l2,
        "arithmetic": FORM_OF.get(getattr(a, "prec", "fx64"), ""),
        "parallelism": "replicas (one problem per GPU)",
    }


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured", pk
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", {}


def source_hash(prec: str = "f32"):
    """Hash of the sources of a form's sketch kernel (a stored traffic figure is
    used only while they are unchanged)."""
    h = hashlib.sha256()
    names = (["sketch_fx64.cu", "fwht_device.cuh", "tmem_device.cuh", "sketch_impl.cuh"]
             if prec == "fx64" else
             ["sketch_impl.cuh", "fwht_device.cuh", "sketch_f32.cu", "sketch_tm.cu",
              "tm_slice.cuh"])
    for name in names:
        with open(os.path.join(ROOT, "paper_2601_09477_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def alu_roofline(kernel: str, ops: float, ms: float, note: str = "") -> dict:
    """Roofline object of an FP32-ALU-bound kernel: algorithmic operations per
    launch / its average launch time, against 152 SMs x 128 FP32 lanes at the
    maximum SM clock."""
    _, _, pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    achieved = ops / (ms * 1e-3) / 1e12
    out = {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3),
           "peak": round(peak, 3), "unit": "Tops/s", "frac": round(achieved / peak, 4),
           "traffic": None, "ops_per_launch": ops,
           "peak_source": "152 SMs x 128 FP32 lanes x %g MHz max SM clock" % sm_max,
           "avg_launch_ms": round(ms, 4)}
    if note:
        out["ops_counted"] = note
    return out


# the arithmetic each form computes in, and its name
DTYPE_OF = {"fx64": "int64", "f32": "f32", "f64": "f64", "bf16tc": "bf16", "f16tc": "f16",
            "ternary": "int16x2"}
FORM_OF = {"fx64": "exact 64-bit fixed-point butterflies, float-float multiply-accumulate, FP64 "
                   "reduction/inverse/extraction (FP64 tolerance)",
           "f32": "FP32 butterflies (fixed-point scatter), FP64 reduction/inverse/extraction",
           "f64": "plain FP64 butterflies and accumulation",
           "bf16tc": "BF16 tensor-core Hadamard blocks, FP32 accumulation",
           "f16tc": "FP16 tensor-core Hadamard blocks, FP32 accumulation",
           "ternary": "exact integer form for -1/0/+1 operands: two inner indices per 32-bit word, "
                      "int32 multiply-accumulate into int64"}


def alu_roofline_for(prec: str, kernel: str, ops: float, ms: float) -> dict:
    """Roofline object of a sketch kernel: its algorithmic operations per launch
    (butterfly add/subs of both sketches and one multiply-accumulate per
    bucket) over its average launch time, against the peak of the unit the
    form's butterflies run on: FP32 lanes (FP32 and tensor-core forms), 32-bit
    integer lanes at two instructions per 64-bit add (exact fixed point), or
    the FP64 pipe (plain FP64)."""
    _, _, pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    lanes = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6
    if prec == "ternary":
        peak, src = lanes * 2 / 1e12, ("152 SMs x 128 integer lanes x %g MHz x 2 (two 16-bit "
                                       "halves per 32-bit add)" % sm_max)
    elif prec == "fx64":
        peak, src = lanes / 2 / 1e12, ("152 SMs x 128 integer lanes x %g MHz / 2 instructions "
                                       "per 64-bit add" % sm_max)
    elif prec == "f64":
        peak, src = SM_COUNT * 2 * sm_max * 1e6 / 1e12, ("152 SMs x 2 FP64 adds per clock x %g "
                                                         "MHz" % sm_max)
    else:
        peak, src = lanes / 1e12, "152 SMs x 128 FP32 lanes x %g MHz max SM clock" % sm_max
    achieved = ops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"bound": "alu", "kernel": kernel, "achieved": round(achieved, 3),
            "peak": round(peak, 3), "unit": "Tops/s", "frac": round(achieved / peak, 4),
            "traffic": None, "ops_per_launch": ops, "peak_source": src,
            "avg_launch_ms": round(ms, 4)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine
    type), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine() or "unknown"


def timed_oracle(fn) -> float:
    """Seconds one call of an oracle function takes on the host cores."""
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self, ready_s: float = 5.0):
        """Start sampling and return once the first sample is written (at most
        `ready_s` seconds): nvidia-smi's start-up queries the driver, and a
        timed region that overlaps it can see one call stalled by tens of ms."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.perf_counter() + ready_s
        while time.perf_counter() < t_end and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        time.sleep(0.25)   # past the second sample as well

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows
                                    if r[3].replace(".", "").isdigit()), default=None)}


@contextlib.contextmanager
def no_gc():
    """The Python garbage collector held off inside a timed region (a full
    collection over the large lists the evaluation builds pauses the host for
    tens of ms, which a synchronous call loop would count)."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of the ranks' values, returned on every rank (the job ends
    when its slowest replica does); world 1 returns the value itself."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms(ms_max: float, world: int) -> float:
    """Time per problem of the whole job: world independent replicas, one
    problem each, all done after ms_max (reported beside `value`, which is the
    step time itself)."""
    return ms_max / max(world, 1)


# --------------------------------------------------------------------------- oracle arm
def oracle_sample(A, B, hp, log2b, n, d, tau, k_sample, rows_sample, threads):
    """Time the FP64 oracle on a bounded sample of the workload and scale it to
    one full step: Compress over k_sample of the n inner indices (the cost is
    linear in k) and Decompress + threshold over rows_sample of the n rows
    (linear in rows)."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    R = orc.compress(np.ascontiguousarray(A[:, :k_sample]), np.ascontiguousarray(B[:k_sample]),
                     hp, log2b, nthreads=threads)
    t1 = time.perf_counter()
    orc.extract(R, hp, n, n, rows=(0, rows_sample), nthreads=threads)
    t2 = time.perf_counter()
    ms = ((t1 - t0) * n / k_sample + (t2 - t1) * n / rows_sample) * 1e3
    if k_sample == n and rows_sample == n:
        sample = ("the whole step: Compress over all %d inner indices and Decompress of all %d "
                  "rows, FP64, %d threads (no scaling)" % (n, n, threads))
    else:
        sample = ("Compress on %d of %d inner indices, Decompress of %d of %d rows, FP64, %d "
                  "threads; scaled linearly to the full step" % (k_sample, n, rows_sample, n,
                                                                threads))
    return ms, sample, (t2 - t0)


def oracle_step(A, B, hp, log2b, n, d, tau, threads, with_R=False):
    """One whole step of the FP64 oracle on the host cores: Compress over all
    inner indices, Decompress of every entry, and the heavy-hitter list
    {(i, j) : |Chat_ij| >= tau} of that estimate.  Returns its time in ms."""
    from oracle import oracle as orc
    t0 = time.perf_counter()
    R = orc.compress(A, B, hp, log2b, nthreads=threads)
    C = orc.extract(R, hp, n, n, nthreads=threads)
    I, J = np.nonzero(np.abs(C) >= tau)
    del C, I, J
    ms = (time.perf_counter() - t0) * 1e3
    if with_R:
        return ms, R
    return ms


# wall-clock bound of the reference arm's timed steps: the arm stops early (and
# reports the steps it ran) rather than exceed it
REFERENCE_BUDGET_S = 240.0


def run_reference(a):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2601_09477_gb300 import workloads as wl
    from oracle import oracle as orc
    A, B, _ = wl.planted_pm1(n=a.n, pairs=64, rho=0.9, seed=1002)
    hp = orc.draw_hashes(2002, a.d)
    threads = orc.max_threads()
    tau = a.n / 2
    w0 = time.perf_counter()
    for _ in range(a.warmup):
        oracle_step(A, B, hp, a.log2b, a.n, a.d, tau, threads)
    times = []
    t0 = time.perf_counter()
    for _ in range(max(a.steps, 1)):
        times.append(oracle_step(A, B, hp, a.log2b, a.n, a.d, tau, threads))
        if len(times) >= a.steps or time.perf_counter() - t0 > REFERENCE_BUDGET_S:
            break
    wall = time.perf_counter() - w0
    v = float(np.mean(times))
    sample = ("the whole step, unscaled: Compress over all %d inner indices, Decompress of all "
              "%d x %d entries and the heavy-hitter list, FP64, %d threads; %d timed steps "
              "after %d warm-up steps" % (a.n, a.n, a.n, threads, len(times), a.warmup))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms",
           "n_gpus": world, "steps": len(times), "steps_requested": a.steps,
           "warmup": a.warmup, "ms_per_step": round(v, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(a),
           "wall_s": round(wall, 2),
           "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": threads,
                            "kind": "oracle", "sample": sample, "cpu_model": cpu_model()},
           "e2e": {"value": round(v, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def run_cmm(a):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2601_09477_gb300 import cmm
    from paper_2601_09477_gb300 import workloads as wl

    n, L, d = a.n, a.log2b, a.d
    tau = n / 2
    A_np, B_np, pairs = wl.planted_pm1(n=n, pairs=64, rho=0.9, seed=1002 + rank)
    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    h = cmm.make_hashes(2002, d, L)
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(cmm.multiply_workspace_bytes(n, n, n, h, torch.float64, a.prec),
                     dtype=torch.uint8, device=dev)
    R = torch.empty((d, 1 << L), dtype=torch.float64, device=dev)
    C = torch.empty((n, n), dtype=torch.float64, device=dev)
    cap = 1 << 22
    hh = (torch.empty(cap, dtype=torch.int32, device=dev),
          torch.empty(cap, dtype=torch.int32, device=dev),
          torch.empty(cap, dtype=torch.float64, device=dev))

    def step(prec):
        # Compress, Decompress and the ordered heavy-hitter list in one call
        _, lst = cmm.multiply_threshold(A, B, h, tau, capacity=cap, prec=prec, R=R, out=C, ws=ws,
                                        hh=hh)
        return lst

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(a.warmup):
        step(a.prec)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    cmm.trace_enable(True)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # one event per step boundary as well (the paper reports min and median)
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps - 1)]
    with no_gc():
        w0 = time.perf_counter()
        e0.record(stream)
        for it in range(a.steps):
            I, J, V = step(a.prec)
            if it + 1 < a.steps:
                marks[it].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
    bounds = [e0] + marks + [e1]
    per_step = sorted(bounds[q].elapsed_time(bounds[q + 1]) for q in range(a.steps))
    wall = time.perf_counter() - w0
    barrier()
    cmm.trace_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    trace = cmm.trace_read()
    ms = max_over_ranks(ms, world, dev)

    # heavy-hitter evaluation (the off-diagonal filter is part of the evaluation)
    Ih, Jh = I.cpu().numpy(), J.cpu().numpy()
    found = set(zip(Ih.tolist(), Jh.tolist()))
    planted = {(int(i), int(j)) for i, j in pairs} | {(int(j), int(i)) for i, j in pairs}
    offdiag = sum(1 for (i, j) in found if i != j)
    recall = sum(1 for q in planted if q in found) / len(planted)

    # dominant kernel and its roofline (ALU-bound butterflies)
    sk_name = "sketch_" + a.prec
    launches = sum(v[0] for v in trace.values())
    sk_launches, sk_ms_total = trace.get(sk_name, (0, 0.0))
    sk_ms = sk_ms_total / a.steps   # one sketch call per step
    b = 1 << L
    ops = d * n * (2.0 * b * L + b)   # butterfly add/sub of both sketches + one MAC per bucket
    hbm_gbs, hbm_kind, pk = peaks()
    roofline = alu_roofline_for(a.prec, sk_name, ops, sk_ms)
    try:
        with open(traffic_path(a.prec, n)) as f:
            tj = json.load(f)
        if (tj.get("prec", "f32") == a.prec and tj.get("source_hash") == source_hash(a.prec)
                and tj.get("n") == n and tj.get("log2b") == L):
            roofline["traffic"] = tj.get("dram_bytes_per_launch")
    except Exception:
        pass
    ab_bytes = 2.0 * n * n * 8
    hbm = {"bytes_A_B": ab_bytes, "achieved_gbs": round(ab_bytes / (ms * 1e-3) / 1e9, 2),
           "peak_gbs": hbm_gbs, "peak_kind": hbm_kind,
           "frac": round(ab_bytes / (ms * 1e-3) / 1e9 / hbm_gbs, 5)}

    result = {"metric": METRIC, "value": round(ms, 4), "unit": "ms",
              "n_gpus": world, "ms_per_problem_whole_job": round(whole_job_ms(ms, world), 4),
              "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 4),
              "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
              "dtype": DTYPE_OF[a.prec], "precision_form": FORM_OF[a.prec],
              "data": "synthetic", "config": workload_config(a),
              "roofline": roofline, "hbm_roofline": hbm, "gpu_launches": int(launches),
              "clocks": clk, "kernels_ms_per_step": {k: round(v[1] / a.steps, 4)
                                                     for k, v in sorted(trace.items())},
              "heavy_hitters": {"count": int(len(Ih)), "offdiag": offdiag,
                                "planted_recall": recall},
              "wall_s_timed": round(wall, 3),
              "step_ms_min": round(per_step[0], 4),
              "step_ms_median": round(per_step[len(per_step) // 2], 4)}

    # the other forms on the same input, each over --compare-steps timed steps
    # after one warm-up step, with its own clock record: time, the sketch
    # kernel's roofline, and its R (compared with the oracle's below)
    R_main = R.clone()
    forms = {}
    if not a.no_fp64:
        for prec in [pr for pr in ("f32", "ternary", "f64") if pr != a.prec]:
            step(prec)
            torch.cuda.synchronize()
            ck = ClockSampler(local)
            ck.start()
            cmm.trace_enable(True)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.compare_steps + 1)]
            ev[0].record(stream)
            for q in range(a.compare_steps):
                step(prec)
                ev[q + 1].record(stream)
            torch.cuda.synchronize()
            cmm.trace_enable(False)
            tr = cmm.trace_read()
            times = sorted(ev[q].elapsed_time(ev[q + 1]) for q in range(a.compare_steps))
            f_ms = float(np.mean(times))
            k_ms = tr.get("sketch_" + prec, (0, 0.0))[1] / a.compare_steps
            forms[prec] = {"form": FORM_OF[prec], "dtype": DTYPE_OF[prec],
                           "ms_per_step": round(f_ms, 3), "step_ms_min": round(times[0], 3),
                           "step_ms_median": round(times[len(times) // 2], 3),
                           "steps": a.compare_steps, "clocks": ck.stop(),
                           "roofline": alu_roofline_for(prec, "sketch_" + prec, ops, k_ms),
                           "speedup_of_headline": round(f_ms / ms, 2),
                           "R": R.clone()}
        result["forms"] = forms
        if "f64" in forms:
            result["speedup_vs_plain_fp64"] = forms["f64"]["speedup_of_headline"]
            for prec, fm in forms.items():
                if prec != "f64":
                    fm["speedup_vs_plain_fp64"] = round(forms["f64"]["ms_per_step"] /
                                                        fm["ms_per_step"], 2)

    # the heavy-hitter list straight from the sketch, without writing C
    # (cmm_heavy_hitters on the step's R): same list as the step's
    if world == 1:
        hfn = lambda: cmm.heavy_hitters(R_main, h, n, n, tau, capacity=cap)
        I2, J2, V2 = hfn()
        same = bool(torch.equal(I2.cpu(), I.cpu()) and torch.equal(J2.cpu(), J.cpu())
                    and torch.equal(V2.cpu(), V.cpu()))
        result["heavy_hitters_from_R"] = {"ms": round(_events_ms(hfn, 5), 3),
                                          "same_list_as_step": same}

    # end to end through the host-buffer C call (pinned host memory)
    if not a.no_e2e:
        Ah = torch.from_numpy(A_np).pin_memory()
        Bh = torch.from_numpy(B_np).pin_memory()
        Ch = torch.empty((n, n), dtype=torch.float64).pin_memory()
        hh = (torch.empty(cap, dtype=torch.int32).pin_memory(),
              torch.empty(cap, dtype=torch.int32).pin_memory(),
              torch.empty(cap, dtype=torch.float64).pin_memory())
        del ws
        wsh = torch.empty(cmm.multiply_host_workspace_bytes(n, n, n, h, torch.float64, a.prec,
                                                            capacity=cap),
                          dtype=torch.uint8, device=dev)
        for _ in range(max(3, a.warmup)):
            cmm.multiply_host(Ah, Bh, h, prec=a.prec, out=Ch, tau=tau, capacity=cap,
                              hh_out=hh, ws=wsh)
        torch.cuda.synchronize()
        barrier()
        calls = []
        eclk = ClockSampler(local)
        eclk.start()
        with no_gc():
            t0 = time.perf_counter()
            for _ in range(a.e2e_steps):
                c0 = time.perf_counter()
                _, (Ie, Je, Ve) = cmm.multiply_host(Ah, Bh, h, prec=a.prec, out=Ch, tau=tau,
                                                    capacity=cap, hh_out=hh, ws=wsh)
                calls.append((time.perf_counter() - c0) * 1e3)
            e2e_s = time.perf_counter() - t0
        eclk = eclk.stop()
        e2e_ms = max_over_ranks(e2e_s * 1e3 / a.e2e_steps, world, dev)
        slowest = int(np.argmax(calls))
        # calls more than 2 ms above the median (host-side stalls: the device-timed
        # steps of the same work show none)
        slow_calls = int(sum(c > float(np.median(calls)) + 2.0 for c in calls))
        calls.sort()
        nhh = int(Ie.numel())
        # one more call, traced: device time of each copy and kernel span (the copies
        # run on the library's copy stream, overlapped with the kernels)
        cmm.trace_enable(True)
        cmm.multiply_host(Ah, Bh, h, prec=a.prec, out=Ch, tau=tau, capacity=cap, hh_out=hh,
                          ws=wsh)
        torch.cuda.synchronize()
        cmm.trace_enable(False)
        e2e_spans = {k: round(v[1], 3) for k, v in sorted(cmm.trace_read().items(),
                                                           key=lambda kv: -kv[1][1])}
        result["e2e"] = {"value": round(e2e_ms, 3), "unit": "ms",
                         "ms_per_problem_whole_job": round(whole_job_ms(e2e_ms, world), 3),
                         "h2d_bytes_per_step": int(2 * n * n * 8),
                         "d2h_bytes_per_step": int(n * n * 8 + nhh * 16),
                         "ms_per_step": round(e2e_ms, 3), "steps": a.e2e_steps,
                         "call_ms_min": round(calls[0], 3),
                         "call_ms_median": round(calls[len(calls) // 2], 3),
                         "call_ms_max": round(calls[-1], 3), "call_max_index": slowest,
                         "calls_over_median_plus_2ms": slow_calls,
                         "clocks": eclk,
                         "api": "cmm_multiply_host (pinned host A, B, C, heavy-hitter list)",
                         "spans_ms_one_call": e2e_spans}
        del wsh

    # cuBLAS DGEMM of the same product on the same GPU (the exact C): time of
    # one call after one warm-up, and the heavy hitters against the exact C
    if not a.no_dgemm and world == 1:
        Cx = torch.matmul(A, B)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        Cx = torch.matmul(A, B)
        g1.record(stream)
        torch.cuda.synchronize()
        dg_ms = g0.elapsed_time(g1)
        true_hh = int((Cx.abs() >= tau).sum().item())
        Ix = torch.from_numpy(Ih.astype(np.int64)).to(dev)
        Jx = torch.from_numpy(Jh.astype(np.int64)).to(dev)
        hits = int((Cx[Ix, Jx].abs() >= tau).sum().item()) if len(Ih) else 0
        result["dgemm"] = {"ms": round(dg_ms, 3), "tflops": round(2.0 * n ** 3 / dg_ms / 1e9, 3),
                           "speedup_of_sketch_step": round(dg_ms / ms, 2),
                           "exact_heavy_hitters": true_hh,
                           "reported_that_are_exact_heavy_hitters": hits,
                           "exact_heavy_hitters_found": hits / max(true_hh, 1)}
        del Cx, Ix, Jx

    # FP64 CPU oracle on a bounded sample (rank 0, single GPU only)
    if not a.no_cpu and rank == 0 and world == 1:
        from oracle import oracle as orc
        threads = orc.max_threads()
        # the whole step at the benchmark size takes the oracle about 5 s on 16 cores
        cpu_ms, R_orc = oracle_step(A_np, B_np, h.params, L, n, d, tau, threads, with_R=True)
        secs = cpu_ms / 1e3
        # every form's R against the oracle's, relative to sum_t ||A_t|| ||B_t||
        scale = float(np.sum(np.linalg.norm(A_np, axis=0) * np.linalg.norm(B_np, axis=1)))
        result["R_error_vs_oracle"] = {
            a.prec: float(np.abs(R_main.cpu().numpy() - R_orc).max() / scale)}
        for prec, fm in forms.items():
            result["R_error_vs_oracle"][prec] = float(
                np.abs(fm["R"].cpu().numpy() - R_orc).max() / scale)
        result["R_error_vs_oracle"]["relative_to"] = "sum_t ||A[:,t]|| ||B[t,:]||"
        sample = ("the whole step, unscaled: Compress over all %d inner indices, Decompress of "
                  "all %d x %d entries and the heavy-hitter list, FP64, %d threads"
                  % (n, n, n, threads))
        # the same oracle on one core, on a sample (Compress over n/64 inner
        # indices, Decompress of n/256 rows) scaled to the whole step
        one_ms, one_sample, one_secs = oracle_sample(A_np, B_np, h.params, L, n, d, tau,
                                                     max(16, n // 64), max(16, n // 256), 1)
        result["cpu_baseline"] = {"value": round(cpu_ms, 1), "unit": "ms", "cores": threads,
                                  "kind": "oracle", "sample": sample,
                                  "sample_seconds": round(secs, 2), "cpu_model": cpu_model(),
                                  "host_cpus": os.cpu_count(),
                                  "one_core": {"value": round(one_ms, 1), "unit": "ms",
                                               "sample": one_sample,
                                               "sample_seconds": round(one_secs, 2)}}
    for fm in forms.values():
        fm.pop("R", None)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _events_ms(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_batched(a):
    """256 uneven problems in one persistent launch, replayed from a CUDA graph;
    default tiles vs autotuned tiles; against the same problems run one call at
    a time (FP32 butterflies and the plain FP64 form)."""
    import torch
    from paper_2601_09477_gb300 import autotune, cmm
    from paper_2601_09477_gb300 import workloads as wl
    torch.cuda.set_device(0)
    d = 5
    raw = wl.batch_problems_device(count=a.batch_count, seed=1004, device="cuda")
    probs = [cmm.Problem(At, B, cmm.make_hashes(7000 + q, d, L)) for q, (At, B, L, _) in enumerate(raw)]
    out = {}
    for label in (("default",) if a.no_tune else ("default", "tuned")):
        if label == "tuned":
            for pb in probs:
                pb.R = pb.C = None
            t0 = time.time()
            autotune.tune_batch(probs, d=d, cache_path=os.path.join(tempfile.gettempdir(),
                                                                    "cmm_tune_bench.json"),
                                budget_s=a.tune_budget)
            out["tune_seconds"] = round(time.time() - t0, 1)
        batch = cmm.Batch(probs, d=d)
        for _ in range(a.warmup):
            batch.launch()
        assert batch.status() == cmm.OK
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            batch.launch()
        clocks = ClockSampler(0)
        clocks.start()
        ms = _events_ms(g.replay, a.steps)
        out[label + "_clocks"] = clocks.stop()
        assert batch.status() == cmm.OK
        out[label + "_ms"] = round(ms, 3)
    flops = sum(d * pb.At.shape[0] * (2.0 * (1 << pb.hashes.log2b) * pb.hashes.log2b +
                                      (1 << pb.hashes.log2b)) for pb in probs)
    outputs = sum(pb.At.shape[1] * pb.B.shape[1] for pb in probs)
    best = min(out["default_ms"], out.get("tuned_ms", out["default_ms"]))
    out["roofline"] = alu_roofline("batched_kernel", flops, best,
                                   "per problem d*k*(2 b log2 b + b): butterflies of both "
                                   "sketches and the MAC")
    # the same problems one call at a time through cmm_multiply, with FP32
    # butterflies and in the plain FP64 form, and the batched sketch's error
    # against the FP64 one (relative to sum_t ||A_t|| ||B_t|| of each problem)
    Rb = [pb.R.clone() for pb in probs]
    R64 = [torch.empty((d, pb.hashes.b), dtype=torch.float64, device="cuda") for pb in probs]
    wsq = torch.empty(max(cmm.multiply_workspace_bytes(pb.At.shape[1], pb.At.shape[0],
                                                       pb.B.shape[1], pb.hashes, torch.float32,
                                                       pr, transA=True)
                          for pb in probs for pr in ("f32", "f64")),
                      dtype=torch.uint8, device="cuda")

    def one_by_one(prec, Rs=None):
        for q, pb in enumerate(probs):
            cmm.multiply(pb.At, pb.B, pb.hashes, prec=prec, transA=True, out=pb.C, ws=wsq,
                         R=Rs[q] if Rs is not None else None)

    one_by_one("f32")
    torch.cuda.synchronize()
    seq32 = _events_ms(lambda: one_by_one("f32"), 1)
    seq64 = _events_ms(lambda: one_by_one("f64", R64), 1)
    err = 0.0
    for q, pb in enumerate(probs):
        sc = float((torch.linalg.vector_norm(pb.At.double(), dim=1) *
                    torch.linalg.vector_norm(pb.B.double(), dim=1)).sum().item())
        err = max(err, float((Rb[q] - R64[q]).abs().max().item()) / max(sc, 1e-300))
    out["one_call_per_problem_ms"] = {"f32": round(seq32, 3), "f64": round(seq64, 3)}
    out["speedup_vs_one_call_per_problem"] = {"f32": round(seq32 / best, 2),
                                              "f64": round(seq64 / best, 2)}
    out["R_err_vs_fp64_rel_to_sum_norms"] = err
    del Rb, R64, wsq
    # the literal reading of the sketch-length rule (next power of two >= 8 x 16
    # planted entries, at least 2^10): every problem at b = 2^10, default tiles,
    # where reading A and B once from HBM is a bound of the same order as the
    # butterflies
    lit = [cmm.Problem(At, B, cmm.make_hashes(7000 + q, d, 10)) for q, (At, B, _, _) in enumerate(raw)]
    lbatch = cmm.Batch(lit, d=d)
    for _ in range(a.warmup):
        lbatch.launch()
    assert lbatch.status() == cmm.OK
    lg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(lg):
        lbatch.launch()
    lclk = ClockSampler(0)
    lclk.start()
    lms = _events_ms(lg.replay, a.steps)
    lclk = lclk.stop()
    assert lbatch.status() == cmm.OK
    lflops = sum(d * pb.At.shape[0] * (2.0 * 1024 * 10 + 1024) for pb in lit)
    lbytes = float(sum((At.numel() + B.numel()) * 4 for (At, B, _, _) in raw))
    hbm_gbs, hbm_kind, _ = peaks()
    # the same launch without the extraction tasks (the problems' R reused, no
    # C): the sketch and finish alone, and Decompress by difference; at b = 2^10
    # each extraction task stages R in shared memory, so its d gathers per entry
    # are shared-memory loads
    skp = [cmm.Problem(pb.At, pb.B, pb.hashes, R=pb.R) for pb in lit]
    sbatch = cmm.Batch(skp, d=d, with_C=False)
    for _ in range(a.warmup):
        sbatch.launch()
    assert sbatch.status() == cmm.OK
    sms = _events_ms(sbatch.launch, a.steps)
    assert sbatch.status() == cmm.OK
    del skp, sbatch
    lgathers = float(sum(d * pb.At.shape[1] * pb.B.shape[1] for pb in lit))
    ext_ms = max(lms - sms, 1e-6)
    out["literal_b1024"] = {
        "ms": round(lms, 3), "clocks": lclk,
        "sketch_and_finish_ms": round(sms, 3),
        "extraction_ms_by_difference": round(lms - sms, 3),
        "extraction_gathers": lgathers,
        "extraction_gathers_per_clock_per_sm": round(lgathers / (ext_ms * 1e-3) / (152 * 2.07e9), 2),
        "roofline": alu_roofline("batched_kernel", lflops, lms,
                                 "per problem d*k*(2 b log2 b + b) at b = 2^10"),
        "hbm_roofline": {"bytes_A_B": lbytes, "achieved_gbs": round(lbytes / (lms * 1e-3) / 1e9, 1),
                         "peak_gbs": hbm_gbs, "peak_kind": hbm_kind,
                         "frac": round(lbytes / (lms * 1e-3) / 1e9 / hbm_gbs, 4)}}
    del lit, lbatch, lg
    if not a.no_cpu:
        out["cpu_baseline"] = batched_oracle(raw, probs, d, nsample=32)
    res = {"metric": "batched: 256 uneven problems (sketch + FP64 finish + median extraction), "
                     "one persistent launch replayed from a CUDA graph, ms",
           "value": best, "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
           "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "%d problems, m,k,p uniform in [512,4096], b=2^10..2^15, d=5, " % a.batch_count +
                                  "16 planted spikes each, FP32, A given as A^T",
                      "l2": l2_note(sum(At.numel() + B.numel() for (At, B, _, _) in raw) * 4)},
           "alu_tops": round(flops / (best * 1e-3) / 1e12, 3), "entries_estimated": outputs,
           "gpu_launches_per_step": 1}
    res.update(out)
    print(json.dumps(res), flush=True)
    return 0


def batched_oracle(raw, probs, d, nsample=8):
    """FP64 oracle (Compress + Decompress of every entry) on the first nsample
    problems of the batch, scaled to all of them: Compress time by the ratio of
    d*k*b*log2 b, Decompress time by the ratio of d*m*p."""
    from oracle import oracle as orc
    threads = orc.max_threads()
    tc = te = 0.0
    cs = es = 0.0
    for q in range(nsample):
        At, B, L, _ = raw[q]
        At64 = At.double().cpu().numpy()
        B64 = B.double().cpu().numpy()
        hp = probs[q].hashes.params
        m, p = At64.shape[1], B64.shape[1]
        box = {}
        tc += timed_oracle(lambda: box.setdefault("R", orc.compress(At64, B64, hp, L, transA=True,
                                                                    nthreads=threads)))
        te += timed_oracle(lambda: orc.extract(box["R"], hp, m, p, nthreads=threads))
    def ccost(pb):
        return d * pb.At.shape[0] * (1 << pb.hashes.log2b) * pb.hashes.log2b
    def ecost(pb):
        return d * pb.At.shape[1] * pb.B.shape[1]
    cs = sum(ccost(pb) for pb in probs[:nsample])
    es = sum(ecost(pb) for pb in probs[:nsample])
    ms = (tc * sum(ccost(pb) for pb in probs) / cs + te * sum(ecost(pb) for pb in probs) / es) * 1e3
    return {"value": round(ms, 1), "unit": "ms", "cores": threads, "kind": "oracle",
            "sample": "Compress + Decompress of the first %d of %d problems, FP64, %d threads; "
                      "scaled by d*k*b*log2 b (Compress) and d*m*p (Decompress)"
                      % (nsample, len(probs), threads),
            "sample_seconds": round(tc + te, 2)}


def run_precision(a):
    """n=16384, b=2^18, d=7: FP32 butterflies, BF16 / FP16 tensor-core Hadamard
    blocks and the exact fixed-point form (and one plain FP64 step) on the same
    input; errors of R against the FP64 form."""
    import torch
    from paper_2601_09477_gb300 import cmm
    from paper_2601_09477_gb300 import workloads as wl
    torch.cuda.set_device(0)
    n, L, d = 16384, 18, 7
    A, B, S = wl.orthogonal_precision(n=n, seed=1003, device="cuda")
    h = cmm.make_hashes(2003, d, L)
    ws = torch.empty(max(cmm.multiply_workspace_bytes(n, n, n, h, torch.float32, p)
                         for p in ("f32", "bf16tc", "f16tc", "fx64", "f64")), dtype=torch.uint8,
                     device="cuda")
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    Rs, times, kernels = {}, {}, {}
    clocks = ClockSampler(0)
    clocks.start()
    for prec, reps in (("f64", 1), ("f32", a.steps), ("bf16tc", a.steps), ("f16tc", a.steps),
                       ("fx64", a.steps)):
        R = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
        fn = lambda: cmm.multiply(A, B, h, prec=prec, R=R, out=C, ws=ws)
        for _ in range(1 if prec == "f64" else a.warmup):
            fn()
        torch.cuda.synchronize()
        cmm.trace_enable(True)
        times[prec] = round(_events_ms(fn, reps), 3)
        cmm.trace_enable(False)
        kernels[prec] = {k: round(v[1] / reps, 4) for k, v in cmm.trace_read().items()}
        Rs[prec] = R
    clk = clocks.stop()
    scale = float((torch.linalg.vector_norm(A.double(), dim=0) *
                   torch.linalg.vector_norm(B.double(), dim=1)).sum().item())
    low = ("f32", "bf16tc", "f16tc", "fx64")
    err = {p: float((Rs[p] - Rs["f64"]).abs().max().item() / scale) for p in low}
    rms = float(Rs["f64"].pow(2).mean().sqrt().item())
    res = {"metric": "precision workload: multiply ms per precision, R error vs the FP64 form",
           "value": times["bf16tc"], "unit": "ms", "n_gpus": 1, "steps": a.steps,
           "warmup": a.warmup, "higher_is_better": False, "dtype": "bf16tc", "data": "synthetic",
           "config": {"workload": "n=16384, A=Q orthogonal, B=Q^T S + 1e-3 noise, 1024 entries "
                                  "N(0,1)*100, b=2^18, d=7, FP32 storage",
                      "l2": l2_note(2 * n * n * 4)},
           "ms": times, "R_err_rel_to_sum_norms": err,
           "R_err_rel_to_rms": {p: float((Rs[p] - Rs["f64"]).abs().max().item() / rms)
                                for p in low},
           "speedup_vs_fp64": {p: round(times["f64"] / times[p], 2) for p in low},
           "kernels_ms_per_call": kernels, "clocks": clk,
           "roofline": alu_roofline("sketch_f32", d * n * (2.0 * (1 << L) * L + (1 << L)),
                                    kernels["f32"].get("sketch_f32", float("nan")),
                                    "d*k*(2 b log2 b + b)")}
    if not a.no_cpu:
        from oracle import oracle as orc
        threads = orc.max_threads()
        ks, rows = 2048, 64
        A64 = A[:, :ks].double().cpu().numpy()
        B64 = B[:ks].double().cpu().numpy()
        box = {}
        tc = timed_oracle(lambda: box.setdefault("R", orc.compress(A64, B64, h.params, L,
                                                                   nthreads=threads)))
        te = timed_oracle(lambda: orc.extract(box["R"], h.params, n, n, rows=(0, rows),
                                              nthreads=threads))
        res["cpu_baseline"] = {
            "value": round((tc * n / ks + te * n / rows) * 1e3, 1), "unit": "ms",
            "cores": threads, "kind": "oracle",
            "sample": "Compress over %d of %d inner indices, Decompress of %d of %d rows, FP64, "
                      "%d threads; scaled linearly to one multiply" % (ks, n, rows, n, threads),
            "sample_seconds": round(tc + te, 2)}
    print(json.dumps(res), flush=True)
    return 0


def run_diff(a):
    """n=4096 differentiable mean estimator: forward (sketch + mean at 4096
    pairs) and backward (adjoint kernel) through the autograd Function."""
    import torch
    from paper_2601_09477_gb300 import cmm
    from paper_2601_09477_gb300 import workloads as wl
    from paper_2601_09477_gb300.autograd_fn import compressed_mean_at_pairs
    torch.cuda.set_device(0)
    A, B, I, J, W = wl.diff_problem(n=4096, spikes=256, pairs=4096, seed=1005)
    h = cmm.make_hashes(2005, 5, 14)
    Ad = torch.from_numpy(A).cuda().requires_grad_()
    Bd = torch.from_numpy(B).cuda().requires_grad_()
    It, Jt, Wt = (torch.from_numpy(x).cuda() for x in (I, J, W))

    def fwd():
        return compressed_mean_at_pairs(Ad, Bd, It, Jt, h, "f32")

    def fwd_bwd():
        Ad.grad = Bd.grad = None
        (fwd().double() * Wt).sum().backward()

    for _ in range(a.warmup):
        fwd_bwd()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    with torch.no_grad():
        f_ms = _events_ms(fwd, a.steps)
    cmm.trace_enable(True)
    fb_ms = _events_ms(fwd_bwd, a.steps)
    cmm.trace_enable(False)
    clk = clocks.stop()
    kernels = {k: round(v[1] / a.steps, 4) for k, v in cmm.trace_read().items()}
    n, L, d = 4096, 14, 5
    fwd_ops = d * n * (2.0 * (1 << L) * L + (1 << L))
    adj_ops = d * n * (4.0 * (1 << L) * L + 2.0 * (1 << L))
    res = {"metric": "differentiation: forward and forward+backward ms (mean estimator, autograd)",
           "value": round(fb_ms, 3), "unit": "ms", "n_gpus": 1, "steps": a.steps,
           "warmup": a.warmup, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "n=4096 FP32, N(0,1)/sqrt(n) + 256 spikes, b=2^14, d=5, "
                                  "loss over 4096 weighted pairs", "l2": l2_note(2 * 4096 * 4096 * 4)},
           "forward_ms": round(f_ms, 3), "forward_backward_ms": round(fb_ms, 3),
           "kernels_ms_per_step": kernels, "clocks": clk,
           "roofline": alu_roofline("adjoint_f32", adj_ops, kernels.get("adjoint_f32", float("nan")),
                                    "d*k*(4 b log2 b + 2 b): per (r, t) the transforms of x_t "
                                    "and y_t, their products with H G and the inverse transforms"),
           "roofline_forward": alu_roofline("sketch_f32", fwd_ops,
                                            kernels.get("sketch_f32", float("nan")),
                                            "d*k*(2 b log2 b + b)")}
    if not a.no_cpu:
        from oracle import oracle as orc
        threads = orc.max_threads()
        box = {}
        tf = timed_oracle(lambda: box.setdefault("y", orc.mean_at_pairs(
            orc.compress(A, B, h.params, L, nthreads=threads), h.params, I, J)))
        tb = timed_oracle(lambda: orc.adjoint(A, B, h.params, L, I, J, W))
        res["cpu_baseline"] = {
            "value": round((tf + tb) * 1e3, 1), "unit": "ms", "cores": threads, "kind": "oracle",
            "sample": "the whole forward (Compress + mean at the 4096 pairs, %d threads) and "
                      "backward (adjoint through dense M, numpy BLAS) once, FP64" % threads,
            "forward_ms": round(tf * 1e3, 1), "backward_ms": round(tb * 1e3, 1)}
    print(json.dumps(res), flush=True)
    return 0


def run_cyclic(a):
    """FWHT form (Algorithm 1) vs Pagh's cyclic FFT form (Sec. 3.1) on the same
    problem: multiply ms of each and their ratio (the paper's FFT / FWHT speedup
    SU3), with the per-kernel trace and the planted-pair recall of each."""
    import torch
    from paper_2601_09477_gb300 import cmm
    from paper_2601_09477_gb300 import workloads as wl
    torch.cuda.set_device(0)
    n, L, d = a.n, a.log2b, a.d
    A, B, pairs = wl.gpu_planted_pm1(n, 64, 0.9, 1002, "cuda", torch.float32)
    h = cmm.make_hashes(2002, d, L)
    ws = torch.empty(max(cmm.multiply_workspace_bytes(n, n, n, h, torch.float32, "f32"),
                         int(cmm.lib.cmm_multiply_cyclic_workspace_bytes(n, n, n, d, L, 1, 1, 0))),
                     dtype=torch.uint8, device="cuda")
    C = torch.empty((n, n), dtype=torch.float64, device="cuda")
    forms = {"fwht": lambda: cmm.multiply(A, B, h, prec="f32", out=C, ws=ws),
             "cyclic": lambda: cmm.multiply_cyclic(A, B, h, out=C, ws=ws)}
    times, kernels, recall = {}, {}, {}
    tau = 0.5 * n
    pl = pairs.tolist()
    planted = {(int(i), int(j)) for i, j in pl} | {(int(j), int(i)) for i, j in pl}
    clocks = ClockSampler(0)
    clocks.start()
    for name, fn in forms.items():
        for _ in range(a.warmup):
            fn()
        torch.cuda.synchronize()
        cmm.trace_enable(True)
        times[name] = round(_events_ms(fn, a.steps), 3)
        cmm.trace_enable(False)
        kernels[name] = {k: round(v[1] / a.steps, 4) for k, v in cmm.trace_read().items()}
        I, J, _ = cmm.threshold(C, tau)
        found = set(zip(I.tolist(), J.tolist()))
        recall[name] = sum(1 for q in planted if q in found) / len(planted)
    res = {"metric": "FWHT vs cyclic FFT form: multiply ms (sketch + finish + extraction) and "
                     "FFT/FWHT ratio", "value": times["cyclic"], "unit": "ms", "n_gpus": 1,
           "steps": a.steps, "warmup": a.warmup, "higher_is_better": False, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "planted +-1 correlations n=%d (64 pairs, rho=0.9, B=A^T, FP32 "
                                  "storage), b=2^%d, d=%d" % (n, L, d), "l2": l2_note(2 * n * n * 4)},
           "ms": times, "fft_over_fwht": round(times["cyclic"] / times["fwht"], 2),
           "kernels_ms_per_step": kernels, "planted_recall": recall, "clocks": clocks.stop(),
           "roofline": alu_roofline("sketch_cyclic", d * n * (5.0 * (1 << L) * L + 4.0 * (1 << L)),
                                    kernels["cyclic"].get("sketch_cyclic", float("nan")),
                                    "d*k*(5 b log2 b + 4 b): two real-input FFTs of length b "
                                    "(2.5 b log2 b flops each) and the complex multiply-add of "
                                    "b/2 bins, per (r, t)")}
    if not a.no_cpu:
        from oracle import oracle as orc
        ks, rows = 128, 64
        A64 = A[:, :ks].double().cpu().numpy()
        B64 = B[:ks].double().cpu().numpy()
        box = {}
        tc = timed_oracle(lambda: box.setdefault("R", orc.compress_cyclic(A64, B64, h.params, L)))
        te = timed_oracle(lambda: orc.extract_cyclic(box["R"], h.params, n, n, rows=(0, rows)))
        res["cpu_baseline"] = {
            "value": round((tc * n / ks + te * n / rows) * 1e3, 1), "unit": "ms", "cores": 1,
            "kind": "oracle",
            "sample": "cyclic Compress (numpy FFT) over %d of %d inner indices, Decompress of %d "
                      "of %d rows, FP64, one thread; scaled linearly to one multiply"
                      % (ks, n, rows, n),
            "sample_seconds": round(tc + te, 2)}
    print(json.dumps(res), flush=True)
    return 0


def run_instances(a):
    """The paper's four instance families (Sec. 5.2) at n = 4096 with the
    parameters of Table 3: multiply ms (FP32 and FP64 butterflies) and the
    counters and category of Sec. 5.3 / 5.6 for each."""
    import torch
    from paper_2601_09477_gb300 import cmm
    from paper_2601_09477_gb300 import evaluate as ev
    torch.cuda.set_device(0)
    n = 4096
    rows = []
    for name, cd, cb in [("logunit", 1.0, 0.5), ("logunit", 0.25, 1.0), ("diagonal", 2.0, 4.0),
                         ("diagonal", 0.75, 4.0), ("covariance", 1.5, 4.0),
                         ("lightbulb", 2.0, 4.0)]:
        d, L = ev.params(n, cd, cb)
        A, B, Ct, big = ev.instance(name, n, seed=1)
        h = cmm.make_hashes(7, d, L)
        row = {"instance": name, "c_d": cd, "c_b": cb, "d": d, "log2b": L}
        for prec in ("f32", "f64"):
            ws = torch.empty(cmm.multiply_workspace_bytes(n, n, n, h, torch.float64, prec),
                             dtype=torch.uint8, device="cuda")
            C = torch.empty((n, n), dtype=torch.float64, device="cuda")
            fn = lambda: cmm.multiply(A, B, h, prec=prec, out=C, ws=ws)
            for _ in range(a.warmup):
                fn()
            row[prec + "_ms"] = round(_events_ms(fn, a.steps), 3)
            cnt = ev.counters(C, big, Ct)
            row[prec + "_category"] = ev.category(cnt, n)
            if prec == "f32":
                row["counters"] = cnt
        rows.append(row)
    res = {"metric": "paper instances at n=4096 (Table 3 parameters): multiply ms and the "
                     "category reached (Sec. 5.3 counters)", "value": rows[0]["f32_ms"],
           "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
           "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Logunit, Diagonal, Covariance, Lightbulb generators, n=4096, "
                                  "FP64 storage", "l2": l2_note(2 * 4096 * 4096 * 8)}, "rows": rows}
    if not a.no_cpu:
        # the oracle on the first row's instance: Compress over ks of the n inner
        # indices and Decompress of `nr` rows, scaled linearly to one multiply
        from oracle import oracle as orc
        threads = orc.max_threads()
        name, cd, cb = "logunit", 1.0, 0.5
        d, L = ev.params(n, cd, cb)
        A, B, _, _ = ev.instance(name, n, seed=1)
        hp = cmm.make_hashes(7, d, L).params
        ks, nr = 1024, 256
        A64 = A[:, :ks].double().cpu().numpy()
        B64 = B[:ks].double().cpu().numpy()
        box = {}
        tc = timed_oracle(lambda: box.setdefault("R", orc.compress(A64, B64, hp, L,
                                                                   nthreads=threads)))
        te = timed_oracle(lambda: orc.extract(box["R"], hp, n, n, rows=(0, nr), nthreads=threads))
        res["cpu_baseline"] = {
            "value": round((tc * n / ks + te * n / nr) * 1e3, 1), "unit": "ms", "cores": threads,
            "kind": "oracle", "instance": "%s c_d=%g c_b=%g (d=%d, b=2^%d)" % (name, cd, cb, d, L),
            "sample": "Compress over %d of %d inner indices, Decompress of %d of %d rows, FP64, "
                      "%d threads; scaled linearly to one multiply" % (ks, n, nr, n, threads),
            "sample_seconds": round(tc + te, 2)}
    print(json.dumps(res), flush=True)
    return 0


# the paper's largest instances that fit one GB300 (Minerva, Table 7: FWHT
# median seconds on 64 cores, FP64): name, n, c_d, c_b, d, log2 b, seconds
PAPER_ROWS = [
    ("Logunit", 1 << 15, 0.25, 0.25, 3, 13, 1.0),
    ("Logunit", 1 << 16, 0.25, 0.25, 5, 14, 7.8),
    ("Diagonal", 1 << 15, 0.75, 4.00, 11, 17, 11.4),
    ("Covariance", 1 << 15, 1.50, 4.00, 23, 17, 23.8),
    ("Lightbulb", 1 << 15, 2.00, 4.00, 31, 17, 32.0),
    ("Lightbulb", 1 << 16, 2.00, 4.00, 33, 18, 161.1),
]


def run_paper(a):
    """The paper's instance sizes (n, d, b of its Table 7 rows up to n = 2^16):
    Compress + Decompress of every entry on one GB300, FP32 butterflies and the
    exact fixed-point form (within the FP64 tolerance: the paper's precision),
    and the plain FP64 form where it takes a few seconds, next to the paper's FWHT
    median on 64 CPU cores.  The time depends on (n, d, b) only, so the
    operands are N(0,1) FP64 matrices of the instance's size (context, not the
    instances' values)."""
    import torch
    from paper_2601_09477_gb300 import cmm
    torch.cuda.set_device(0)
    rows = []
    cur_n, A, B, C = None, None, None, None
    for name, n, cd, cb, d, L, paper_s in PAPER_ROWS:
        if n != cur_n:
            A = B = C = None
            torch.cuda.empty_cache()
            g = torch.Generator(device="cuda")
            g.manual_seed(n)
            A = torch.randn((n, n), generator=g, dtype=torch.float64, device="cuda")
            B = torch.randn((n, n), generator=g, dtype=torch.float64, device="cuda")
            C = torch.empty((n, n), dtype=torch.float64, device="cuda")
            cur_n = n
        h = cmm.make_hashes(4000 + d, d, L)
        row = {"instance": name, "n": n, "c_d": cd, "c_b": cb, "d": d, "log2b": L,
               "paper_fwht_s_64_cores": paper_s}
        butterflies = d * n * 2.0 * (1 << L) * L
        # the exact fixed-point form (the FP64 tolerance, the paper's precision)
        # always; the plain FP64 form where its butterflies take a few seconds
        precs = ["f32", "fx64"] + (["f64"] if butterflies / 0.45e12 < 3.0 else [])
        for prec in precs:
            ws = torch.empty(cmm.multiply_workspace_bytes(n, n, n, h, torch.float64, prec),
                             dtype=torch.uint8, device="cuda")
            fn = lambda: cmm.multiply(A, B, h, prec=prec, out=C, ws=ws)
            fn()
            ms = _events_ms(fn, 1)
            row[prec + "_s"] = round(ms / 1e3, 4)
            row[prec + "_speedup_vs_paper"] = round(paper_s / (ms / 1e3), 1)
            del ws
        rows.append(row)
    res = {"metric": "paper-scale instances: Compress + Decompress seconds on one GB300 vs the "
                     "paper's FWHT median on 64 CPU cores (context)",
           "value": rows[-1]["f32_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "sizes of the paper's Table 7 rows up to n=2^16, N(0,1) FP64 "
                                  "operands, d and b from the paper's parameter rule",
                      "l2": l2_note(2 * 2**15 * 2**15 * 8)},
           "rows": rows}
    print(json.dumps(res), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batched":
        return run_batched(a)
    if a.workload == "precision":
        return run_precision(a)
    if a.workload == "diff":
        return run_diff(a)
    if a.workload == "cyclic":
        return run_cyclic(a)
    if a.workload == "paper":
        return run_paper(a)
    if a.workload == "instances":
        return run_instances(a)
    return run_cmm(a)


if __name__ == "__main__":
    sys.exit(main())
