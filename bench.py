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
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "sketch_f32_n8192_traffic.json")
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
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=10)
    return ap.parse_args()


def workload_config(a):
    return {
        "workload": "planted +-1 correlations n=%d (64 row pairs, rho=0.9, B=A^T, FP64 storage), "
                    "b=2^%d, d=%d, median, heavy hitters |C|>=n/2" % (a.n, a.log2b, a.d),
        "n": a.n, "m": a.n, "k": a.n, "p": a.n, "log2b": a.log2b, "d": a.d,
        "tau": a.n / 2, "input_dtype": "f64", "l2": "inputs (%.0f MiB) larger than L2" %
        (2 * a.n * a.n * 8 / 2**20), "parallelism": "replicas (one problem per GPU)",
    }


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured", pk
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", {}


def source_hash():
    h = hashlib.sha256()
    for name in ["sketch_impl.cuh", "fwht_device.cuh", "sketch_f32.cu", "sketch_tm.cu"]:
        with open(os.path.join(ROOT, "paper_2601_09477_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

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


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
    sample = ("Compress on %d of %d inner indices, Decompress of %d of %d rows, FP64, %d threads; "
              "scaled linearly to the full step" % (k_sample, n, rows_sample, n, threads))
    return ms, sample, (t2 - t0)


def run_reference(a):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_2601_09477_gb300 import workloads as wl
    from oracle import oracle as orc
    A, B, _ = wl.planted_pm1(n=a.n, pairs=64, rho=0.9, seed=1002)
    hp = orc.draw_hashes(2002, a.d)
    threads = orc.max_threads()
    k_s = max(16, a.n // 64)
    rows_s = max(16, a.n // 256)
    times = []
    for it in range(a.warmup + a.steps):
        ms, sample, _ = oracle_sample(A, B, hp, a.log2b, a.n, a.d, a.n / 2, k_s, rows_s, threads)
        if it >= a.warmup:
            times.append(ms)
    v = float(np.mean(times))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms",
           "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(v, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(a),
           "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": threads,
                            "kind": "oracle", "sample": sample},
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

    def step(prec):
        cmm.multiply(A, B, h, prec=prec, R=R, out=C, ws=ws)
        return cmm.threshold(C, tau, capacity=cap)

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
    w0 = time.perf_counter()
    e0.record(stream)
    for _ in range(a.steps):
        I, J, V = step(a.prec)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    barrier()
    cmm.trace_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    trace = cmm.trace_read()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

    # heavy-hitter evaluation (the off-diagonal filter is part of the evaluation)
    Ih, Jh = I.cpu().numpy(), J.cpu().numpy()
    found = set(zip(Ih.tolist(), Jh.tolist()))
    planted = {(int(i), int(j)) for i, j in pairs} | {(int(j), int(i)) for i, j in pairs}
    offdiag = sum(1 for (i, j) in found if i != j)
    recall = sum(1 for q in planted if q in found) / len(planted)

    # dominant kernel and its roofline (ALU-bound FP32 butterflies)
    sk_name = "sketch_" + a.prec
    launches = sum(v[0] for v in trace.values())
    sk_launches, sk_ms_total = trace.get(sk_name, (0, 0.0))
    sk_ms = sk_ms_total / max(sk_launches, 1)
    b = 1 << L
    ops = d * n * (2.0 * b * L + b)   # butterfly add/sub of both sketches + one FMA per bucket
    hbm_gbs, hbm_kind, pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12   # Tops/s
    achieved = ops / (sk_ms * 1e-3) / 1e12
    traffic = None
    try:
        with open(TRAFFIC_PATH) as f:
            tj = json.load(f)
        if tj.get("source_hash") == source_hash() and tj.get("n") == n and tj.get("log2b") == L:
            traffic = tj.get("dram_bytes_per_launch")
    except Exception:
        pass
    roofline = {"bound": "alu", "kernel": sk_name, "achieved": round(achieved, 3),
                "peak": round(alu_peak, 3), "unit": "Tops/s", "frac": round(achieved / alu_peak, 4),
                "traffic": traffic, "ops_per_launch": ops,
                "peak_source": "152 SMs x 128 FP32 lanes x %.0f MHz max SM clock" % sm_max,
                "avg_launch_ms": round(sk_ms, 4)}
    ab_bytes = 2.0 * n * n * 8
    hbm = {"bytes_A_B": ab_bytes, "achieved_gbs": round(ab_bytes / (ms * 1e-3) / 1e9, 2),
           "peak_gbs": hbm_gbs, "peak_kind": hbm_kind,
           "frac": round(ab_bytes / (ms * 1e-3) / 1e9 / hbm_gbs, 5)}

    result = {"metric": METRIC, "value": round(ms / world, 4), "unit": "ms", "n_gpus": world,
              "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 4),
              "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
              "dtype": a.prec, "data": "synthetic", "config": workload_config(a),
              "roofline": roofline, "hbm_roofline": hbm, "gpu_launches": int(launches),
              "clocks": clk, "kernels_ms_per_step": {k: round(v[1] / a.steps, 4)
                                                     for k, v in sorted(trace.items())},
              "heavy_hitters": {"count": int(len(Ih)), "offdiag": offdiag,
                                "planted_recall": recall},
              "wall_s_timed": round(wall, 3)}

    # plain FP64 form on the same input: time and R agreement
    if not a.no_fp64 and a.prec != "f64":
        R32 = R.clone()
        step("f64")
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        step("f64")
        f1.record(stream)
        torch.cuda.synchronize()
        f64_ms = f0.elapsed_time(f1)
        dR = float((R32 - R).abs().max().item())
        result["fp64"] = {"ms_per_step": round(f64_ms, 3), "speedup": round(f64_ms / ms, 2),
                          "max_abs_R_diff_vs_fp32": dR,
                          "equal_error": dR == 0.0}

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
        for _ in range(2):
            cmm.multiply_host(Ah, Bh, h, prec=a.prec, out=Ch, tau=tau, capacity=cap,
                              hh_out=hh, ws=wsh)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            _, (Ie, Je, Ve) = cmm.multiply_host(Ah, Bh, h, prec=a.prec, out=Ch, tau=tau,
                                                capacity=cap, hh_out=hh, ws=wsh)
        e2e_ms = (time.perf_counter() - t0) * 1e3 / a.e2e_steps
        nhh = int(Ie.numel())
        result["e2e"] = {"value": round(e2e_ms / world, 3), "unit": "ms",
                         "h2d_bytes_per_step": int(2 * n * n * 8),
                         "d2h_bytes_per_step": int(n * n * 8 + nhh * 16),
                         "ms_per_step": round(e2e_ms, 3), "steps": a.e2e_steps,
                         "api": "cmm_multiply_host (pinned host A, B, C, heavy-hitter list)"}
        del wsh

    # FP64 CPU oracle on a bounded sample (rank 0, single GPU only)
    if not a.no_cpu and rank == 0 and world == 1:
        from oracle import oracle as orc
        threads = orc.max_threads()
        cpu_ms, sample, secs = oracle_sample(A_np, B_np, h.params, L, n, d, tau,
                                             max(16, n // 4), max(16, n // 16), threads)
        result["cpu_baseline"] = {"value": round(cpu_ms, 1), "unit": "ms", "cores": threads,
                                  "kind": "oracle", "sample": sample,
                                  "sample_seconds": round(secs, 2)}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_cmm(a)


if __name__ == "__main__":
    sys.exit(main())
