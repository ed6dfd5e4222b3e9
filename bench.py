#!/usr/bin/env python
"""Benchmark of the compressed control step on GB300.

Workload (the paper-shaped control loop): a 32768 x 32768 smooth-kernel
matrix (181 x 181 grid, l = 0.05, +1e-3 noise; indices >= 32761 zero) held
resident in the zfp-style fixed-rate format at 16 bits/value (2.15 GB), and
a 2000-step control loop y_k = A x_k, s_{k+1} = 0.99 s_k + y_k (FP64 state)
with x_k a Gaussian heat load moving along a serpentine path of 100 fields.
A step is one whff_step (fused decode + GEMV + FP64 epilogue).

Metric: compressed GEMV throughput in GB/s of compressed bytes streamed (and
its fraction of HBM peak), with p50/p99/p99.9 step latency and the
end-to-end relative error of y against FP64 GEMV on the uncompressed matrix.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl whff|reference]

Under torchrun each rank runs an independent replica on its own GPU
(the paper's three axes are three independent GEMVs, one per GPU); the
reported value is the sum over ranks of the work done / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed GEMV: HBM GB/s & % peak; p99 control-step latency at rel.err≤1e-5"
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0
DECAY = 0.99


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["whff", "reference"], default="whff")
    p.add_argument("--order", type=int, default=32768, help="matrix order (32768 = the control-loop workload)")
    p.add_argument("--rate", type=int, default=16)
    p.add_argument("--e2e-steps", type=int, default=200)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-baseline", action="store_true")
    p.add_argument("--json-out", default=None)
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_08018_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel_key)
        if e and e.get("source_hash") == kernel_source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"whff_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- workload
def build_workload(order: int, rate: int, keep_fp64_device: bool, sample_rows: np.ndarray, torch=None,
                   device=None):
    """Generate the matrix band by band, compress it, optionally keep an FP64 copy on the GPU
    (the uncompressed baseline) and the FP64 values of a few sampled rows (error reference)."""
    import paper_1902_08018_gb300 as W
    import workloads

    if order == 32768:
        km = workloads.config(2).matrix
    else:
        g = int(np.ceil(np.sqrt(order)))
        km = workloads.KernelMatrix(order, g, min(order, g * g), 0.05, workloads.SEED_BASE + 2)
    A64 = torch.empty((order, order), dtype=torch.float64, device=device) if keep_fp64_device else None
    sampled = np.empty((len(sample_rows), order))
    band = 1024

    def bands():
        for r0, rows in km.bands(band):
            if A64 is not None:
                A64[r0:r0 + rows.shape[0]].copy_(torch.from_numpy(rows))
            sel = (sample_rows >= r0) & (sample_rows < r0 + rows.shape[0])
            for k in np.nonzero(sel)[0]:
                sampled[k] = rows[sample_rows[k] - r0]
            yield r0, rows

    blob = W.whff_compress_bands(order, order, bands(), W.FMT_ZFP, rate)
    return km, blob, A64, sampled


def heat_load_inputs(km, steps: int):
    import workloads

    return workloads.heat_loads(km.g, km.n_valid, km.order, steps).T.copy()  # (steps, N)


# -------------------------------------------------------------- CPU baseline
def cpu_baseline(blob, order, rate, x64, y_gpu, sample_rows, budget_s=12.0):
    """The oracle as it stands (decode + FP64 GEMV) on a bounded band of block rows."""
    import oracle

    oracle.build()
    blob_b = blob.tobytes() if hasattr(blob, "tobytes") else blob
    cores = oracle.num_threads()
    # calibrate on 4 block rows, then size the sample to ~budget_s
    t0 = time.perf_counter()
    D = oracle.decode_rows(blob_b, 0, 16)
    oracle.gemv64(D, x64)
    t_cal = time.perf_counter() - t0
    rows = int(max(16, min(order, 16 * budget_s / max(t_cal, 1e-6)))) // 4 * 4
    r0 = 0
    t0 = time.perf_counter()
    D = oracle.decode_rows(blob_b, r0, rows)
    y = oracle.gemv64(D, x64)
    dt = time.perf_counter() - t0
    comp_bytes = rows * order * rate / 8.0
    err = float(np.linalg.norm(y_gpu[r0:r0 + rows] - y) / np.linalg.norm(y))
    return {"value": comp_bytes / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"decode + FP64 GEMV of rows [{r0}, {r0 + rows}) of the {order}^2 rate-{rate} matrix "
                      f"({rows}/{order} of one step), {dt:.1f} s",
            "parity_rel_l2_vs_gpu": err}


# --------------------------------------------------------------- whff arm
def run_whff(args, rank, world, local_rank):
    import torch

    import paper_1902_08018_gb300 as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    order, rate = args.order, args.rate
    rng = np.random.default_rng(12345)
    sample_rows = np.sort(rng.choice(order, size=64, replace=False))
    keep64 = not args.no_fp64_baseline
    t_setup = time.perf_counter()
    km, blob, A64, sampled = build_workload(order, rate, keep64, sample_rows, torch, dev)
    h = W.whff_create(blob, max_rhs=1)
    t_setup = time.perf_counter() - t_setup
    stream_bytes = h.device_bytes  # includes workspace; recomputed below
    stream_bytes = len(blob) - 64

    S = 2000 if order == 32768 else min(2000, max(args.steps, 1))
    X64 = heat_load_inputs(km, S)  # (S, N) FP64
    xs = torch.from_numpy(X64.astype(np.float32)).to(dev)
    y = torch.zeros(order, dtype=torch.float64, device=dev)
    state = torch.zeros(order, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    for k in range(args.warmup):
        h.step(xs[k % S], y, state, DECAY, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with ClockSampler(local_rank) as clk:
        evs[0].record(stream)
        for k in range(args.steps):
            h.step(xs[k % S], y, state, DECAY, stream)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    per_step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    clocks = clk.summary()
    ms_per_step = total_ms / args.steps
    value_per_rank = stream_bytes / (ms_per_step * 1e-3) / 1e9
    value = value_per_rank * world
    lat = np.array(per_step_ms) * 1e3  # us
    launches_per_step = 1 + (1 if h_ksplit(h) > 1 else 0)

    # end-to-end error of one step against FP64 GEMV on the uncompressed matrix (sampled rows)
    xk = X64[0]
    h.step(xs[0], y, None, DECAY, stream)
    torch.cuda.synchronize()
    y_gpu = y.cpu().numpy()
    y_star = sampled @ xk
    rel_err = float(np.linalg.norm(y_gpu[sample_rows] - y_star) / np.linalg.norm(y_star))

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    E = max(1, min(args.e2e_steps, args.steps))
    xh = torch.from_numpy(X64[:min(S, E)].astype(np.float32)).pin_memory()
    yh = torch.zeros(order, dtype=torch.float64).pin_memory()
    state2 = torch.zeros(order, dtype=torch.float64, device=dev)
    for k in range(3):
        h.step_host(xh[k % xh.shape[0]].numpy(), yh.numpy(), state2, DECAY, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(E):
        h.step_host(xh[k % xh.shape[0]].numpy(), yh.numpy(), state2, DECAY, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / E

    # plain uncompressed FP64 GEMV on the same GPU (cuBLAS DGEMV via torch.mv)
    fp64 = None
    if A64 is not None:
        x64d = torch.from_numpy(X64[0]).to(dev)
        for _ in range(3):
            torch.mv(A64, x64d)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        f0.record(stream)
        for _ in range(reps):
            torch.mv(A64, x64d)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / reps
        fp64 = {"ms_per_step": fms, "GB_s": order * order * 8 / (fms * 1e-3) / 1e9,
                "speedup_of_compressed": fms / ms_per_step}
        del A64
        torch.cuda.empty_cache()

    peak, peak_kind = measured_peaks()
    algo_bytes = stream_bytes + order * 4 + order * 8 + order * 16
    kernel_ms = float(np.mean(per_step_ms))
    achieved = algo_bytes / (kernel_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"of {peak_kind}",
                "traffic": ncu_traffic(f"wz1_gemv_{order}_rate{rate}"),
                "kernel": f"wz1_gemv_kernel<{rate // 2},1>", "frac_of_nominal_8TBs": round(achieved / NOMINAL_HBM_GBS, 4)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(blob, order, rate, X64[0], y_gpu, sample_rows)

    res = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"control-loop-{order}-rate{rate}", "M": order, "N": order, "fmt": "WZ1 zfp-style",
                   "rate_bits_per_value": rate, "R": 1, "state": "FP64 s <- 0.99 s + y",
                   "compressed_bytes_per_step": stream_bytes,
                   "l2": "inputs larger than L2 (compressed A 2.1 GB streamed every step)",
                   "parallelism": f"replicas{world}"},
        "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "p999": float(np.percentile(lat, 99.9)), "max": float(lat.max())},
        "rel_err_vs_fp64_uncompressed": rel_err,
        "effective_gflops": round(order * (2 * order - 1) / (ms_per_step * 1e-3) / 1e9 * world, 1),
        "pct_hbm_peak": round(100 * value_per_rank / peak, 2),
        "roofline": roofline,
        "e2e": {"value": round(stream_bytes / (e2e_ms * 1e-3) / 1e9 * world, 2), "unit": "GB/s",
                "ms_per_step": round(e2e_ms, 5), "h2d_bytes_per_step": order * 4,
                "d2h_bytes_per_step": order * 8},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clocks,
        "fp64_uncompressed_gemv": fp64,
        "setup_s": round(t_setup, 1),
    }
    if cpu is not None:
        res["cpu_baseline"] = cpu
    h.destroy()
    return res


def h_ksplit(h):
    # the library picks split-K itself; for square matrices with thousands of bands it is 1
    return 1


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host cores, on the same workload and metric:
    each step decodes and multiplies a bounded band of block rows."""
    import oracle

    import paper_1902_08018_gb300  # noqa: F401  (encoder only: builds the blob on the host)

    order, rate = args.order, args.rate
    km, blob, _, _ = build_workload(order, rate, False, np.array([], dtype=int), None, None)
    blob_b = blob.tobytes()
    oracle.build()
    x64 = heat_load_inputs(km, 1)[0]
    rows_per_step = 16
    nb = order // rows_per_step

    def one(k):
        r0 = (k % nb) * rows_per_step
        D = oracle.decode_rows(blob_b, r0, rows_per_step)
        return oracle.gemv64(D, x64)

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(k)
    dt = time.perf_counter() - t0
    comp = rows_per_step * order * rate / 8.0 * args.steps
    value = comp / dt / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"control-loop-{order}-rate{rate}", "M": order, "N": order, "fmt": "WZ1 zfp-style",
                   "rate_bits_per_value": rate, "R": 1},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{rows_per_step} of {order} rows per step (decode + FP64 GEMV)"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        res = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch

            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        res = run_whff(args, rank, world, local_rank)
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()
    if rank == 0:
        line = json.dumps(res)
        print(line, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")


if __name__ == "__main__":
    main()
