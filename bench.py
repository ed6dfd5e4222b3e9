#!/usr/bin/env python
"""Benchmark of the compressed control step on GB300.

Workload (the paper-shaped control loop): a 32768 x 32768 smooth-kernel
matrix (181 x 181 grid, l = 0.05, +1e-3 noise; indices >= 32761 zero) held
resident at 16 bits/value (2.15 GB), and a 2000-step control loop
y_k = A x_k, s_{k+1} = 0.99 s_k + y_k (FP64 state) with x_k a Gaussian heat
load moving along a serpentine path of 100 fields.  One step = one whff_step
(fused decode + GEMV + FP64 epilogue).

Metric: GB/s of compressed bytes streamed per step (and its fraction of
the measured HBM peak), with p50/p99/p99.9 step latency and the end-to-end
relative error of y against FP64 GEMV on the uncompressed matrix.  The
headline format is the fixed-allocation zfp-style variant (--fmt); the
embedded-coder format, other rates and the scaled formats are measured on
the same matrix in the same run (--sweep), and the p99 latency is also
reported for the lowest-byte format whose error is <= 1e-5.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl whff|reference]

Under torchrun each rank runs an independent replica on its own GPU (the
paper's three axes are three independent GEMVs, one per GPU); value = the
sum over ranks of bytes streamed / the max-over-ranks time.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed GEMV: HBM GB/s & % peak; p99 control-step latency at rel.err≤1e-5"
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0
DECAY = 0.99
FMT_CODES = {"wz1": 1, "bf16": 2, "fp16": 3, "fp8": 4, "wz2-lift": 5, "wz2-bfp": 6, "fp32": 7, "wz3": 8}
FMT_NAMES = {v: k for k, v in FMT_CODES.items()}
ERR_TARGET = 1e-5


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["whff", "reference"], default="whff")
    p.add_argument("--order", type=int, default=32768, help="matrix order (32768 = the control-loop workload)")
    p.add_argument("--fmt", default="wz2-lift", choices=sorted(FMT_CODES))
    p.add_argument("--rate", type=int, default=16)
    p.add_argument("--sweep", default="wz1:16,wz2-lift:8,wz2-lift:12,wz2-bfp:16,wz2-lift:20,wz2-bfp:20,wz2-lift:24,"
                                      "fp8:0,fp16:0,bf16:0,wz3:1e-7",
                   help="extra fmt:rate pairs timed on the same matrix ('' for none; wz3 takes its "
                        "absolute tolerance in place of a rate)")
    p.add_argument("--sweep-steps", type=int, default=400)
    p.add_argument("--sweep-rhs", type=int, default=1, help="1: also time every sweep format with 32 right-hand sides")
    p.add_argument("--e2e-steps", type=int, default=200)
    p.add_argument("--rhs-sweep", default="8,16,32",
                   help="right-hand-side counts timed on the headline matrix, on both engines")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-baseline", action="store_true")
    p.add_argument("--no-host-resident", action="store_true", help="skip the matrix-over-the-link leg")
    p.add_argument("--no-tune", action="store_true", help="time the default launch shape instead of whff_tune's")
    p.add_argument("--no-slits", action="store_true", help="skip the moving-slit graph leg")
    p.add_argument("--slit-steps", type=int, default=2000)
    p.add_argument("--no-fields", action="store_true", help="skip the streamed-field pipeline leg")
    p.add_argument("--launch-shape", default="",
                   help="unroll,ctas_per_sm,fold for the headline WZ2 handle instead of tuning (e.g. 4,3,1)")
    p.add_argument("--json-out", default=None)
    p.add_argument("--serve", action="store_true", help="run the serving workload instead of the control loop")
    p.add_argument("--serve-fmt", default="wz2-lift:8")
    p.add_argument("--serve-orders", default="8192,16384,32768,49152,65536,65536,32768,16384")
    p.add_argument("--serve-seconds", type=float, default=2.0)
    p.add_argument("--serve-hz", type=float, default=2000.0)
    p.add_argument("--deadline-us", type=float, default=500.0)
    p.add_argument("--firm", type=int, default=1, help="1: drop requests past their deadline (firm real time)")
    p.add_argument("--shapes", action="store_true",
                   help="the paper's three GEMV shapes (wide, tall, square) in FP32 and compressed formats")
    p.add_argument("--shapes-fmts", default="fp32:0,wz2-lift:16,wz2-lift:12,wz1:16,bf16:0")
    p.add_argument("--precision", action="store_true",
                   help="the precision sweep: every format at 1 and 32 right-hand sides on the control-loop matrix")
    p.add_argument("--precision-fmts",
                   default="wz1:8,wz1:12,wz1:16,wz2-lift:8,wz2-lift:12,wz2-lift:16,wz2-bfp:8,wz2-bfp:12,wz2-bfp:16,"
                           "bf16:0,fp16:0,fp8:0")
    p.add_argument("--batched", action="store_true", help="run the batched uneven-instances workload")
    p.add_argument("--batched-fmt", default="wz2-lift:12")
    p.add_argument("--batched-crossover", type=int, default=0,
                   help="fewest columns of a tensor-core pass for the batch's handles (0: their default)")
    p.add_argument("--no-serve-leg", action="store_true",
                   help="leave the bounded serving and batched runs out of the default line")
    return p.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("gemv_kernels.cuh", "wz1_decode.cuh", "wz2_kernels.cuh", "wz2_dispatch.cuh", "wz2_stream.cuh", "bulk.cuh")


def kernel_source_hash():
    """Hash of the device-kernel sources the ncu counters in profiles/ were taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_08018_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            e = json.load(f).get(kernel_key)
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
        self.path = os.path.join("/tmp", f"whff_clocks_{os.getpid()}_{id(self)}.csv")
        self._summary = None

    def __enter__(self):
        self.fh = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if self.fh:
                self.fh.close()
                try:
                    os.remove(self.path)
                except OSError:
                    pass
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
        """Median SM clock, the largest maximum clock, median power and the throttle
        reasons seen (read once; the sample file is removed afterwards)."""
        if self._summary is None:
            self._summary = self._read()
        return self._summary

    def _read(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [s.strip() for s in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ multi-rank
def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's time (every rank gets it); one process: x itself."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_step_per_rank: float, ms_per_step: float, world: int) -> float:
    """Replicas: every rank streams its own matrix each step; GB/s of all ranks over the slowest time."""
    return bytes_per_step_per_rank * world / (ms_per_step * 1e-3) / 1e9


def psnr_db(nrmse: float) -> float:
    """PSNR of Table 2: 20 log10(range / (2 RMSE)) = -20 log10(2 NRMSE), NRMSE = RMSE / range."""
    return float("inf") if nrmse == 0 else -20.0 * math.log10(2.0 * nrmse)


def table2_metrics(A: np.ndarray, Ahat: np.ndarray, stored_bytes: int, values: int) -> dict:
    """The columns of Table 2 for a decoded matrix (or a sample of its rows) against the
    matrix it encodes: bits per value and Rate = 32 / bits per value (the FP32 matrix's
    size over the stored size), RMSE, NRMSE = RMSE / (max - min), the largest pointwise
    error and PSNR."""
    d = Ahat.astype(np.float64) - A.astype(np.float64)
    rmse = float(np.sqrt(np.mean(d * d)))
    span = float(A.max() - A.min())
    nrmse = rmse / span if span > 0 else 0.0
    bpv = 8.0 * stored_bytes / values
    return {"bits_per_value": round(bpv, 3), "rate": round(32.0 / bpv, 2), "rmse": rmse, "nrmse": nrmse,
            "max_pointwise_error": float(np.abs(d).max()),
            "psnr_db": round(psnr_db(nrmse), 2) if nrmse > 0 else None}  # None: lossless (strict JSON has no inf)


# ----------------------------------------------------------------- workload
def parse_specs(args):
    specs = [(FMT_CODES[args.fmt], args.rate)]
    for item in filter(None, args.sweep.split(",")):
        name, rate = item.split(":")
        code = FMT_CODES[name]
        spec = (code, float(rate) if code == 8 else int(rate) if code in (1, 5, 6) else 0)
        if spec not in specs:
            specs.append(spec)
    return specs


def matrix_for(order: int):
    import workloads

    if order == 32768:
        return workloads.config(2).matrix
    g = int(np.ceil(np.sqrt(order)))
    return workloads.KernelMatrix(order, g, min(order, g * g), 0.05, workloads.SEED_BASE + 2)


def build_workload(order: int, specs, keep_fp64_device: bool, sample_rows: np.ndarray, torch=None, device=None):
    """Generate the matrix band by band and compress every band into every requested
    format; optionally keep an FP64 copy on the GPU (the uncompressed baseline) and the
    FP64 values of a few sampled rows (reference for the end-to-end error)."""
    import paper_1902_08018_gb300 as W

    km = matrix_for(order)
    L = W.library()
    blobs = {}
    accuracy = [spec for spec in specs if spec[0] == 8]  # fixed accuracy: its bands appended in row order
    acc_bufs = {}
    for spec in accuracy:
        cap = int(L.whff_accuracy_max_size(order, order))
        acc_bufs[spec] = np.empty(cap, dtype=np.uint8)  # untouched pages are never backed
        if L.whff_accuracy_begin(acc_bufs[spec].ctypes.data, cap, order, order, float(spec[1])) != 0:
            raise RuntimeError(L.whff_last_error().decode())
    for fmt, rate in specs:
        if fmt == 8:
            continue
        n = W.compressed_size(fmt, rate, order, order)
        b = np.empty(n, dtype=np.uint8)
        if L.whff_blob_init(b.ctypes.data, n, fmt, rate, order, order) != 0:
            raise RuntimeError(f"blob init failed for {fmt}:{rate}")
        blobs[(fmt, rate)] = b
    A64 = torch.empty((order, order), dtype=torch.float64, device=device) if keep_fp64_device else None
    sampled = np.empty((len(sample_rows), order))
    for r0, rows in km.bands(1024):
        if A64 is not None:
            A64[r0:r0 + rows.shape[0]].copy_(torch.from_numpy(rows))
        for spec, buf in acc_bufs.items():
            if L.whff_compress_accuracy_band(buf.ctypes.data, buf.size, rows.ctypes.data, r0, rows.shape[0], order,
                                             0) != 0:
                raise RuntimeError(L.whff_last_error().decode())
        sel = (sample_rows >= r0) & (sample_rows < r0 + rows.shape[0])
        for k in np.nonzero(sel)[0]:
            sampled[k] = rows[sample_rows[k] - r0]
        for b in blobs.values():
            e = L.whff_compress_band(b.ctypes.data, b.size, rows.ctypes.data, r0, rows.shape[0], order, 0)
            if e != 0:
                raise RuntimeError(L.whff_last_error().decode())
    for b in blobs.values():
        L.whff_blob_seal(b.ctypes.data, b.size)
    for spec, buf in acc_bufs.items():
        used = ctypes.c_size_t()
        if L.whff_accuracy_seal(buf.ctypes.data, buf.size, ctypes.byref(used)) != 0:
            raise RuntimeError(L.whff_last_error().decode())
        blobs[spec] = buf[: used.value].copy()
    del acc_bufs
    return km, blobs, A64, sampled


def heat_load_inputs(km, steps: int):
    import workloads

    return workloads.heat_loads(km.g, km.n_valid, km.order, steps).T.copy()  # (steps, N)


# -------------------------------------------------------------- CPU baseline
def cpu_baseline(blob, order, rate_bits, x64, y_gpu, budget_s=12.0):
    """The oracle as it stands (decode + FP64 GEMV) on a bounded band of block rows."""
    import oracle

    oracle.build()
    blob_b = blob.tobytes()
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    D = oracle.decode_rows(blob_b, 0, 16)
    oracle.gemv64(D, x64)
    t_cal = time.perf_counter() - t0
    rows = int(max(16, min(order, 16 * budget_s / max(t_cal, 1e-6)))) // 4 * 4
    t0 = time.perf_counter()
    D = oracle.decode_rows(blob_b, 0, rows)
    y = oracle.gemv64(D, x64)
    dt = time.perf_counter() - t0
    comp_bytes = rows * order * rate_bits / 8.0
    err = float(np.linalg.norm(y_gpu[:rows] - y) / np.linalg.norm(y))
    return {"value": comp_bytes / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"decode + FP64 GEMV of rows [0, {rows}) of the {order}^2 matrix "
                      f"({rows}/{order} of one step, {dt:.1f} s)",
            "parity_rel_l2_vs_gpu": err}


# --------------------------------------------------------------- whff arm
def time_format(h, xs, S, steps, warmup, stream, torch, dev, order, with_clocks=None):
    y = torch.zeros(order, dtype=torch.float64, device=dev)
    state = torch.zeros(order, dtype=torch.float64, device=dev)
    for k in range(warmup):
        h.step(xs[k % S], y, state, DECAY, stream)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        h.step(xs[k % S], y, state, DECAY, stream)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(steps)])
    total = evs[0].elapsed_time(evs[-1])
    return total, per


def rhs32_entry(h, spec, sb, X, X64, sampled, sample_rows, peak, stream, torch, dev, order, reps=20):
    """One pass of 32 right-hand sides: time, stored-byte rate, engine, worst column error vs FP64."""
    R = X.shape[0]
    Y = torch.zeros((R, order), dtype=torch.float64, device=dev)
    for _ in range(3):
        h.step(X, Y, None, DECAY, stream)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        h.step(X, Y, None, DECAY, stream)
    f1.record(stream)
    torch.cuda.synchronize()
    ms = f0.elapsed_time(f1) / reps
    Yh = Y.cpu().numpy()[:, sample_rows].T
    Ys = sampled @ X64.T
    err = max(float(np.linalg.norm(Yh[:, r] - Ys[:, r]) / np.linalg.norm(Ys[:, r])) for r in range(R))
    engine = "tcgen05" if (spec[0] in (2, 3, 4, 5, 6) and R >= h.crossover) else "cuda-core"
    return {"ms_per_step": round(ms, 4), "GB_s": round(sb / (ms * 1e-3) / 1e9, 1),
            "pct_hbm": round(100 * sb / (ms * 1e-3) / 1e9 / peak, 2),
            "effective_tflops": round(R * order * (2 * order - 1) / (ms * 1e-3) / 1e12, 2), "engine": engine,
            "rel_err": err}


def achievable_read(W, torch, dev, stream, nbytes: int, reps: int = 20) -> float:
    """GB/s of the library's read-only streaming probe over a buffer the size of the
    compressed stream (larger than L2): the third roofline line, beside the copy peak
    and the nominal figure."""
    buf = torch.ones(nbytes // 16 * 16, dtype=torch.uint8, device=dev)
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(3):
        W.whff_read_probe(buf, out, stream)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(reps):
        W.whff_read_probe(buf, out, stream)
    f1.record(stream)
    torch.cuda.synchronize()
    gbs = buf.numel() * reps / (f0.elapsed_time(f1) * 1e-3) / 1e9
    del buf
    torch.cuda.empty_cache()
    return gbs


def end_to_end_error(h, xs, X64, sampled, sample_rows, stream, torch, dev, order):
    y = torch.zeros(order, dtype=torch.float64, device=dev)
    h.step(xs[0], y, None, DECAY, stream)
    torch.cuda.synchronize()
    y_gpu = y.cpu().numpy()
    y_star = sampled @ X64[0]
    return float(np.linalg.norm(y_gpu[sample_rows] - y_star) / np.linalg.norm(y_star)), y_gpu


def run_whff(args, rank, world, local_rank):
    import torch

    import paper_1902_08018_gb300 as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    order = args.order
    specs = parse_specs(args)
    head = specs[0]
    rng = np.random.default_rng(12345)
    sample_rows = np.sort(rng.choice(order, size=64, replace=False))
    t_setup = time.perf_counter()
    km, blobs, A64, sampled = build_workload(order, specs, not args.no_fp64_baseline, sample_rows, torch, dev)
    t_setup = time.perf_counter() - t_setup

    S = 2000 if order == 32768 else min(2000, max(args.steps, 1))
    X64 = heat_load_inputs(km, S)  # (S, N) FP64
    xs = torch.from_numpy(X64.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()

    # ---------------- headline format: the timed control loop
    h = W.whff_create(blobs[head], max_rhs=1)
    stream_bytes = blobs[head].size - 64
    tuned = None
    if args.launch_shape and head[0] in (5, 6):  # a given shape (e.g. to profile the tuned instantiation alone)
        u, c, f = (int(v) for v in args.launch_shape.split(","))
        h.set_config(u, c, f)
        tuned = {"unroll": u, "ctas_per_sm": c, "fold": f}
    elif not args.no_tune and head[0] in (5, 6):  # the library's tuner picks the launch shape on this machine
        tuned = h.tune(iters=10, stream=stream)
    ksplit, launches = h.plan()
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clk:
        total_ms, per_ms = time_format(h, xs, S, args.steps, args.warmup, stream, torch, dev, order)
    total_ms = max_over_ranks(total_ms, world, dev)
    clocks = clk.summary()
    ms_per_step = total_ms / args.steps
    value = whole_job_gbs(stream_bytes, ms_per_step, world)
    lat = per_ms * 1e3
    rel_err, y_gpu = end_to_end_error(h, xs, X64, sampled, sample_rows, stream, torch, dev, order)

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    E = max(1, min(args.e2e_steps, args.steps))
    xh = torch.from_numpy(X64[:min(S, E)].astype(np.float32)).pin_memory()
    yh = torch.zeros(order, dtype=torch.float64).pin_memory()
    st2 = torch.zeros(order, dtype=torch.float64, device=dev)
    for k in range(3):
        h.step_host(xh[k % xh.shape[0]].numpy(), yh.numpy(), st2, DECAY, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(E):
        h.step_host(xh[k % xh.shape[0]].numpy(), yh.numpy(), st2, DECAY, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / E
    h.destroy()

    # ---------------- the other formats on the same matrix
    formats = {}
    head_name = f"{FMT_NAMES[head[0]]}-{head[1]}" if head[1] else FMT_NAMES[head[0]]
    formats[head_name] = {"GB_s": round(stream_bytes / (ms_per_step * 1e-3) / 1e9, 1),
                          "pct_hbm": round(100 * stream_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 2),
                          "bytes": int(stream_bytes), "ms_per_step": round(ms_per_step, 5),
                          "p99_us": float(np.percentile(lat, 99)), "rel_err": rel_err}
    for spec in specs[1:]:
        hh = W.whff_create(blobs[spec], max_rhs=32 if args.sweep_rhs else 1)
        shape = "default"
        if spec[0] in (5, 6) and not args.no_tune:  # WZ2: the launch shape the tuner picks, as for the headline
            hh.tune(iters=3, stream=stream)
            shape = dict(zip(("unroll", "ctas_per_sm", "fold"), hh.config()))
        sb = blobs[spec].size - 64
        tot, per = time_format(hh, xs, S, args.sweep_steps, 5, stream, torch, dev, order)
        err, _ = end_to_end_error(hh, xs, X64, sampled, sample_rows, stream, torch, dev, order)
        ms = tot / args.sweep_steps
        name = f"{FMT_NAMES[spec[0]]}-{spec[1]}" if spec[1] else FMT_NAMES[spec[0]]
        formats[name] = {"GB_s": round(sb / (ms * 1e-3) / 1e9, 1), "pct_hbm": round(100 * sb / (ms * 1e-3) / 1e9 / peak, 2),
                         "bytes": int(sb), "ms_per_step": round(ms, 5), "p99_us": float(np.percentile(per * 1e3, 99)),
                         "rel_err": err, "launch_shape": shape}
        if args.sweep_rhs:  # the same format with 32 right-hand sides (heat loads of steps 0..31)
            formats[name]["R32"] = rhs32_entry(hh, spec, sb, xs[:32], X64[:32], sampled, sample_rows, peak, stream,
                                               torch, dev, order)
        hh.destroy()
    # ---------------- many right-hand sides on the headline matrix, on both engines
    multi = {}
    sb = blobs[head].size - 64
    for Rm in [int(v) for v in filter(None, args.rhs_sweep.split(","))]:
        hh = W.whff_create(blobs[head], max_rhs=Rm)
        default_min = hh.crossover
        Xr = torch.from_numpy(np.random.default_rng(Rm).standard_normal((Rm, order)).astype(np.float32)).to(dev)
        Yr = torch.zeros((Rm, order), dtype=torch.float64, device=dev)
        entry = {"default_engine": "tcgen05" if Rm >= default_min else "cuda-core"}
        engines = [("cuda-core", 33)] + ([("tcgen05", 2)] if Rm >= 2 and default_min <= 32 else [])
        for eng, cross in engines:
            hh.crossover = cross
            for _ in range(3):
                hh.step(Xr, Yr, None, DECAY, stream)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(5, min(50, args.sweep_steps // 8))
            f0.record(stream)
            for _ in range(reps):
                hh.step(Xr, Yr, None, DECAY, stream)
            f1.record(stream)
            torch.cuda.synchronize()
            ms = f0.elapsed_time(f1) / reps
            entry[eng] = {"ms_per_step": round(ms, 4), "GB_s": round(sb / (ms * 1e-3) / 1e9, 1),
                          "pct_hbm": round(100 * sb / (ms * 1e-3) / 1e9 / peak, 2),
                          "effective_tflops": round(Rm * order * (2 * order - 1) / (ms * 1e-3) / 1e12, 2)}
        multi[str(Rm)] = entry
        hh.destroy()

    ok = [(v["bytes"], k) for k, v in formats.items() if v["rel_err"] <= ERR_TARGET]
    at_target = None
    if ok:
        _, best = min(ok)
        at_target = dict(formats[best], format=best)

    # ---------------- plain uncompressed FP64 GEMV on the same GPU (cuBLAS via torch.mv)
    fp64 = None
    if A64 is not None:
        x64d = torch.from_numpy(X64[0]).to(dev)
        for _ in range(3):
            torch.mv(A64, x64d)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 20
        f0.record(stream)
        for _ in range(reps):
            torch.mv(A64, x64d)
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / reps
        fp64 = {"ms_per_step": round(fms, 4), "GB_s": round(order * order * 8 / (fms * 1e-3) / 1e9, 1),
                "speedup_of_headline": round(fms / ms_per_step, 2)}
        del A64
        torch.cuda.empty_cache()

    # ---------------- the matrix streamed over the CPU-GPU link every step (Sec. 4.2: the
    # paper's system moves the matrix over the host link; compression divides its bytes)
    host = None
    if not args.no_host_resident:
        hh = W.whff_create(blobs[head], max_rhs=1, host_resident=True)
        xs0 = xs[0] if xs.dim() == 2 else xs
        yh = torch.zeros(order, dtype=torch.float64, device=dev)
        for _ in range(3):
            hh.step(xs0, yh, None, DECAY, stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        f0.record(stream)
        for _ in range(reps):
            hh.step(xs0, yh, None, DECAY, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        hms = f0.elapsed_time(f1) / reps
        hh.destroy()
        # the link's plain copy rate (pinned host -> HBM), and what an uncompressed FP64
        # matrix would cost per step over it
        hbuf = torch.empty(1 << 30, dtype=torch.uint8).pin_memory()
        dbuf = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        dbuf.copy_(hbuf, non_blocking=True)
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(3):
            dbuf.copy_(hbuf, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        link = 3 * (1 << 30) / (f0.elapsed_time(f1) * 1e-3) / 1e9
        del hbuf, dbuf
        torch.cuda.empty_cache()
        host = {"ms_per_step": round(hms, 4), "GB_s": round(stream_bytes / (hms * 1e-3) / 1e9, 1),
                "h2d_copy_GB_s": round(link, 1),
                "fp64_uncompressed_over_link_ms": round(order * order * 8 / (link * 1e9) * 1e3, 3),
                "note": "compressed stream in pinned host memory, read by the fused kernel over the link"}

    algo_bytes = stream_bytes + order * 4 + order * 8 + order * 16
    kernel_ms = float(np.mean(per_ms))  # one launch per step when ksplit == 1
    achieved = algo_bytes / (kernel_ms * 1e-3) / 1e9
    kname = {1: "wz1_gemv_kernel", 5: "wz2_gemv_kernel", 6: "wz2_gemv_kernel"}.get(head[0], "scaled_range_kernel")
    if tuned and head[0] in (5, 6) and tuned["fold"] & 4:  # bulk-staged kernel
        kname = "wz2_stream_kernel"
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"of {peak_kind}",
                "traffic": ncu_traffic(f"{head_name}_{order}"), "kernel": kname,
                "launches_per_step": launches, "frac_of_nominal_8TBs": round(achieved / NOMINAL_HBM_GBS, 4)}
    read_gbs = achievable_read(W, torch, dev, stream, stream_bytes)
    roofline["achievable_read_GB_s"] = round(read_gbs, 1)
    roofline["frac_of_achievable_read"] = round(achieved / read_gbs, 4)

    slits = fields = None
    if not args.no_slits:
        slits = slit_graph_leg(W, torch, blobs[head], order, xs, stream, steps=args.slit_steps)
    if not args.no_fields:
        fields = field_pipeline_leg(W, torch, dev, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(blobs[head], order, head[1] if head[1] else 16, X64[0], y_gpu)

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
        "config": {"workload": f"control-loop-{order}-rate{head[1]}", "M": order, "N": order,
                   "fmt": head_name, "rate_bits_per_value": head[1], "R": 1, "state": "FP64 s <- 0.99 s + y",
                   "compressed_bytes_per_step": int(stream_bytes), "ksplit": ksplit,
                   "launch_shape": ({k: tuned[k] for k in ("unroll", "ctas_per_sm", "fold")} if tuned
                                    else "default"),
                   "l2": "inputs larger than L2 (the compressed matrix, >1 GB, is streamed every step)",
                   "parallelism": f"replicas{world}"},
        "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "p999": float(np.percentile(lat, 99.9)), "max": float(lat.max())},
        "rel_err_vs_fp64_uncompressed": rel_err,
        "p99_at_rel_err_1e-5": at_target,
        "effective_gflops": round(order * (2 * order - 1) / (ms_per_step * 1e-3) / 1e9 * world, 1),
        "pct_hbm_peak": round(100 * value / world / peak, 2),
        "roofline": roofline,
        "e2e": {"value": round(stream_bytes / (e2e_ms * 1e-3) / 1e9 * world, 2), "unit": "GB/s",
                "ms_per_step": round(e2e_ms, 5), "h2d_bytes_per_step": order * 4,
                "d2h_bytes_per_step": order * 8},
        "gpu_launches": args.steps * launches,
        "clocks": clocks,
        "formats": formats,
        "multi_rhs": multi,
        "fp64_uncompressed_gemv": fp64,
        "host_resident": host,
        "slit_graph": slits,
        "field_pipeline": fields,
        "setup_s": round(t_setup, 1),
    }
    if cpu is not None:
        res["cpu_baseline"] = cpu
    return res


# ------------------------------------------------- slits and streamed fields
def slit_graph_leg(W, torch, blob, order, xs, stream, nrows=378, steps=2000):
    """One instantiated slit graph moved over the resident control-loop matrix (Sec. 2.1:
    C_slit of 378 rows, Sec. 5.1's M, fetched from C_field every step): per step the host
    moves the slit (whff_graph_set_rows: re-capture + in-place parameter update) and
    replays; device time per replay from CUDA events, host time of the move."""
    h = W.whff_create(blob, max_rhs=1)
    y = torch.zeros(order, dtype=torch.float64, device=xs.device)
    s = torch.zeros(order, dtype=torch.float64, device=xs.device)
    x = xs[0].clone()
    offs = [((order - nrows) * (k % 97) // 96) // 4 * 4 for k in range(steps)]
    g = W.whff_graph_create_rows(h, offs[0], nrows, x, y, s, DECAY, stream)
    for k in range(20):
        g.set_rows(offs[k])
        g.launch(stream)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
    host = []
    for k in range(steps):
        t0 = time.perf_counter()
        g.set_rows(offs[k])
        host.append(time.perf_counter() - t0)
        evs[2 * k].record(stream)
        g.launch(stream)
        evs[2 * k + 1].record(stream)
    torch.cuda.synchronize()
    dev_us = np.array([evs[2 * k].elapsed_time(evs[2 * k + 1]) * 1e3 for k in range(steps)])
    host_us = np.array(host) * 1e6
    g.destroy()
    h.destroy()
    sb = nrows * order * 2  # rate 16: 2 bytes per value
    return {"slit_rows": nrows, "field_rows": order, "steps": steps, "bytes_per_step": sb,
            "replay_us": {"p50": float(np.percentile(dev_us, 50)), "p99": float(np.percentile(dev_us, 99)),
                          "mean": float(dev_us.mean())},
            "move_host_us": {"p50": float(np.percentile(host_us, 50)), "p99": float(np.percentile(host_us, 99))},
            "GB_s_at_p50": round(sb / (np.percentile(dev_us, 50) * 1e-6) / 1e9, 1),
            "note": "one instantiated graph; the slit offset is updated in place before each replay"}


def field_pipeline_leg(W, torch, dev, stream, L=2016, S=256000, slit=378, steps_per_field=20, fields=8):
    """Sec. 4.3 (Fig. compression_cost, Table comp_metrics) and Sec. 5.2 (Fig.
    decompression_overhead) on GB300: exposure fields of L x S (the paper's C_field,
    2067 MB in FP32) cross the CPU-GPU link into two resident slots while the slit steps of
    the previous field run (20 slits of 378 rows per field).  Measured: the copy of one
    field (T_tr, compressed and FP32), its 20 slit steps alone (T_comp), the pipelined
    period and one field's latency, against the table's formulas (T_dec = 0: decode is
    fused into the step); and the breakdown of Fig. decompression_overhead."""
    import workloads

    t0 = time.perf_counter()
    A = workloads.RectKernelMatrix(L, S, 0.05, workloads.SEED_BASE + 80).dense()
    X = torch.from_numpy(np.random.default_rng(80).standard_normal((steps_per_field, S)).astype(np.float32)).to(dev)
    offs = [((L - slit) * j // (steps_per_field - 1)) // 4 * 4 for j in range(steps_per_field)]
    out = {"field": [L, S], "slit_rows": slit, "slit_steps_per_field": steps_per_field, "fields": fields}
    copy = torch.cuda.Stream(dev)
    kinds = (("wz2-lift-16", 5, 16), ("fp32", 7, 0))
    hosts = {}
    for name, fmt, rate in kinds:
        blob = W.whff_compress(A, fmt, rate or 16)
        hosts[name] = torch.from_numpy(blob).pin_memory()
        del blob
    del A
    for name, fmt, rate in kinds:
        host = hosts.pop(name).numpy()
        nbytes = host.size - 64
        x = torch.zeros(S, dtype=torch.float32, device=dev)
        y = torch.zeros(L, dtype=torch.float64, device=dev)
        st = torch.zeros(L, dtype=torch.float64, device=dev)
        align = 4 if fmt in (1, 5, 6) else 128
        offs_f = [o // align * align for o in offs]
        F = W.Fields(fmt, rate, L, S, nbuf=2, max_rhs=1, stream=stream)
        F.load(0, host, copy)
        h0 = F.acquire(0, stream)
        g = W.whff_graph_create_rows(h0, offs_f[0], slit, x, y, st, DECAY, stream)

        def field_steps(h):
            for j, r0 in enumerate(offs_f):
                x.copy_(X[j], non_blocking=True)
                g.set_rows(r0, h)
                g.launch(stream)

        field_steps(h0)
        F.release(0, stream)
        torch.cuda.synchronize()
        ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
        # the copy alone
        a, b = ev(), ev()
        a.record(copy)
        F.load(1, host, copy)
        b.record(copy)
        torch.cuda.synchronize()
        t_tr = a.elapsed_time(b)
        # the slit steps of one field alone (resident)
        h1 = F.acquire(1, stream)
        field_steps(h1)
        torch.cuda.synchronize()
        a.record(stream)
        field_steps(h1)
        b.record(stream)
        torch.cuda.synchronize()
        t_comp = a.elapsed_time(b)
        F.release(1, stream)
        # one field's latency: its copy starts, then its steps (nothing else in flight)
        torch.cuda.synchronize()
        a.record(copy)
        F.load(0, host, copy)
        h = F.acquire(0, stream)
        field_steps(h)
        b.record(stream)
        F.release(0, stream)
        torch.cuda.synchronize()
        lat = a.elapsed_time(b)
        # the pipeline: field k+1 crosses the link while field k's slits run
        done = [ev() for _ in range(fields)]
        copied = [ev() for _ in range(fields)]
        t_start = ev()
        t_start.record(copy)
        F.load(0, host, copy)
        copied[0].record(copy)
        host_t = time.perf_counter()
        for k in range(fields):
            slot = k % 2
            if k + 1 < fields:
                F.load(1 - slot, host, copy)
                copied[k + 1].record(copy)
            h = F.acquire(slot, stream)
            field_steps(h)
            F.release(slot, stream)
            done[k].record(stream)
        host_t = time.perf_counter() - host_t
        torch.cuda.synchronize()
        gaps = [done[k - 1].elapsed_time(done[k]) for k in range(2, fields)]
        period = float(np.mean(gaps))
        timeline = {"copy_done_ms": [round(t_start.elapsed_time(e), 3) for e in copied],
                    "steps_done_ms": [round(t_start.elapsed_time(e), 3) for e in done],
                    "host_issue_ms": round(host_t * 1e3, 3)}
        g.destroy()
        F.destroy()
        del host
        out[name] = {"field_bytes": int(nbytes), "T_transfer_ms": round(t_tr, 3),
                     "link_GB_s": round(nbytes / (t_tr * 1e-3) / 1e9, 1), "T_comp_ms": round(t_comp, 4),
                     "period_ms": round(period, 3), "period_model_ms": round(max(t_tr, t_comp), 3),
                     "latency_ms": round(lat, 3), "latency_model_ms": round(t_tr + t_comp, 3), "timeline": timeline}
    c, u = out["wz2-lift-16"], out["fp32"]
    before = u["T_transfer_ms"] + u["T_comp_ms"]
    out["ratio_R"] = round(u["field_bytes"] / c["field_bytes"], 3)
    out["breakdown_normalised"] = {  # Fig. decompression_overhead's bars, before = 100
        "before": {"computation": round(100 * u["T_comp_ms"] / before, 2),
                   "transfer": round(100 * u["T_transfer_ms"] / before, 2), "decompression": 0.0},
        "after": {"computation_with_fused_decode": round(100 * c["T_comp_ms"] / before, 2),
                  "transfer": round(100 * c["T_transfer_ms"] / before, 2), "decompression": 0.0}}
    out["period_speedup"] = round(u["period_ms"] / c["period_ms"], 3)
    out["setup_s"] = round(time.perf_counter() - t0, 1)
    return out


# ------------------------------------------------------------ serving arm
def run_serve(args, rank, world, local_rank):
    """Resident control models served through the C++ request server: Poisson
    arrivals per model, continuous batching into graph-replayed passes,
    admission by device-memory footprint; latency = host-observed completion
    of the pass that carried a request minus its arrival."""
    import torch

    import paper_1902_08018_gb300 as W
    import workloads

    torch.cuda.set_device(local_rank)
    fmt_name, rate = args.serve_fmt.split(":")
    fmt, rate = FMT_CODES[fmt_name], int(rate)
    orders = [int(v) for v in args.serve_orders.split(",")]
    free, _ = torch.cuda.mem_get_info()
    t0 = time.perf_counter()
    handles, blobs_bytes = [], []
    made = {}  # models of equal order share the matrix values (each has its own resident copy and state)
    for k, n in enumerate(orders):
        if n not in made:
            g = int(np.ceil(np.sqrt(n)))
            km = workloads.KernelMatrix(n, g, n, 0.05, workloads.SEED_BASE + 5 + 1000 * k)
            made[n] = W.whff_compress_bands(n, n, km.bands(2048), fmt, rate)
        blob = made[n]
        handles.append(W.whff_create(blob, max_rhs=8))
        if not args.no_tune and fmt in (5, 6):  # launch shape and engine crossover per model, on this machine
            handles[-1].tune(iters=5)
        blobs_bytes.append(blob.size - 64)
        del blob
    made.clear()
    setup_s = time.perf_counter() - t0
    # each model's single pass alone (its tuned shape, R = 1, stream resident): the kernels' own rate
    dev = torch.device("cuda", local_rank)
    alone_ms = []
    for h in handles:
        xa = torch.zeros(h.N, dtype=torch.float32, device=dev)
        ya = torch.zeros(h.M, dtype=torch.float64, device=dev)
        for _ in range(2):
            h.step(xa, ya, None, DECAY)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            h.step(xa, ya, None, DECAY)
        e1.record()
        torch.cuda.synchronize()
        alone_ms.append(e0.elapsed_time(e1) / 5)
    budget = int(free * 0.9)
    rng = np.random.default_rng(workloads.SEED_BASE + 5)
    events = []
    for k, n in enumerate(orders):
        arr = workloads.poisson_arrivals(args.serve_hz, args.serve_seconds, workloads.SEED_BASE + 50 + k)
        events += [(t, k) for t in arr]
    events.sort()
    model = np.array([m for _, m in events], dtype=np.int32)
    arrival = np.array([t for t, _ in events], dtype=np.float64)
    pools = []  # per model: 64 heat-load-like vectors
    for k, n in enumerate(orders):
        pools.append([rng.standard_normal(n).astype(np.float32) for _ in range(64)])
    xs = [pools[m][i % 64] for i, m in enumerate(model)]
    admitted, refused = [], []
    with ClockSampler(local_rank) as clk, W.Server(budget, max_batch=8, nstreams=8) as srv:
        ids = {}
        for k, h in enumerate(handles):
            try:
                ids[k] = srv.add_model(h, DECAY)
                admitted.append(k)
            except W.WhffError:
                refused.append(k)
        keep = np.isin(model, admitted)
        remap = np.array([ids.get(k, -1) for k in range(len(orders))])
        m_ids = remap[model[keep]]
        xs_k = [x for x, kp in zip(xs, keep) if kp]
        # short warm-up trace (first 200 requests' pattern), then the measured trace
        drop = args.deadline_us * 1e-6 if args.firm else 0.0
        srv.run(m_ids[:200], arrival[keep][:200] - arrival[keep][0], xs_k[:200], drop_after_s=drop)
        lat, bat, _, status = srv.run(m_ids, arrival[keep], xs_k, max_wait_s=args.serve_seconds * 60 + 60,
                                      drop_after_s=drop, return_status=True)
    clocks = clk.summary()
    lat_us = lat * 1e6
    served = status != 2
    miss = (status != 0) | (lat_us > args.deadline_us)

    def pct(v, q):
        return float(np.percentile(v, q)) if v.size else None

    per = {}
    for k in admitted:
        sel = model[keep] == k
        l = lat_us[sel & served]
        per[f"N={orders[k]}#{k}"] = {"requests": int(sel.sum()), "served": int((sel & served).sum()),
                                   "p50_us": pct(l, 50), "p99_us": pct(l, 99), "p999_us": pct(l, 99.9),
                                   "miss_rate": float(miss[sel].mean()),
                                   "mean_batch": float(bat[sel & served].mean()) if l.size else 0.0,
                                   "pass_bytes": blobs_bytes[k]}
    passes = sum(1.0 / b for b in bat[served])  # each pass counted once over its requests
    streamed = sum(blobs_bytes[model[keep][i]] / bat[i] for i in np.nonzero(served)[0])
    wall = float(np.max(arrival[keep] + lat)) if len(arrival) else 0.0
    lat_us = lat_us[served]
    shapes = [list(h.config()) + [h.crossover] if fmt in (5, 6) else None for h in handles]  # before destroy
    for h in handles:
        h.destroy()
    return {
        "mode": "serve", "metric": "serving: p50/p99/p99.9 control-step latency and deadline misses",
        "value": float(np.percentile(lat_us, 99)), "unit": "us (p99, all requests)", "higher_is_better": False,
        "n_gpus": world, "config": {"workload": f"serving-{len(orders)}-models-{fmt_name}-{rate}", "orders": orders,
                                    "arrival_hz_per_model": args.serve_hz, "seconds": args.serve_seconds,
                                    "deadline_us": args.deadline_us, "max_batch": 8, "streams": 8,
                                    "hbm_budget_bytes": budget,
                                    "launch_shapes": shapes},
        "admitted": admitted, "refused": refused, "requests": int(keep.sum()),
        "p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
        "p999_us": float(np.percentile(lat_us, 99.9)), "miss_rate": float(miss.mean()),
        "dropped": int((status == 2).sum()), "firm": bool(args.firm),
        "passes": round(passes), "mean_batch": float(np.mean(bat[served])),
        "streamed_GB_s": round(streamed / max(wall, 1e-9) / 1e9, 1),
        "kernels_alone_GB_s": round(sum(blobs_bytes) / (sum(alone_ms) * 1e-3) / 1e9, 1),
        "pass_alone_ms": [round(v, 4) for v in alone_ms],
        "round_alone_ms": round(sum(alone_ms), 3),
        "per_model": per, "clocks": clocks, "setup_s": round(setup_s, 1),
    }


# ------------------------------------------------------------ batched arm
def run_batched(args, rank, world, local_rank):
    """64 independent smooth-kernel matrices of uneven order (log-uniform in
    2048..16384, seeded) with 1, 4, 8 or 32 right-hand sides each, stepped by
    one batch (one persistent launch per right-hand-side class), against
    stepping every matrix on its own."""
    import torch

    import paper_1902_08018_gb300 as W
    import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    fmt_name, rate = args.batched_fmt.split(":")
    fmt, rate = FMT_CODES[fmt_name], int(rate)
    inst = workloads.batched_instances()
    t0 = time.perf_counter()
    handles, sizes = [], []
    for N, R in inst:
        km = workloads.instance_matrix(N)
        blob = W.whff_compress_bands(N, N, km.bands(2048), fmt, rate)
        handles.append(W.whff_create(blob, max_rhs=32))
        if args.batched_crossover:
            handles[-1].crossover = args.batched_crossover
        sizes.append(blob.size - 64)
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(4)
    X = [torch.from_numpy(rng.standard_normal((R, N)).astype(np.float32)).to(dev) for N, R in inst]
    Y = [torch.zeros((R, N), dtype=torch.float64, device=dev) for N, R in inst]
    S = [torch.zeros(N, dtype=torch.float64, device=dev) for N, R in inst]
    Rs = [R for _, R in inst]
    stream = torch.cuda.current_stream(dev)
    steps = max(1, min(args.steps, 50))
    with W.Batch(handles, Rs) as b:
        for _ in range(3):
            b.step(X, Y, S, DECAY, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local_rank) as clk:
            e0.record(stream)
            for _ in range(steps):
                b.step(X, Y, S, DECAY, stream)
            e1.record(stream)
            torch.cuda.synchronize()
        batch_ms = e0.elapsed_time(e1) / steps
    # every matrix on its own (same kernels, one whff_step per matrix)
    for _ in range(2):
        for h, x, y, s in zip(handles, X, Y, S):
            h.step(x, y, s, DECAY, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, steps // 5)):
        for h, x, y, s in zip(handles, X, Y, S):
            h.step(x, y, s, DECAY, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / max(1, steps // 5)
    once = sum(sizes)
    # bytes read per step: a matrix stepped on the tensor cores (R >= its crossover) is read once per
    # 32 columns; the CUDA-core classes read it once per class (8, 4, 2, 1) that R uses
    streamed = 0
    for sz, R, h in zip(sizes, Rs, handles):
        if R >= h.crossover:
            streamed += sz * ((R + 31) // 32)
        else:
            streamed += sz * (R // 8 + bin(R % 8).count("1"))
    peak, peak_kind = measured_peaks()
    flops = sum(R * N * (2 * N - 1) for N, R in inst)
    xover = handles[0].crossover
    for h in handles:
        h.destroy()
    return {
        "mode": "batched", "metric": "batched compressed GEMV: HBM GB/s & % peak",
        "value": round(once / (batch_ms * 1e-3) / 1e9, 1), "unit": "GB/s (compressed bytes of all matrices)",
        "higher_is_better": True, "n_gpus": world, "steps": steps,
        "config": {"workload": f"batched-64-uneven-{fmt_name}-{rate}", "instances": len(inst),
                   "orders_min_max": [min(n for n, _ in inst), max(n for n, _ in inst)],
                   "R_counts": {str(r): Rs.count(r) for r in sorted(set(Rs))},
                   "crossover": xover},
        "ms_per_step": round(batch_ms, 4), "compressed_bytes": once, "bytes_streamed_per_step": streamed,
        "streamed_GB_s": round(streamed / (batch_ms * 1e-3) / 1e9, 1),
        "pct_hbm_peak_streamed": round(100 * streamed / (batch_ms * 1e-3) / 1e9 / peak, 2), "peak_kind": peak_kind,
        "effective_gflops": round(flops / (batch_ms * 1e-3) / 1e9, 1),
        "one_matrix_at_a_time_ms": round(single_ms, 4), "batch_speedup": round(single_ms / batch_ms, 2),
        "clocks": clk.summary(), "setup_s": round(setup_s, 1),
    }


def run_shapes(args, rank, world, local_rank):
    """The paper's three GEMV shapes (Sec. 5.1, Fig. results_throughput): wide 378 x 256000, tall
    256000 x 378, square 10000 x 10000, each stored uncompressed in FP32 (the
    paper's mixed precision, Sec. 4.4) and compressed, against plain FP64 GEMV
    on the same GPU.  One right-hand side; every timed step reads a matrix that
    is not in L2 (a 512 MB buffer is written between steps, outside the
    events).  rel_err: y against FP64 A x on the uncompressed matrix."""
    import torch

    import paper_1902_08018_gb300 as W
    import workloads

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(5, min(args.steps, 100))
    specs = []
    for item in filter(None, args.shapes_fmts.split(",")):
        name, rate = item.split(":")
        specs.append((name, FMT_CODES[name], int(rate)))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            fn()
        ts = []
        for _ in range(steps):
            flush.fill_(1)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    # the paper's P100 figures (Sec. 5.1, Fig. results_throughput), GFLOP/s: context, not a target
    p100 = {"wide": {"gpu_mp_cuda": 198.3, "cublas_dgemv": 14.59},
            "tall": {"gpu_mp_cuda": 65.9, "cublas_dgemv": 99.69},
            "square": {"gpu_mp_cuda": 202.62, "cublas_dgemv": 87.83}}
    out = {}
    for sname, M, N in workloads.PAPER_SHAPES:
        A = workloads.RectKernelMatrix(M, N, 0.05, workloads.SEED_BASE + 70).dense()
        x64 = np.random.default_rng(workloads.SEED_BASE + 71).standard_normal(N)
        y_star = A @ x64
        flops = M * (2 * N - 1)
        entry = {"M": M, "N": N, "paper_p100_gflops": p100[sname]}
        xd = torch.from_numpy(x64.astype(np.float32)).to(dev)
        yd = torch.zeros(M, dtype=torch.float64, device=dev)
        for name, fmt, rate in specs:
            blob = W.whff_compress(A, fmt, rate if rate else 16)
            nbytes = blob.size - 64
            with W.whff_create(blob, max_rhs=1) as h:
                ms = timed(lambda: h.step(xd, yd, None, DECAY, stream))
                torch.cuda.synchronize()
                y = yd.cpu().numpy()
            key = f"{name}-{rate}" if rate else name
            entry[key] = {"ms": round(ms, 4), "bytes": int(nbytes), "GB_s": round(nbytes / (ms * 1e-3) / 1e9, 1),
                          "pct_hbm": round(100 * nbytes / (ms * 1e-3) / 1e9 / peak, 2),
                          "effective_gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                          "rel_err": float(np.linalg.norm(y - y_star) / np.linalg.norm(y_star))}
            del blob
        if not args.no_fp64_baseline:
            Ad = torch.from_numpy(A).to(dev)
            xd64 = torch.from_numpy(x64).to(dev)
            ms = timed(lambda: torch.mv(Ad, xd64))
            entry["fp64_torch_mv"] = {"ms": round(ms, 4), "bytes": A.nbytes,
                                      "GB_s": round(A.nbytes / (ms * 1e-3) / 1e9, 1),
                                      "effective_gflops": round(flops / (ms * 1e-3) / 1e9, 1)}
            del Ad
        out[sname] = entry
        del A
    return {"mode": "shapes", "metric": "compressed GEMV on the paper's shapes: GB/s, GFLOP/s, % HBM peak",
            "unit": "GB/s", "higher_is_better": True, "n_gpus": world, "steps": steps, "peak_GB_s": peak,
            "peak_kind": peak_kind, "data": "synthetic smooth-kernel matrices of the paper's shapes",
            "l2": "flushed between steps (512 MB write, outside the events)", "shapes": out}


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host cores, on the same workload and metric.
    Its input is made by the oracle's own encoder (no library code on this arm): bands
    of 32 rows per host thread (eight 4-row block rows each, so every core has work) at
    four places of the matrix, each encoded once as a matrix of its own -- its stream
    is byte for byte that band's part of the whole matrix's stream.  Each step decodes
    one band, multiplies it by that step's heat load in FP64 and updates the band's
    FP64 state; steps cycle over the bands."""
    import oracle
    import workloads

    oracle.build()
    order = args.order
    fmt, rate = FMT_CODES[args.fmt], args.rate
    km = matrix_for(order)
    cores = oracle.num_threads()
    rows_per_step = min(order // 4 * 4 or 4, 32 * cores)
    starts = sorted({(order * k // 4) // 4 * 4 for k in range(4)})
    starts = [min(r0, max(0, order - rows_per_step) // 4 * 4) for r0 in starts]
    bands = []
    for r0 in starts:
        A = km.rows(r0, r0 + rows_per_step)
        bands.append(oracle.encode(A, fmt, rate))
        del A
    S = max(1, min(100, args.steps + args.warmup))
    X64 = workloads.heat_loads(km.g, km.n_valid, order, S).T.copy()  # (S, N)
    state = [np.zeros(rows_per_step) for _ in bands]

    def one(k):
        b = k % len(bands)
        D = oracle.decode_rows(bands[b], 0, rows_per_step)
        y = oracle.gemv64(D, X64[k % S])
        state[b] = oracle.state_update(state[b], y, DECAY)
        return y

    for k in range(args.warmup):
        one(k)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(args.warmup + k)
    dt = time.perf_counter() - t0
    comp = rows_per_step * order * rate / 8.0 * args.steps
    value = comp / dt / 1e9
    name = f"{args.fmt}-{rate}"
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"control-loop-{order}-rate{rate}", "M": order, "N": order, "fmt": name,
                   "rate_bits_per_value": rate, "R": 1},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows_per_step} of {order} rows per step ({rows_per_step // 4} block rows over "
                                   f"{cores} threads), bands at rows {starts}, oracle encode once, then per step "
                                   f"oracle decode + FP64 GEMV + FP64 state update"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------- precision sweep
def run_precision(args, rank, world, local_rank):
    """Every storage format of the precision layer on the control-loop matrix, at one
    right-hand side (the heat load of step 0) and at 32 (the heat loads of steps 0..31):
    step time, GB/s of stored bytes, and the relative L2 error of y against FP64 GEMV on
    the uncompressed matrix (64 sampled rows, the worst of the 32 columns); and Table 2's
    columns (bits per value, rate, RMSE, NRMSE, largest pointwise error, PSNR) of the
    decoded sample rows against the matrix rounded to FP32."""
    import torch

    import paper_1902_08018_gb300 as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    order = args.order
    specs = []
    for item in filter(None, args.precision_fmts.split(",")):
        name, rate = item.split(":")
        specs.append((FMT_CODES[name], int(rate) if FMT_CODES[name] in (1, 5, 6) else 0))
    rng = np.random.default_rng(12345)
    sample_rows = np.sort(rng.choice(order, size=64, replace=False))
    t_setup = time.perf_counter()
    km, blobs, _, sampled = build_workload(order, specs, False, sample_rows, torch, dev)
    t_setup = time.perf_counter() - t_setup
    X64 = heat_load_inputs(km, 32)  # (32, N)
    Y_star = sampled @ X64.T        # (64, 32) FP64 reference on the uncompressed rows
    X = torch.from_numpy(X64.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = measured_peaks()
    table = {}
    with ClockSampler(local_rank) as clk:
        for spec in specs:
            name = f"{FMT_NAMES[spec[0]]}-{spec[1]}" if spec[1] else FMT_NAMES[spec[0]]
            h = W.whff_create(blobs[spec], max_rhs=32)
            sb = blobs[spec].size - 64
            entry = {"bytes": int(sb)}
            # Table 2's columns: the decoded sample rows against the matrix rounded to FP32
            D = torch.empty((order, order), dtype=torch.float64, device=dev)
            h.decompress(D, stream)
            Ahat = D[torch.from_numpy(sample_rows).to(dev)].cpu().numpy()
            del D
            entry["table2"] = table2_metrics(sampled.astype(np.float32), Ahat, sb, order * order)
            for R, reps in ((1, max(10, args.steps)), (32, max(5, args.steps // 10))):
                Y = torch.zeros((R, order), dtype=torch.float64, device=dev)
                for _ in range(3):
                    h.step(X[:R], Y, None, DECAY, stream)
                torch.cuda.synchronize()
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                for _ in range(reps):
                    h.step(X[:R], Y, None, DECAY, stream)
                f1.record(stream)
                torch.cuda.synchronize()
                ms = f0.elapsed_time(f1) / reps
                Yh = Y.cpu().numpy()[:, sample_rows].T  # (64, R)
                err = max(float(np.linalg.norm(Yh[:, r] - Y_star[:, r]) / np.linalg.norm(Y_star[:, r]))
                          for r in range(R))
                engine = "tcgen05" if (spec[0] in (2, 3, 4, 5, 6) and R >= h.crossover) else "cuda-core"
                entry[f"R{R}"] = {"ms_per_step": round(ms, 4), "GB_s": round(sb / (ms * 1e-3) / 1e9, 1),
                                  "pct_hbm": round(100 * sb / (ms * 1e-3) / 1e9 / peak, 2),
                                  "effective_tflops": round(R * order * (2 * order - 1) / (ms * 1e-3) / 1e12, 2),
                                  "rel_err_vs_fp64_uncompressed": err, "engine": engine}
            table[name] = entry
            h.destroy()
    head = table.get("wz2-lift-16", next(iter(table.values())))
    return {"mode": "precision", "metric": "precision sweep: GB/s & % peak and rel. L2 error vs FP64 per format",
            "value": head["R1"]["GB_s"], "unit": "GB/s (stored bytes, wz2-lift-16, R = 1)", "higher_is_better": True,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"precision-sweep-{order}", "order": order, "R": [1, 32],
                       "x": "heat loads of control steps 0..31 (serpentine path)",
                       "error_rows": "64 sampled rows, FP64 GEMV on the uncompressed matrix"},
            "peak_gbs": peak, "peak_kind": peak_kind, "formats": table, "clocks": clk.summary(),
            "setup_s": round(t_setup, 1)}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        res = run_reference(args, rank, world)
    elif args.serve:
        res = run_serve(args, rank, world, local_rank)
    elif args.batched:
        res = run_batched(args, rank, world, local_rank)
    elif args.shapes:
        res = run_shapes(args, rank, world, local_rank)
    elif args.precision:
        res = run_precision(args, rank, world, local_rank)
    else:
        if world > 1:
            import torch

            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        res = run_whff(args, rank, world, local_rank)
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()
        elif not args.no_serve_leg:  # the serving loop and the batched instances, bounded, same process
            import torch

            torch.cuda.empty_cache()
            res["serving"] = run_serve(args, rank, world, local_rank)
            torch.cuda.empty_cache()
            res["batched"] = run_batched(args, rank, world, local_rank)
    if rank == 0:
        line = json.dumps(res)
        print(line, flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(line + "\n")


if __name__ == "__main__":
    main()
