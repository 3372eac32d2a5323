#!/usr/bin/env python
"""Throughput of the streaming tensor-ring update on GB300.

Workload (one "step" = one STR update, every row of the hot path):
  order-4 tensor 64x64x64xT, T = 400, TR-ranks all 8, Gaussian cores, noise at
  SNR 30 dB, initial cores = true cores + 0.05 N(0,1) on 40 slices, then
  updates of 10 slices, 5 sweeps per update, FP32 slab and FP32 slab-side
  arithmetic (FP64 Gram, P_n/Q_n state).  Inputs are synthetic, built on the
  host in FP64 (the same bytes feed the CPU oracle) and already resident in HBM
  when the timed region starts.

Printed as one JSON line by rank 0.  `--impl reference` times the FP64 CPU
oracle on the same workload and the same input bytes (one update per step).
Secondary rows (same line): the plain FP64 GPU arm of the same workload,
rSTR-U/L/K updates on a 512x512xT BF16 workload (ranks 10, sketch size 2000),
batched updates of 256 uneven order-3 streams, the masked TR fit loss and its
backward on a 32x32x32x32x100 FP32 tensor, and STR updates on a 60^5 stand-in
of the paper's largest synthetic tensor (ranks 5, 5-slice slabs).  Every row
states its step roofline (t_bound / t_update, t_bound = max(F_alg / pipe
peak, B_alg / HBM peak) with the pipe peaks measured in this run) and, at
N = 1 on rank 0, its relative fit error against the FP64 oracle run on the
same bytes for the first updates (the CPU-oracle leg).
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "STR/rSTR tensor entries/s per update, % roofline, rel. fit err vs FP64"
# DRAM bytes (read + write) of one stage-1 launch on the order-4 workload, from an
# ncu capture of this bench (dram__bytes_read.sum + dram__bytes_write.sum); set to
# None whenever the stage-1 kernel changes until it is captured again
STAGE1_DRAM_BYTES = 10549760
W2 = synth.WORKLOADS["order4"]
W3 = synth.WORKLOADS["rand3"]
WORKLOAD_DESC = ("order4: 64x64x64xT, T=400, TR-ranks all 8, Gaussian cores, SNR 30 dB, "
                 "init = true cores + 0.05 N(0,1) on 40 slices, updates of 10 slices, 5 sweeps, FP32 slab")
FLUSH_BYTES = 256 << 20     # > 129 MB L2
INIT_PERTURB = 0.05
CHECK_UPDATES = 3           # updates compared with the oracle (order-4 rows)
LOSS_NOISE = 1e-2
BATCH_NOISE = 1e-2


def args_parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-rstr", action="store_true", help="skip the rSTR rows")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU arm")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-streams row")
    ap.add_argument("--no-loss", action="store_true", help="skip the masked-loss row")
    ap.add_argument("--no-large", action="store_true", help="skip the 60^5 stand-in row")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--evidence", default=None, choices=["stage1_r12", "sampling_m1e6", "batch256", "masked_loss"],
                    help="run one kernel-evidence workload (for ncu captures) and print its line")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(torch, value, world, device):
    """The largest of every rank's value: the job ends when its slowest rank does."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the max-over-ranks time."""
    return world * units_per_rank / seconds


def step_roofline(t_ms, flop, pipe_peak_tflops, nbytes, hbm_gbs, pipe):
    """Step roofline of one update: t_bound = max(F_alg / pipe peak, B_alg / HBM
    peak); frac_step = t_bound / t_update."""
    t_f = flop / (pipe_peak_tflops * 1e12) if pipe_peak_tflops else 0.0
    t_b = nbytes / (hbm_gbs * 1e9)
    t_bound = max(t_f, t_b)
    return {"t_bound_us": round(t_bound * 1e6, 3), "t_update_us": round(t_ms * 1e3, 2),
            "frac_step": round(t_bound / (t_ms / 1e3), 5), "bound": pipe if t_f >= t_b else "hbm",
            "flop_alg": flop, "bytes_alg": nbytes, "pipe_peak_tflops": pipe_peak_tflops, "hbm_gbs": hbm_gbs}


# ---------------------------------------------------------------------------
# inputs: built on the host in FP64 (the same bytes feed both arms and the oracle)
# ---------------------------------------------------------------------------
def host_tr_tensor(G, t0=0, t1=None):
    """TR(G) over temporal rows [t0, t1) as a float64 array X[i_1..i_N]: the
    trace formula of the TR format, X(i) = Trace(G_1(i_1)..G_N(i_N)), for all
    entries at once (the spatial slices multiplied left to right, then the
    trace against the temporal core's slices)."""
    T = G[0]
    for g in G[1:-1]:
        T = np.tensordot(T, g, axes=([T.ndim - 1], [0]))       # (R_1, I_1, .., I_k, R_{k+1})
    GN = G[-1][:, t0:t1, :]                                     # (R_N, t, R_1)
    return np.tensordot(T, GN, axes=([0, T.ndim - 1], [2, 0]))  # sum over r_1, r_N


def host_workload(w, seed):
    """True cores, X = TR(G) + noise (relative Frobenius level w.noise) over all
    T slices, and the initial cores (true cores + 0.05 N(0,1), temporal core cut
    to t_init rows)."""
    G = synth.gaussian_cores(tuple(w.dims) + (w.T,), w.ranks, seed)
    X = host_tr_tensor(G)
    if w.noise > 0:
        X = synth.add_noise(X, synth.gaussian_tensor(X.shape, seed + 100), w.noise)
    rng = np.random.default_rng(seed + 200)
    init = [g + INIT_PERTURB * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :w.t_init, :]
    return G, X, init


def to_device(torch, X, dtype=None):
    """numpy X[i_1..i_N] -> CUDA tensor indexed the same way with i_1 fastest."""
    rev = list(range(X.ndim - 1, -1, -1))
    t = torch.from_numpy(np.ascontiguousarray(X.transpose(rev)))
    t = t.to("cuda", dtype) if dtype is not None else t.to("cuda")
    return t.permute(rev)


def bf16_device(torch, X):
    """BF16 copy of X whose values are exactly synth.to_bf16_values(X)."""
    rev = list(range(X.ndim - 1, -1, -1))
    bits = synth.bf16_bits(np.ascontiguousarray(X.transpose(rev)))
    t = torch.from_numpy(bits.view(np.int16)).to("cuda").view(torch.bfloat16)
    return t.permute(rev)


def slab(X, w, j, dtype=None):
    nsl = (w.T - w.t_init) // w.t_new
    t0 = w.t_init + (j % nsl) * w.t_new
    s = X[..., t0:t0 + w.t_new]
    return s if dtype is None else s.to(dtype)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# peaks: HBM and BF16 from the driver's measurement file (else the fallback),
# TF32 tensor, FP32 and FP64 FMA pipes measured here with CUDA events
# ---------------------------------------------------------------------------
def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "of measured"
    except Exception:
        return fallback, "of fallback"


def event_ms(torch, fn, reps):
    """Best of `reps` CUDA-event timings of fn() on the current stream."""
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def measure_peaks(p, torch):
    hbm, hbm_src = measured_peak("hbm_gbs", 6800.0)
    bf16, bf16_src = measured_peak("bf16_tflops", 1900.0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # TF32: cuBLAS FP32 GEMM with TF32 tensor cores allowed, 8192^3
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    n = 8192
    A = torch.randn(n, n, device="cuda")
    B = torch.randn(n, n, device="cuda")
    C = torch.empty(n, n, device="cuda")
    for _ in range(3):
        torch.matmul(A, B, out=C)
    ms = event_ms(torch, lambda: [torch.matmul(A, B, out=C) for _ in range(5)], 3) / 5
    tf32 = 2.0 * n ** 3 / (ms / 1e3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = prev
    del A, B, C
    # FP32 / FP64 FMA pipes: the library's probe kernel, 8 blocks of 256 threads per SM
    ctas = 8 * sms
    rates = {}
    for dt, iters in (("f32", 20000), ("f64", 400)):
        out = torch.empty(ctas, dtype=torch.float32 if dt == "f32" else torch.float64, device="cuda")
        flop = p.fma_probe(dt, ctas, iters, out)
        ms = event_ms(torch, lambda: p.fma_probe(dt, ctas, iters, out), 3)
        rates[dt] = flop / (ms / 1e3) / 1e12
    torch.cuda.synchronize()
    return {"hbm_gbs": hbm, "hbm_note": hbm_src, "bf16_tflops": bf16, "bf16_note": bf16_src,
            "tf32_tflops": round(tf32, 1), "tf32_note": "measured here: torch.matmul FP32 8192^3 with TF32 allowed",
            "fp32_fma_tflops": round(rates["f32"], 2), "fp64_fma_tflops": round(rates["f64"], 3),
            "fma_note": f"measured here: str_fma_probe, {ctas} blocks x 256 threads, 8 FMA chains per thread",
            "sms": sms}


# ---------------------------------------------------------------------------
# timed loops
# ---------------------------------------------------------------------------
def timed_updates(p, torch, ctx, slabs, steps, warmup, randomized=False, flush=None, profile=False):
    """Warm-up, then `steps` updates, each bracketed by CUDA events on the
    launching stream with an L2 flush before it (outside the events).  Runs on
    a dedicated (non-default) stream so STR updates replay captured graphs."""
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        return _timed_updates(p, torch, ctx, slabs, steps, warmup, randomized, flush, profile, stream)


def _timed_updates(p, torch, ctx, slabs, steps, warmup, randomized, flush, profile, stream):
    upd = ctx.rupdate if randomized else ctx.update
    for j in range(warmup):
        upd(slabs(j))
    torch.cuda.synchronize()
    ctx.stats()                                   # reset profile counters
    times = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for j in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = evs[j]
        a.record(stream)
        upd(slabs(warmup + j))
        b.record(stream)
    torch.cuda.synchronize()
    for a, b in evs:
        times.append(a.elapsed_time(b))
    st = ctx.stats()
    # every update of a workload launches the same kernels; kernel_launches is the last one's count
    launches = sum(st["class_launches"].values()) if profile else steps * st["kernel_launches"]
    return times, launches, st


def str_flop(dims, t_new, ranks, sweeps):
    """F_alg of one STR update: per mode 2 E R_n R_{n+1} (the MTTKRP), every mode, every sweep."""
    E = int(np.prod(dims)) * t_new
    N = len(ranks)
    return 2.0 * E * sum(ranks[n] * ranks[(n + 1) % N] for n in range(N)) * sweeps


def main_ours(a):
    import torch
    import paper_2307_00719_gb300 as p
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    seed = W2.seed + 1000 * rank                       # independent replica per rank
    G, Xh, cores0 = host_workload(W2, seed)
    X = to_device(torch, Xh)                           # FP64, i_1 fastest
    X32 = to_device(torch, Xh, torch.float32)
    peaks = measure_peaks(p, torch)
    hbm = peaks["hbm_gbs"]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    E = int(np.prod(W2.dims)) * W2.t_new
    cap = W2.t_init + (a.warmup + a.steps + 2) * W2.t_new
    F2 = str_flop(W2.dims, W2.t_new, W2.ranks, W2.sweeps)

    def make(compute, xsrc, profile=0):
        return p.str_init_cores(cores0, X0=p.paper_layout(xsrc[..., :W2.t_init]), compute=compute,
                                sweeps=W2.sweeps, t_capacity=cap, async_status=1, profile=profile)

    # ---- main arm: FP32, device-resident slabs, L2 flushed between steps ----
    ctx = make("f32", X32)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, launches, _ = timed_updates(p, torch, ctx, lambda j: slab(X32, W2, j), a.steps, a.warmup,
                                       flush=flush)
    clk = clocks.stop()
    total_ms = max_over_ranks(torch, sum(times), world, "cuda")
    value = job_rate(a.steps * E, world, total_ms / 1e3)
    ctx.close()

    # ---- profile pass: per-class kernel times (same steps, events per launch) ----
    ctxp = make("f32", X32, profile=1)
    ptimes, _, pst = timed_updates(p, torch, ctxp, lambda j: slab(X32, W2, j), a.steps, a.warmup,
                                   flush=flush, profile=True)
    ctxp.close()
    k_ms, k_n = pst["class_ms"], pst["class_launches"]
    mt_avg_ms = k_ms["mttkrp"] / max(1, k_n["mttkrp"])
    slab_bytes = E * 4                                  # one read of the FP32 slab per launch
    achieved = slab_bytes / (mt_avg_ms / 1e3) / 1e9
    tot = sum(k_ms.values())
    c_avg_ms = k_ms["contract"] / max(1, k_n["contract"])
    RRk = W2.ranks[0] * W2.ranks[1]
    ms_step = total_ms / a.steps
    roofline = {"kernel": "stage1_ws_kernel (tcgen05 kind::tf32, 3-term split, TMA-fed, warp-specialised)",
                "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": STAGE1_DRAM_BYTES,
                "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one launch, ncu --set full "
                                "on this workload",
                "peak_note": f"HBM copy bandwidth, {peaks['hbm_note']}",
                "algorithmic_per_launch": {"bytes": slab_bytes, "flop": 2.0 * E * RRk,
                                           "note": "one read of the 64^3 x 10 FP32 slab; 2 E R_1 R_2 flop"},
                "avg_launch_ms": round(mt_avg_ms, 5), "launches": int(k_n["mttkrp"]),
                "tensor_tflops": round(2.0 * E * RRk / (mt_avg_ms / 1e3) / 1e12, 2),
                "stage2": {"kernel": "stage2_kernel (SIMT contraction with chain tables)",
                           "avg_launch_ms": round(c_avg_ms, 5), "launches": int(k_n["contract"]),
                           "read_gbs": round(E // W2.dims[0] * RRk * 4 / max(c_avg_ms, 1e-9) / 1e6, 1)},
                "step": step_roofline(ms_step, F2, peaks["tf32_tflops"], E * 4, hbm, "tf32"),
                "step_note": ("t_bound = max(F_alg / TF32 peak, one FP32 slab read / HBM); F_alg = 2 E sum_n "
                              "R_n R_{n+1} x 5 sweeps")}
    kernel_share = {k: round(v / tot, 4) for k, v in k_ms.items() if tot > 0 and v > 0}

    out = {"metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "precision": ("FP32 slab arithmetic (3-term TF32 split on tcgen05, FP32 accumulate), FP64 Gram / "
                         "P_n / Q_n state, FP32 factor of Q_n refined with a double-FP32 residual; fit error "
                         "against the FP64 oracle in fit_err_vs_oracle"),
           "config": {"workload": WORKLOAD_DESC, "entries_per_update": E,
                      "inputs": "host-built FP64 TR(G) + noise, rounded to FP32; same bytes as the oracle's",
                      "l2": "flushed between steps (256 MB write outside the timed events)",
                      "parallelism": f"replicas x{world} (independent streams, no collective)"},
           "roofline": roofline, "peaks": peaks, "kernel_time_share": kernel_share,
           "gpu_launches": int(launches), "clocks": clk}

    # ---- e2e: public API with pinned host slabs, status + core read back per step ----
    ctx_e = p.str_init_cores(cores0, X0=p.paper_layout(X32[..., :W2.t_init]), compute="f32",
                             sweeps=W2.sweeps, t_capacity=cap)
    nsl = min(a.steps + a.warmup, (W2.T - W2.t_init) // W2.t_new)
    host = []
    for j in range(nsl):
        d = slab(X32, W2, j)
        rev = list(range(d.dim() - 1, -1, -1))
        h = torch.empty(list(d.shape)[::-1], dtype=d.dtype, pin_memory=True)
        h.copy_(d.permute(rev))
        host.append(h.permute(rev))
    st_e = torch.cuda.Stream()
    with torch.cuda.stream(st_e):
        for j in range(a.warmup):
            ctx_e.update(host[j % nsl])
            ctx_e.core(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(a.steps):
            ctx_e.update(host[(a.warmup + j) % nsl])
            ctx_e.core(1)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(torch, time.perf_counter() - t0, world, "cuda")
    ctx_e.close()
    out["e2e"] = {"value": job_rate(a.steps * E, world, e2e_s), "unit": "entries/s",
                  "h2d_bytes_per_step": E * 4, "d2h_bytes_per_step": 4 + 64 * 64 * 8,
                  "note": "str_update with on_host=1 pinned slab (copy inside the call, status read) "
                          "+ str_get_core(1), wall clock"}

    # ---- accuracy checks (GPU side): the first CHECK_UPDATES updates of each arm ----
    tchk = W2.t_init + CHECK_UPDATES * W2.t_new
    checks = {}
    ctxc = make("f32", X32)
    for j in range(CHECK_UPDATES):
        ctxc.update(slab(X32, W2, j))
    checks["order4_f32"] = {"gpu_fit": ctxc.fit_error(X32[..., :tchk]), "cores": ctxc.cores()}
    ctxc.close()

    # ---- plain FP64 GPU arm (same steps and warm-up as the headline) ----
    if not a.no_fp64:
        ctx64 = make("f64", X)
        t64, l64, _ = timed_updates(p, torch, ctx64, lambda j: slab(X, W2, j), a.steps, a.warmup, flush=flush)
        ctx64.close()
        ms64 = sum(t64) / a.steps
        out["fp64_arm"] = {"value": a.steps * E / (sum(t64) / 1e3), "unit": "entries/s", "ms_per_step": ms64,
                           "steps": a.steps, "warmup": a.warmup, "dtype": "f64", "gpu_launches": int(l64),
                           "step": step_roofline(ms64, F2, peaks["fp64_fma_tflops"], E * 8, hbm, "fp64"),
                           "step_note": "t_bound = max(F_alg / measured FP64 FMA peak, one FP64 slab read / HBM)"}
        ctxc = make("f64", X)
        for j in range(CHECK_UPDATES):
            ctxc.update(slab(X, W2, j))
        checks["order4_f64"] = {"gpu_fit": ctxc.fit_error(X[..., :tchk]), "cores": ctxc.cores()}
        ctxc.close()
        c32, c64 = checks["order4_f32"]["cores"], checks["order4_f64"]["cores"]
        out["fp64_arm"]["f32_vs_f64_arm"] = {
            "max_core_rel_diff": max(float(np.linalg.norm(u - v) / np.linalg.norm(v)) for u, v in zip(c32, c64)),
            "fit_rel_diff": abs(checks["order4_f32"]["gpu_fit"] - checks["order4_f64"]["gpu_fit"]) /
            checks["order4_f64"]["gpu_fit"], "updates": CHECK_UPDATES}
    del X
    # ---- secondary rows ----
    if not a.no_rstr:
        out["rstr"] = rstr_rows(p, torch, flush, rank, peaks, checks)
    if not a.no_batch:
        out["batch"] = batch_rows(p, torch, flush, rank, peaks, checks)
    if not a.no_loss:
        out["loss"] = loss_rows(p, torch, flush, rank, peaks, checks)
    if not a.no_large:
        out["standin_60x5"] = large_rows(p, torch, flush, rank, peaks)
    # ---- CPU oracle leg (rank 0, N = 1): baseline timing and fit errors on the same bytes ----
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu, fits = cpu_oracle_leg(Xh, cores0, checks, a)
        out["cpu_baseline"] = cpu
        out["fit_err_vs_oracle"] = fits["order4_f32"]
        if "order4_f64" in fits and "fp64_arm" in out:
            out["fp64_arm"]["fit_err_vs_oracle"] = fits["order4_f64"]
        for k in ("uniform", "leverage", "ksrft"):
            if "rstr" in out and f"rstr_{k}" in fits:
                out["rstr"][k]["fit_err_vs_oracle"] = fits[f"rstr_{k}"]
        if "batch" in out and "batch" in fits:
            out["batch"]["fit_err_vs_oracle"] = fits["batch"]
        if "loss" in out and "loss" in fits:
            out["loss"]["loss_vs_oracle"] = fits["loss"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def rstr_rows(p, torch, flush, rank, peaks, checks, steps=4, warmup=2, nchk=2):
    """rSTR-U/L/K updates on the 512x512xT BF16 workload (sketch 2000, Philox seed 7)."""
    seed = W3.seed + 1000 * rank
    G, Xh, _ = host_workload(W3, seed)
    rng = np.random.default_rng(seed + 300)
    init = [g + INIT_PERTURB * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :W3.t_init, :]
    Xb = bf16_device(torch, Xh)
    E = int(np.prod(W3.dims)) * W3.t_new
    m, R = W3.sketch_m, W3.ranks[0]
    # F_alg per update: sampled MTTKRPs 2 I_n m R^2 (spatial modes) + 2 t_new m R^2 (temporal),
    # sketched Grams 2 m R^4 per mode (FP32 pipe, pair arithmetic); bytes: the BF16 slab once
    f_mma = 2.0 * m * R * R * (sum(W3.dims) + W3.t_new)
    f_gram = 2.0 * m * R ** 4 * len(W3.ranks)
    rows = {}
    tchk = W3.t_init + nchk * W3.t_new
    for sk in ("uniform", "leverage", "ksrft"):
        def make(profile=0):
            return p.str_init_cores(init, X0=p.paper_layout(Xb[..., :W3.t_init]), compute="f32", sketch=sk,
                                    m=m, seed=W3.philox_seed, async_status=1, profile=profile,
                                    t_capacity=W3.t_init + (steps + warmup + 2) * W3.t_new)
        ctx = make()
        times, launches, _ = timed_updates(p, torch, ctx, lambda j: slab(Xb, W3, j), steps, warmup,
                                           randomized=True, flush=flush)
        ctx.close()
        ctxp = make(profile=1)
        _, _, pst = timed_updates(p, torch, ctxp, lambda j: slab(Xb, W3, j), steps, warmup,
                                  randomized=True, flush=flush, profile=True)
        ctxp.close()
        tot = sum(pst["class_ms"].values())
        ms = sum(times) / steps
        f = f_mma + f_gram + (5.0 * E * np.log2(E) if sk == "ksrft" else 0.0)
        rows[sk] = {"value": steps * E / (sum(times) / 1e3), "unit": "entries/s",
                    "ms_per_step": ms, "gpu_launches_per_step": launches / steps,
                    "kernel_time_share": {k: round(v / tot, 4) for k, v in pst["class_ms"].items() if v > 0},
                    "step": step_roofline(ms, f, peaks["tf32_tflops"], E * 2 + (E * 16 if sk == "ksrft" else 0),
                                          peaks["hbm_gbs"], "tf32")}
        # accuracy check: the first nchk updates, fit over the data seen, on the BF16 values and
        # on the original FP64 values
        ctxc = make()
        for j in range(nchk):
            ctxc.rupdate(slab(Xb, W3, j))
        Xo = to_device(torch, Xh[..., :tchk])
        checks[f"rstr_{sk}"] = {"gpu_fit_bf16_data": ctxc.fit_error(Xb[..., :tchk]),
                                "gpu_fit_original_data": ctxc.fit_error(Xo)}
        ctxc.close()
        del Xo
    checks["rstr_data"] = {"X": Xh[..., :tchk], "init": init, "updates": nchk}
    rows["workload"] = ("rand3: 512x512xT, T=200, TR-ranks all 10, BF16 slab, FP32 slab-side arithmetic, "
                        "sketch size 2000, Philox seed 7, init = true cores + 0.05 N(0,1) on 40 slices, "
                        "updates of 5 slices")
    rows["step_note"] = ("t_bound = max((2 m R^2 (I_1 + I_2 + t_new) + 2 N m R^4 [+ 5 E log2 E for KSRFT]) / "
                         "TF32 peak, BF16 slab [+ complex mixed slab] bytes / HBM)")
    return rows


def batch_rows(p, torch, flush, rank, peaks, checks, steps=4, warmup=6, count=256, nchk=16):
    """Batched streams: `count` independent order-3 streams of uneven sizes
    (spatial dims in [16,128], TR-ranks in {2..12}, each stream with its own
    number of new slices in 1..16 per step, held for the run), Gaussian cores
    plus noise at 1e-2 relative, initial cores = true cores + 0.05 N(0,1), BF16
    slabs, FP32 slab-side arithmetic, one sweep.  One str_update_batch per step
    (the work-list launches, one CUDA graph per step) against one str_update per
    context per step, same data.  Streams whose own update takes the tensor-core
    MTTKRP differ from the batch (SIMT MTTKRP for every stream) by rounding."""
    specs = synth.uneven_streams(count=count, steps=1, seed=5 + 1000 * rank)
    data, entries, flop, nbytes = [], 0, 0.0, 0
    for i, sp in enumerate(specs):
        tn = sp.t_news[0]
        T = sp.t_init + (warmup + steps + 1) * tn
        G = synth.gaussian_cores(tuple(sp.dims) + (T,), sp.ranks, 7000 + i)
        Xh = synth.add_noise(host_tr_tensor(G), synth.gaussian_tensor(tuple(sp.dims) + (T,), 7100 + i), BATCH_NOISE)
        Xb = bf16_device(torch, Xh)
        rng = np.random.default_rng(7200 + i)
        init = [g + INIT_PERTURB * rng.standard_normal(g.shape) for g in G]
        init[-1] = init[-1][:, :sp.t_init, :]
        data.append((sp, tn, Xb, init, Xh if i < nchk else None))
        e = int(np.prod(sp.dims)) * tn
        entries += e
        flop += str_flop(sp.dims, tn, sp.ranks, 1)
        nbytes += 2 * e

    def make():
        return [p.str_init_cores(init, X0=p.paper_layout(Xb[..., :sp.t_init]), compute="f32", sweeps=1,
                                 t_capacity=sp.t_init + (warmup + steps + 1) * tn, async_status=1)
                for sp, tn, Xb, init, _ in data]

    def slabs(j):
        return [Xb[..., sp.t_init + j * tn:sp.t_init + (j + 1) * tn] for sp, tn, Xb, _, _ in data]

    def run(step_fn):
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for j in range(warmup):
                step_fn(j)
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for j in range(steps):
                flush.zero_()
                evs[j][0].record(stream)
                step_fn(warmup + j)
                evs[j][1].record(stream)
            torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    ctxs = make()
    ms_batch = run(lambda j: p.str_update_batch(ctxs, slabs(j)))
    seq = make()
    ms_seq = run(lambda j: [c.update(x) for c, x in zip(seq, slabs(j))])
    diff = max(float(np.linalg.norm(a.core(n) - b.core(n)) / np.linalg.norm(b.core(n)))
               for a, b in zip(ctxs, seq) for n in (1, 2, 3))
    launches = ctxs[0].stats()["kernel_launches"]
    for c in ctxs + seq:
        c.close()
    # accuracy check: one batched update of every stream, fit of the first nchk streams
    ctxs = make()
    p.str_update_batch(ctxs, slabs(0))
    fits = []
    for (sp, tn, Xb, init, Xh), c in zip(data[:nchk], ctxs[:nchk]):
        t1 = sp.t_init + tn
        fits.append({"bf16_data": c.fit_error(Xb[..., :t1]),
                     "original_data": c.fit_error(to_device(torch, Xh[..., :t1]))})
    for c in ctxs:
        c.close()
    checks["batch"] = {"gpu": fits, "data": [(d[4], d[3], d[1], d[0].t_init) for d in data[:nchk]]}
    ms = ms_batch / steps
    return {"value": steps * entries / (ms_batch / 1e3), "unit": "entries/s",
            "ms_per_step": ms,
            "sequential": {"value": steps * entries / (ms_seq / 1e3), "ms_per_step": ms_seq / steps},
            "max_core_rel_diff_vs_sequential": diff,
            "gpu_launches_per_step": launches,
            "entries_per_step": entries,
            "step": step_roofline(ms, flop, peaks["tf32_tflops"], nbytes, peaks["hbm_gbs"], "tf32"),
            "step_note": "t_bound = max(sum over streams of 2 E sum_n R_n R_{n+1} / TF32 peak, BF16 slabs / HBM)",
            "workload": (f"{count} independent order-3 streams, spatial dims uniform in [16,128], TR-ranks "
                         "in {2..12}, 1-16 new slices per step (fixed per stream), Gaussian cores, noise 1e-2, "
                         "init = true cores + 0.05 N(0,1), BF16 slabs, FP32 slab-side arithmetic, 1 sweep; one "
                         "str_update_batch per step vs one str_update per stream")}


def large_rows(p, torch, flush, rank, peaks, steps=3, warmup=3):
    """Stand-in for the paper's largest synthetic tensor (60 x 60 x 60 x 60 x 60,
    Sec. 4.3): Gaussian TR cores of rank 5 plus Gaussian noise (relative 1e-3),
    decomposition of the first 12 slices (20%) given as the perturbed true cores,
    then STR updates of 5 slices (64.8 M entries, 259 MB FP32 per slab), one
    sweep, FP32 slab arithmetic.  The tensor is made on the device by the
    library's reconstruction (so this row has no oracle comparison: the oracle's
    inputs never come from the library).  Reports the update rate and the
    stage-1 kernel's achieved HBM bandwidth at this size."""
    dims, T, R, t_init, t_new = (60, 60, 60, 60), 60, 5, 12, 5
    seed = 77 + 1000 * rank
    G = synth.gaussian_cores(dims + (T,), (R,) * 5, seed)
    truth = p.str_init_cores(G, X0=None, t_capacity=T)
    X = truth.reconstruct(0, T, dtype=torch.float32)
    truth.close()
    gen = torch.Generator(device="cuda").manual_seed(seed + 100)
    noise = torch.randn(X.shape, generator=gen, device="cuda", dtype=torch.float32)
    X.add_(noise, alpha=float(1e-3 * X.norm() / noise.norm()))
    del noise
    X = p.paper_layout(X)
    rng = np.random.default_rng(seed + 200)
    init = [g + 0.05 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :t_init, :]
    E = int(np.prod(dims)) * t_new

    def sl(j):
        return X[..., t_init + j * t_new:t_init + (j + 1) * t_new]

    def make(profile=0):
        return p.str_init_cores(init, X0=X[..., :t_init], compute="f32", sweeps=1, async_status=1,
                                t_capacity=T, profile=profile)
    ctx = make()
    times, launches, _ = timed_updates(p, torch, ctx, sl, steps, warmup, flush=flush)
    ctx.close()
    ctxp = make(profile=1)
    _, _, pst = timed_updates(p, torch, ctxp, sl, steps, warmup, flush=flush, profile=True)
    ctxp.close()
    k_ms, k_n = pst["class_ms"], pst["class_launches"]
    s1 = k_ms["mttkrp"] / max(1, k_n["mttkrp"])
    gbs = E * 4 / (s1 / 1e3) / 1e9
    tot = sum(k_ms.values())
    ms = sum(times) / steps
    hbm = peaks["hbm_gbs"]
    return {"value": steps * E / (sum(times) / 1e3), "unit": "entries/s", "ms_per_step": ms,
            "gpu_launches_per_step": launches / steps,
            "stage1": {"kernel": "stage1_ws_kernel", "avg_launch_ms": round(s1, 5), "launches": int(k_n["mttkrp"]),
                       "bytes_per_launch": E * 4, "achieved_gbs": round(gbs, 1), "peak": hbm,
                       "frac": round(gbs / hbm, 4), "peak_note": f"HBM copy bandwidth, {peaks['hbm_note']}"},
            "step": step_roofline(ms, str_flop(dims, t_new, (R,) * 5, 1), peaks["tf32_tflops"], E * 4, hbm, "tf32"),
            "kernel_time_share": {k: round(v / tot, 4) for k, v in k_ms.items() if tot > 0 and v > 0},
            "fit_err_vs_oracle": None,
            "fit_err_note": "not compared: this row's tensor is made by the library on the device",
            "workload": ("60x60x60x60x60 stand-in (Sec. 4.3 largest synthetic tensor): TR-ranks 5, Gaussian cores, "
                         "noise 1e-3, init on 12 slices, updates of 5 slices (64.8 M entries, FP32), 1 sweep")}


def loss_rows(p, torch, flush, rank, peaks, checks, steps=3, warmup=3):
    """Masked TR fit loss and its backward on the 32x32x32x32x100 FP32 tensor
    (TR-ranks 6, 30% of the entries hidden, mask as packed bits): one forward
    (loss) and one backward (gradients of all five cores) per step.  The tensor
    is the TR tensor of Gaussian cores plus Gaussian noise at 1e-2 relative
    Frobenius norm (so the residual is well above FP32 rounding), built on the
    host; the cores are the true cores rounded to FP32."""
    W = synth.WORKLOADS["masked5"]
    dims = tuple(W.dims) + (W.T,)
    seed = W.seed + 1000 * rank
    G = synth.gaussian_cores(dims, W.ranks, seed)
    G32 = [g.astype(np.float32).astype(np.float64) for g in G]
    Xh = synth.add_noise(host_tr_tensor(G), synth.gaussian_tensor(dims, seed + 100), LOSS_NOISE).astype(np.float32)
    X = to_device(torch, Xh)
    mask = synth.bernoulli_keep_mask(dims, 0.3, seed)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = [torch.from_numpy(a).to("cuda", torch.float32) for a in p.cores_to_abi(G32)]
    E = int(np.prod(dims))

    def timed(fn):
        stream = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for j in range(steps):
                flush.zero_()
                evs[j][0].record(stream)
                fn()
                evs[j][1].record(stream)
            torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    ms_f = timed(lambda: p.tr_masked_loss_fwd(cores, X, bits))
    ms_b = timed(lambda: p.tr_masked_loss_bwd(cores, X, bits, 1.0))
    loss = float(p.tr_masked_loss_fwd(cores, X, bits).item())
    checks["loss"] = {"gpu": loss, "X": Xh, "cores": G32, "mask": mask}
    in_bytes = E * 4 + bits.numel() * 4
    hbm = peaks["hbm_gbs"]
    t_bound_ms = in_bytes / (hbm * 1e9) * 1e3
    return {"value": E / ((ms_f + ms_b) / 1e3), "unit": "entries/s", "ms_fwd": ms_f, "ms_bwd": ms_b,
            "fwd_read_gbs": in_bytes / (ms_f / 1e3) / 1e9, "fwd_frac_of_hbm": in_bytes / (ms_f / 1e3) / 1e9 / hbm,
            "t_bound_fused_fwd_bwd_ms": t_bound_ms, "frac_step": t_bound_ms / (ms_f + ms_b), "loss": loss,
            "step_note": "t_bound = one read of X and the mask bits / HBM (one fused pass serves fwd and bwd)",
            "workload": ("masked5: 32x32x32x32x100 FP32 (104.9 M entries, 419 MB), TR-ranks all 6, noise 1e-2, "
                         "Bernoulli(0.3) "
                         "hidden entries as packed mask bits; one tr_masked_loss_fwd + one tr_masked_loss_bwd "
                         "(all 5 core gradients) per step")}


# ---------------------------------------------------------------------------
# CPU oracle leg (the cpu_baseline and the fit errors against the oracle) and
# the reference arm
# ---------------------------------------------------------------------------
def oracle_sample(Xh, cores0, nupd=1):
    """The FP64 oracle's STR update (Alg. 4, 5 sweeps) on the order4 workload:
    initialisation stage on 40 slices (untimed), then `nupd` timed updates.
    Returns (seconds, final state, temporal rows seen)."""
    from oracle import stream as ost
    st = ost.str_init(Xh[..., :W2.t_init], cores0)
    t = W2.t_init
    t0 = time.perf_counter()
    for _ in range(nupd):
        ost.str_update(st, Xh[..., t:t + W2.t_new], sweeps=W2.sweeps)
        t += W2.t_new
    return time.perf_counter() - t0, st, t


def cpu_threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


def _rel(a, b):
    return abs(a - b) / abs(b) if b else None


def single_thread_sample(Xh, cores0):
    """One oracle update timed in a child process with every BLAS pool at one
    thread (the variables must be set before numpy loads)."""
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "sample.npz")
        np.savez(path, X=Xh[..., :W2.t_init + W2.t_new], **{f"G{k}": g for k, g in enumerate(cores0)})
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", path],
                           capture_output=True, text=True, env=env, timeout=600)
        if r.returncode != 0:
            return {"error": (r.stderr.strip().splitlines() or ["failed"])[-1]}
        return json.loads(r.stdout.strip().splitlines()[-1])


def main_oracle_sample(path):
    z = np.load(path)
    cores0 = [z[f"G{k}"] for k in range(len(W2.ranks))]
    secs, _, _ = oracle_sample(z["X"], cores0, 1)
    E = int(np.prod(W2.dims)) * W2.t_new
    print(json.dumps({"value": E / secs, "unit": "entries/s", "seconds": secs, "cores": cpu_threads()}))


def cpu_oracle_leg(Xh, cores0, checks, a):
    """The FP64 oracle on the host cores, on bounded samples of each row's
    workload and the same bytes its GPU arm read: timing (the cpu_baseline) and
    the relative fit error of each GPU arm against it."""
    from oracle import loss as olo
    from oracle import stream as ost
    from oracle import tr as otr
    fits = {}
    E = int(np.prod(W2.dims)) * W2.t_new
    # order-4, FP32 arm: the oracle on the FP32-rounded bytes; FP64 arm: on the FP64 bytes
    X32h = Xh.astype(np.float32).astype(np.float64)
    secs, st, t = oracle_sample(X32h, cores0, CHECK_UPDATES)
    e_or = otr.fit_error(X32h[..., :t], st.cores)
    g = checks["order4_f32"]
    fits["order4_f32"] = {"gpu": g["gpu_fit"], "oracle": e_or, "rel_diff": _rel(g["gpu_fit"], e_or),
                          "max_core_rel_diff": max(float(np.linalg.norm(u - v) / np.linalg.norm(v))
                                                   for u, v in zip(g["cores"], st.cores)),
                          "updates": CHECK_UPDATES, "data": "FP32-rounded slab values, as the GPU arm read them"}
    cpu = {"value": CHECK_UPDATES * E / secs, "unit": "entries/s", "cores": cpu_threads(), "kind": "oracle",
           "sample": (f"{CHECK_UPDATES} STR updates of 10 slices (5 sweeps) of the order4 workload, FP64 numpy "
                      "oracle, after its initialisation stage (untimed)"), "seconds": secs}
    if "order4_f64" in checks:
        _, st64, t = oracle_sample(Xh, cores0, CHECK_UPDATES)
        e64 = otr.fit_error(Xh[..., :t], st64.cores)
        g = checks["order4_f64"]
        fits["order4_f64"] = {"gpu": g["gpu_fit"], "oracle": e64, "rel_diff": _rel(g["gpu_fit"], e64),
                              "max_core_rel_diff": max(float(np.linalg.norm(u - v) / np.linalg.norm(v))
                                                       for u, v in zip(g["cores"], st64.cores)),
                              "updates": CHECK_UPDATES, "data": "FP64 slab values"}
    cpu["single_thread"] = single_thread_sample(Xh, cores0)
    # rSTR rows: the oracle on the BF16 values and on the original values
    if "rstr_data" in checks:
        rd = checks["rstr_data"]
        Xo = rd["X"]
        Xr = synth.to_bf16_values(Xo)
        for sk in ("uniform", "leverage", "ksrft"):
            g = checks[f"rstr_{sk}"]
            res = {"updates": rd["updates"]}
            for name, Xd, gk in (("bf16_data", Xr, "gpu_fit_bf16_data"),
                                 ("original_data", Xo, "gpu_fit_original_data")):
                st = ost.rstr_init(Xd[..., :W3.t_init], rd["init"], sk, W3.sketch_m, W3.philox_seed)
                t = W3.t_init
                for _ in range(rd["updates"]):
                    ost.rstr_update(st, Xd[..., t:t + W3.t_new])
                    t += W3.t_new
                e = otr.fit_error(Xd[..., :t], st.cores)
                res[name] = {"gpu": g[gk], "oracle": e, "rel_diff": _rel(g[gk], e)}
            fits[f"rstr_{sk}"] = res
    # batched streams: the first streams, one update each
    if "batch" in checks:
        out = []
        for (Xo, init, tn, t_init), g in zip(checks["batch"]["data"], checks["batch"]["gpu"]):
            rec = {}
            for name, Xd in (("bf16_data", synth.to_bf16_values(Xo)), ("original_data", Xo)):
                st = ost.str_init(Xd[..., :t_init], init)
                ost.str_update(st, Xd[..., t_init:t_init + tn])
                e = otr.fit_error(Xd[..., :t_init + tn], st.cores)
                rec[name] = _rel(g[name], e)
            out.append(rec)
        fits["batch"] = {"streams": len(out), "updates": 1,
                         "max_rel_diff_bf16_data": max(r["bf16_data"] for r in out),
                         "max_rel_diff_original_data": max(r["original_data"] for r in out),
                         "first_stream": checks["batch"]["gpu"][0]}
    # masked loss: the loss value on the same FP32 bytes and FP32-rounded cores
    if "loss" in checks:
        lc = checks["loss"]
        ref = olo.masked_loss(lc["X"].astype(np.float64), lc["cores"], lc["mask"])
        fits["loss"] = {"gpu": lc["gpu"], "oracle": ref, "rel_diff": _rel(lc["gpu"], ref)}
    return cpu, fits


def main_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from oracle import stream as ost
    _, X, init = host_workload(W2, W2.seed)
    X = X.astype(np.float32).astype(np.float64)        # the FP32 slab values the GPU arm reads
    st = ost.str_init(X[..., :W2.t_init], init)
    nsl = (W2.T - W2.t_init) // W2.t_new
    times = []
    for j in range(a.warmup + a.steps):
        t = W2.t_init + (j % nsl) * W2.t_new
        t0 = time.perf_counter()
        ost.str_update(st, X[..., t:t + W2.t_new], sweeps=W2.sweeps)
        if j >= a.warmup:
            times.append(time.perf_counter() - t0)
    E = int(np.prod(W2.dims)) * W2.t_new
    value = a.steps * E / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / a.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "entries_per_update": E,
                                           "inputs": "host-built FP64 TR(G) + noise, rounded to FP32; same "
                                                     "bytes and initial cores as the GPU arm"},
           "cpu_baseline": {"value": value, "unit": "entries/s", "kind": "oracle", "cores": cpu_threads(),
                            "sample": "each step = one STR update of 10 slices (5 sweeps) by the FP64 oracle"},
           "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# kernel evidence at enlarged shapes (each prints one JSON line; run under ncu
# with a kernel filter for the counters)
# ---------------------------------------------------------------------------
def evidence_stage1_r12(p, torch, steps=2, warmup=1):
    """Stage 1 at a shape where its arithmetic intensity crosses the tensor
    ridge: order 5, 60 x 60 x 60 x 60 spatial, TR-ranks 12 (R_k R_{k+1} = 144),
    5-slice FP32 slabs (64.8 M entries, 259 MB), one sweep.  Algorithmic
    intensity 2 R^2 / 4 = 72 flop/B; the 3-term TF32 split executes 3 times the
    MMA work (216 flop/B, above the TF32 / HBM ridge)."""
    dims, R, t_init, t_new = (60, 60, 60, 60), 12, 12, 5
    T = t_init + (steps + warmup) * t_new
    G = synth.gaussian_cores(dims + (T,), (R,) * 5, 88)
    truth = p.str_init_cores(G, X0=None, t_capacity=T)
    X = p.paper_layout(truth.reconstruct(0, T, dtype=torch.float32))
    truth.close()
    rng = np.random.default_rng(288)
    init = [g + 0.05 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :t_init, :]
    E = int(np.prod(dims)) * t_new
    ctx = p.str_init_cores(init, X0=X[..., :t_init], compute="f32", sweeps=1, async_status=1, profile=1,
                           t_capacity=T)
    times, _, st = timed_updates(p, torch, ctx, lambda j: X[..., t_init + j * t_new:t_init + (j + 1) * t_new],
                                 steps, warmup)
    ctx.close()
    s1 = st["class_ms"]["mttkrp"] / max(1, st["class_launches"]["mttkrp"])
    peaks = measure_peaks(p, torch)
    flop_alg, flop_exec = 2.0 * E * R * R, 6.0 * E * R * R
    return {"evidence": "stage1_r12", "workload": "60^4 x 5 FP32 slab, TR-ranks 12 (R_k R_{k+1} = 144), one sweep",
            "ms_per_update": sum(times) / steps, "stage1_avg_launch_ms": s1, "stage1_launches": st["class_launches"]["mttkrp"],
            "stage1_hbm_gbs": E * 4 / (s1 / 1e3) / 1e9, "stage1_alg_tflops": flop_alg / (s1 / 1e3) / 1e12,
            "stage1_exec_tflops": flop_exec / (s1 / 1e3) / 1e12, "tf32_tflops": peaks["tf32_tflops"],
            "hbm_gbs": peaks["hbm_gbs"], "hbm_note": peaks["hbm_note"],
            "kernel_time_share": {k: round(v / sum(st["class_ms"].values()), 4)
                                  for k, v in st["class_ms"].items() if v > 0}}


def evidence_sampling_m1e6(p, torch, steps=2, warmup=1):
    """Sampling, gather and sketched-Gram kernels at a sketch size of one
    million rows: order 3, 500 x 500 spatial (the paper's 500^3 synthetic
    tensor, Sec. 4.3), TR-ranks 10, 5-slice BF16 slabs, rSTR-U and rSTR-L with
    m = 10^6."""
    dims, R, t_init, t_new, m = (500, 500), 10, 20, 5, 1000000
    T = t_init + (steps + warmup) * t_new
    G = synth.gaussian_cores(dims + (T,), (R,) * 3, 99)
    truth = p.str_init_cores(G, X0=None, t_capacity=T)
    Xb = p.paper_layout(truth.reconstruct(0, T, dtype=torch.float32).to(torch.bfloat16))
    truth.close()
    rng = np.random.default_rng(299)
    init = [g + 0.05 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :t_init, :]
    E = int(np.prod(dims)) * t_new
    out = {"evidence": "sampling_m1e6", "workload": "500 x 500 x 5 BF16 slabs, TR-ranks 10, sketch size 10^6"}
    for sk in ("uniform", "leverage"):
        ctx = p.str_init_cores(init, X0=Xb[..., :t_init], compute="f32", sketch=sk, m=m, seed=7, profile=1,
                               async_status=1, t_capacity=T)
        times, _, st = timed_updates(p, torch, ctx, lambda j: Xb[..., t_init + j * t_new:t_init + (j + 1) * t_new],
                                     steps, warmup, randomized=True)
        ctx.close()
        out[sk] = {"ms_per_update": sum(times) / steps,
                   "class_ms_per_update": {k: round(v / steps, 4) for k, v in st["class_ms"].items() if v > 0},
                   "gathered_bytes_per_update": 3 * m * dims[0] * 2 * 2,
                   "note": "gathered fibres: m I_n BF16 values read and written per spatial mode"}
    return out


def evidence_batch256(p, torch, steps=3, warmup=2):
    """The work-list batch alone: 256 uneven order-3 streams as in the bench's
    batch row, a few steps (for ncu captures of the batched Gram, ring and
    solve kernels)."""
    specs = synth.uneven_streams(count=256, steps=1, seed=5)
    data = []
    for i, sp in enumerate(specs):
        tn = sp.t_news[0]
        T = sp.t_init + (warmup + steps + 1) * tn
        Gc = synth.gaussian_cores(tuple(sp.dims) + (T,), sp.ranks, 7000 + i)
        Xh = synth.add_noise(host_tr_tensor(Gc), synth.gaussian_tensor(tuple(sp.dims) + (T,), 7100 + i), BATCH_NOISE)
        init = [g.copy() for g in Gc]
        init[-1] = init[-1][:, :sp.t_init, :]
        data.append((sp, tn, bf16_device(torch, Xh), init))
    ctxs = [p.str_init_cores(init, X0=p.paper_layout(Xb[..., :sp.t_init]), compute="f32", sweeps=1, async_status=1,
                             t_capacity=sp.t_init + (warmup + steps + 1) * tn) for sp, tn, Xb, init in data]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    ms = []
    with torch.cuda.stream(stream):
        for j in range(warmup + steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p.str_update_batch(ctxs, [Xb[..., sp.t_init + j * tn:sp.t_init + (j + 1) * tn] for sp, tn, Xb, _ in data])
            b.record(stream)
            stream.synchronize()
            if j >= warmup:
                ms.append(a.elapsed_time(b))
    launches = ctxs[0].stats()["kernel_launches"]
    for c in ctxs:
        c.close()
    return {"evidence": "batch256", "ms_per_step": sum(ms) / len(ms), "gpu_launches_per_step": launches}


def evidence_masked_loss(p, torch, steps=2, warmup=1):
    """The masked-loss row alone (forward and backward on the 32^4 x 100 FP32
    tensor), a few steps: for the launch list of the loss path."""
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    row = loss_rows(p, torch, flush, 0, {"hbm_gbs": measured_peak("hbm_gbs", 6800.0)[0]}, {}, steps=steps,
                    warmup=warmup)
    return {"evidence": "masked_loss", "ms_fwd": row["ms_fwd"], "ms_bwd": row["ms_bwd"], "loss": row["loss"]}


def main_evidence(a):
    import torch
    import paper_2307_00719_gb300 as p
    torch.cuda.set_device(0)
    fn = {"stage1_r12": evidence_stage1_r12, "sampling_m1e6": evidence_sampling_m1e6,
          "batch256": evidence_batch256, "masked_loss": evidence_masked_loss}[a.evidence]
    print(json.dumps(fn(p, torch)), flush=True)


if __name__ == "__main__":
    args = args_parse()
    if args.evidence:
        main_evidence(args)
    elif args.oracle_sample:
        main_oracle_sample(args.oracle_sample)
    elif args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)
