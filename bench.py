#!/usr/bin/env python
"""Throughput of the streaming tensor-ring update on GB300.

Workload (one "step" = one STR update, every row of the hot path):
  order-4 tensor 64x64x64xT, T = 400, TR-ranks all 8, Gaussian cores, noise at
  SNR 30 dB, initial decomposition on 40 slices, then updates of 10 slices,
  5 sweeps per update, FP32 slab and FP32 slab-side arithmetic (FP64 Gram,
  P_n/Q_n and solves).  Inputs are synthetic and already resident in HBM.

Printed as one JSON line by rank 0.  `--impl reference` times the FP64 CPU
oracle on the same workload (a bounded sample per step) instead.
Secondary rows (same line): the plain FP64 GPU arm of the same workload,
rSTR-U/L/K updates on a 512x512xT BF16 workload (ranks 10, sketch size 2000),
batched updates of 256 uneven order-3 streams, the masked TR fit loss and its
backward on a 32x32x32x32x100 FP32 tensor, and STR updates on a 60^5 stand-in
of the paper's largest synthetic tensor (ranks 5, 5-slice slabs).
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
                 "init on 40 slices, updates of 10 slices, 5 sweeps, FP32 slab")
FLUSH_BYTES = 256 << 20     # > 129 MB L2


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-rstr", action="store_true", help="skip the rSTR rows")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU arm")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-streams row")
    ap.add_argument("--no-loss", action="store_true", help="skip the masked-loss row")
    ap.add_argument("--no-large", action="store_true", help="skip the 60^5 stand-in row")
    return ap.parse_args()


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


# ---------------------------------------------------------------------------
# workload construction (GPU)
# ---------------------------------------------------------------------------
def build_tensor(p, torch, w, seed):
    """X = TR(G_true) + noise, built on the GPU with the library's reconstruct."""
    G = synth.gaussian_cores(tuple(w.dims) + (w.T,), w.ranks, seed)
    truth = p.str_init_cores(G, X0=None, t_capacity=w.T)
    X = truth.reconstruct(0, w.T)                          # FP64, i_1 fastest
    truth.close()
    if w.noise > 0:
        g = torch.Generator(device="cuda").manual_seed(seed + 100)
        E = torch.randn(X.shape[::-1], generator=g, device="cuda", dtype=torch.float64)
        E = E.permute(list(range(E.dim() - 1, -1, -1)))
        X = X + (w.noise * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(E)) * E
    return G, p.paper_layout(X)


def init_cores(p, torch, w, G, X, seed, iters=20):
    """Initial decomposition of the first t_init slices by TR-ALS-NE on the GPU,
    started from the true cores perturbed by 0.3 N(0,1)."""
    rng = np.random.default_rng(seed + 200)
    guess = [g + 0.3 * rng.standard_normal(g.shape) for g in G]
    guess[-1] = guess[-1][:, :w.t_init, :]
    ctx = p.str_init(p.paper_layout(X[..., :w.t_init]), w.ranks, guess, init_max_it=iters)
    cores = ctx.cores()
    ctx.close()
    return cores


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


def main_ours(a):
    import torch
    import paper_2307_00719_gb300 as p
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    seed = W2.seed + 1000 * rank                       # independent replica per rank
    G, X = build_tensor(p, torch, W2, seed)
    cores0 = init_cores(p, torch, W2, G, X, seed)
    X32 = p.paper_layout(X.float())
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    E = int(np.prod(W2.dims)) * W2.t_new
    cap = W2.t_init + (a.warmup + a.steps + 2) * W2.t_new

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
    fit32 = ctx.fit_error(X32[..., :ctx.time_rows()])
    cores32 = ctx.cores()
    ctx.close()

    # ---- profile pass: per-class kernel times (same steps, events per launch) ----
    ctxp = make("f32", X32, profile=1)
    ptimes, _, pst = timed_updates(p, torch, ctxp, lambda j: slab(X32, W2, j), a.steps, a.warmup,
                                   flush=flush, profile=True)
    ctxp.close()
    k_ms, k_n = pst["class_ms"], pst["class_launches"]
    mt_avg_ms = k_ms["mttkrp"] / max(1, k_n["mttkrp"])
    peak_hbm = measured_peak("hbm_gbs", 6685.5)
    slab_bytes = E * 4                                  # one read of the FP32 slab per launch
    achieved = slab_bytes / (mt_avg_ms / 1e3) / 1e9
    sm_clock = (clk.get("sm_mhz") or 1900.0)
    tot = sum(k_ms.values())
    c_avg_ms = k_ms["contract"] / max(1, k_n["contract"])
    RRk = W2.ranks[0] * W2.ranks[1]
    roofline = {"kernel": "stage1_ws_kernel (tcgen05 kind::tf32, 3-term split, TMA-fed, warp-specialised)",
                "bound": "hbm", "achieved": round(achieved, 1), "peak": peak_hbm, "unit": "GB/s",
                "frac": round(achieved / peak_hbm, 4), "traffic": STAGE1_DRAM_BYTES,
                "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one launch, ncu --set full "
                                "on this workload",
                "peak_note": "measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs), of measured",
                "algorithmic_per_launch": {"bytes": slab_bytes, "flop": 2.0 * E * RRk,
                                           "note": "one read of the 64^3 x 10 FP32 slab; 2 E R_1 R_2 flop"},
                "avg_launch_ms": round(mt_avg_ms, 5), "launches": int(k_n["mttkrp"]),
                "tensor_tflops": round(2.0 * E * RRk / (mt_avg_ms / 1e3) / 1e12, 2),
                "stage2": {"kernel": "stage2_kernel (SIMT contraction with chain tables)",
                           "avg_launch_ms": round(c_avg_ms, 5), "launches": int(k_n["contract"]),
                           "read_gbs": round(E // W2.dims[0] * RRk * 4 / max(c_avg_ms, 1e-9) / 1e6, 1)},
                "sm_mhz_median": sm_clock}
    kernel_share = {k: round(v / tot, 4) for k, v in k_ms.items() if tot > 0 and v > 0}

    out = {"metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD_DESC, "entries_per_update": E,
                      "l2": "flushed between steps (256 MB write outside the timed events)",
                      "parallelism": f"replicas x{world} (independent streams, no collective)"},
           "roofline": roofline, "kernel_time_share": kernel_share,
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

    # ---- plain FP64 GPU arm (same steps): throughput and fit error reference ----
    if not a.no_fp64:
        X64 = X
        ctx64 = make("f64", X64)
        t64, _, _ = timed_updates(p, torch, ctx64, lambda j: slab(X64, W2, j), min(a.steps, 4), a.warmup,
                                  flush=flush)
        steps64 = min(a.steps, 4)
        fit64 = ctx64.fit_error(X64[..., :ctx64.time_rows()])
        out["fp64_arm"] = {"value": steps64 * E / (sum(t64) / 1e3), "unit": "entries/s",
                           "ms_per_step": sum(t64) / steps64, "steps": steps64}
        # the FP32 arm over the same first warmup+steps64 updates vs FP64
        ctxc = make("f32", X32)
        for j in range(a.warmup + steps64):
            ctxc.update(slab(X32, W2, j))
        fitc = ctxc.fit_error(X32[..., :ctxc.time_rows()])
        core_rel = max(float(np.linalg.norm(c - d) / np.linalg.norm(d))
                       for c, d in zip(ctxc.cores(), ctx64.cores()))
        ctxc.close()
        ctx64.close()
        out["fit_error"] = {"f32_arm": fitc, "f64_arm": fit64, "rel_diff": abs(fitc - fit64) / fit64,
                            "max_core_rel_diff": core_rel, "f32_arm_after_all_steps": fit32,
                            "updates_compared": a.warmup + steps64}
    # ---- rSTR rows ----
    if not a.no_rstr:
        out["rstr"] = rstr_rows(p, torch, flush, rank)
    if not a.no_batch:
        out["batch"] = batch_rows(p, torch, flush, rank)
    if not a.no_loss:
        out["loss"] = loss_rows(p, torch, flush, rank, peak_hbm)
    if not a.no_large:
        out["standin_60x5"] = large_rows(p, torch, flush, rank, peak_hbm)
    # ---- CPU oracle baseline (rank 0, N = 1) ----
    if rank == 0 and world == 1 and not a.no_cpu:
        out["cpu_baseline"] = cpu_baseline(X, cores0)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback


def rstr_rows(p, torch, flush, rank, steps=4, warmup=2):
    """rSTR-U/L/K updates on the 512x512xT BF16 workload (sketch 2000, Philox seed 7)."""
    seed = W3.seed + 1000 * rank
    G, X = build_tensor(p, torch, W3, seed)
    Xb = p.paper_layout(X.to(torch.bfloat16))
    del X
    rng = np.random.default_rng(seed + 300)
    init = [g + 0.05 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :W3.t_init, :]
    E = int(np.prod(W3.dims)) * W3.t_new
    rows = {}
    for sk in ("uniform", "leverage", "ksrft"):
        ctx = p.str_init_cores(init, X0=p.paper_layout(Xb[..., :W3.t_init]), compute="f32", sketch=sk,
                               m=W3.sketch_m, seed=W3.philox_seed, async_status=1,
                               t_capacity=W3.t_init + (steps + warmup + 2) * W3.t_new)
        times, launches, _ = timed_updates(p, torch, ctx, lambda j: slab(Xb, W3, j), steps, warmup,
                                           randomized=True, flush=flush)
        ctxp = p.str_init_cores(init, X0=p.paper_layout(Xb[..., :W3.t_init]), compute="f32", sketch=sk,
                                m=W3.sketch_m, seed=W3.philox_seed, async_status=1, profile=1,
                                t_capacity=W3.t_init + (steps + warmup + 2) * W3.t_new)
        _, _, pst = timed_updates(p, torch, ctxp, lambda j: slab(Xb, W3, j), steps, warmup,
                                  randomized=True, flush=flush, profile=True)
        tot = sum(pst["class_ms"].values())
        rows[sk] = {"value": steps * E / (sum(times) / 1e3), "unit": "entries/s",
                    "ms_per_step": sum(times) / steps, "gpu_launches_per_step": launches / steps,
                    "kernel_time_share": {k: round(v / tot, 4) for k, v in pst["class_ms"].items() if v > 0}}
        ctx.close()
        ctxp.close()
    rows["workload"] = ("rand3: 512x512xT, T=200, TR-ranks all 10, BF16 slab, FP32 slab-side arithmetic, "
                        "sketch size 2000, Philox seed 7, updates of 5 slices")
    return rows


def batch_rows(p, torch, flush, rank, steps=4, warmup=6, count=256):
    """Batched streams: `count` independent order-3 streams of uneven sizes
    (spatial dims in [16,128], TR-ranks in {2..12}, each stream with its own
    number of new slices in 1..16 per step, held for the run), BF16 slabs, FP32
    slab-side arithmetic, one sweep.  One str_update_batch per step (all
    contexts as concurrent branches of one replayed graph) against one
    str_update per context per step (each context's own graph), same data."""
    specs = synth.uneven_streams(count=count, steps=1, seed=5 + 1000 * rank)
    data, entries = [], 0
    for i, sp in enumerate(specs):
        tn = sp.t_news[0]
        T = sp.t_init + (warmup + steps + 1) * tn
        G = synth.gaussian_cores(tuple(sp.dims) + (T,), sp.ranks, 7000 + i)
        truth = p.str_init_cores(G, X0=None, t_capacity=T)
        Xb = p.paper_layout(truth.reconstruct(0, T).to(torch.bfloat16))
        truth.close()
        init = [g.copy() for g in G]
        init[-1] = init[-1][:, :sp.t_init, :]
        data.append((sp, tn, Xb, init))
        entries += int(np.prod(sp.dims)) * tn

    def make():
        return [p.str_init_cores(init, X0=p.paper_layout(Xb[..., :sp.t_init]), compute="f32", sweeps=1,
                                 t_capacity=sp.t_init + (warmup + steps + 1) * tn, async_status=1)
                for sp, tn, Xb, init in data]

    def slabs(j):
        return [Xb[..., sp.t_init + j * tn:sp.t_init + (j + 1) * tn] for sp, tn, Xb, _ in data]

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
    same = all(np.array_equal(a.core(n), b.core(n)) for a, b in zip(ctxs[:8], seq[:8]) for n in (1, 2, 3))
    for c in ctxs + seq:
        c.close()
    return {"value": steps * entries / (ms_batch / 1e3), "unit": "entries/s",
            "ms_per_step": ms_batch / steps,
            "sequential": {"value": steps * entries / (ms_seq / 1e3), "ms_per_step": ms_seq / steps},
            "bit_identical_to_sequential": bool(same),
            "entries_per_step": entries,
            "workload": (f"{count} independent order-3 streams, spatial dims uniform in [16,128], TR-ranks "
                         "in {2..12}, 1-16 new slices per step (fixed per stream), BF16 slabs, FP32 slab-side "
                         "arithmetic, 1 sweep; one str_update_batch per step vs one str_update per stream")}


def large_rows(p, torch, flush, rank, peak_hbm, steps=3, warmup=3):
    """Stand-in for the paper's largest synthetic tensor (60 x 60 x 60 x 60 x 60,
    Sec. 4.3): Gaussian TR cores of rank 5 plus Gaussian noise (relative 1e-3),
    decomposition of the first 12 slices (20%) given as the perturbed true cores,
    then STR updates of 5 slices (64.8 M entries, 259 MB FP32 per slab), one
    sweep, FP32 slab arithmetic.  The tensor is made on the device by the
    library's reconstruction.  Reports the update rate and the stage-1 kernel's
    achieved HBM bandwidth at this size."""
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
    return {"value": steps * E / (sum(times) / 1e3), "unit": "entries/s", "ms_per_step": sum(times) / steps,
            "gpu_launches_per_step": launches / steps,
            "stage1": {"kernel": "stage1_ws_kernel", "avg_launch_ms": round(s1, 5), "launches": int(k_n["mttkrp"]),
                       "bytes_per_launch": E * 4, "achieved_gbs": round(gbs, 1), "peak": peak_hbm,
                       "frac": round(gbs / peak_hbm, 4), "peak_note": "measured HBM copy bandwidth, of measured"},
            "kernel_time_share": {k: round(v / tot, 4) for k, v in k_ms.items() if tot > 0 and v > 0},
            "workload": ("60x60x60x60x60 stand-in (Sec. 4.3 largest synthetic tensor): TR-ranks 5, Gaussian cores, "
                         "noise 1e-3, init on 12 slices, updates of 5 slices (64.8 M entries, FP32), 1 sweep")}


def loss_rows(p, torch, flush, rank, peak_hbm, steps=3, warmup=3):
    """Masked TR fit loss and its backward on the 32x32x32x32x100 FP32 tensor
    (TR-ranks 6, 30% of the entries hidden, mask as packed bits): one forward
    (loss) and one backward (gradients of all five cores) per step.  The tensor
    is the TR tensor of Gaussian cores (no noise), made on the device by the
    library's reconstruction."""
    W = synth.WORKLOADS["masked5"]
    dims = tuple(W.dims) + (W.T,)
    seed = W.seed + 1000 * rank
    G = synth.gaussian_cores(dims, W.ranks, seed)
    truth = p.str_init_cores(G, X0=None, t_capacity=W.T)
    X = p.paper_layout(truth.reconstruct(0, W.T, dtype=torch.float32))
    truth.close()
    bits = torch.from_numpy(synth.pack_mask_bits(synth.bernoulli_keep_mask(dims, 0.3, seed))
                            .view(np.int32)).cuda()
    cores = [torch.from_numpy(a).to("cuda", torch.float32) for a in p.cores_to_abi(G)]
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
    in_bytes = E * 4 + bits.numel() * 4
    return {"value": E / ((ms_f + ms_b) / 1e3), "unit": "entries/s", "ms_fwd": ms_f, "ms_bwd": ms_b,
            "fwd_read_gbs": in_bytes / (ms_f / 1e3) / 1e9, "fwd_frac_of_measured_hbm": in_bytes / (ms_f / 1e3) / 1e9 / peak_hbm,
            "t_bound_fused_fwd_bwd_ms": in_bytes / (peak_hbm * 1e9) * 1e3, "loss": loss,
            "workload": ("masked5: 32x32x32x32x100 FP32 (104.9 M entries, 419 MB), TR-ranks all 6, Bernoulli(0.3) "
                         "hidden entries as packed mask bits; one tr_masked_loss_fwd + one tr_masked_loss_bwd "
                         "(all 5 core gradients) per step")}


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_sample(Xh, cores0, nupd=1):
    """The FP64 oracle's STR update (Alg. 4, 5 sweeps) on the order4 workload:
    initialisation stage on 40 slices (untimed), then `nupd` timed updates."""
    from oracle import stream as ost
    st = ost.str_init(Xh[..., :W2.t_init], cores0)
    t = W2.t_init
    t0 = time.perf_counter()
    for _ in range(nupd):
        ost.str_update(st, Xh[..., t:t + W2.t_new], sweeps=W2.sweeps)
        t += W2.t_new
    return time.perf_counter() - t0


def cpu_threads():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


def cpu_baseline(X, cores0, nupd=2):
    Xh = X[..., :W2.t_init + nupd * W2.t_new].double().cpu().numpy()
    secs = oracle_sample(Xh, cores0, nupd)
    E = int(np.prod(W2.dims)) * W2.t_new
    return {"value": nupd * E / secs, "unit": "entries/s", "cores": cpu_threads(), "kind": "oracle",
            "sample": f"{nupd} STR updates of 10 slices (5 sweeps) of the order4 workload, FP64 numpy oracle",
            "seconds": secs}


def main_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    # inputs: same recipe on the host (oracle builds TR(G) itself)
    from oracle import stream as ost
    from oracle import tr as otr
    nsl = a.warmup + a.steps
    G = synth.gaussian_cores(tuple(W2.dims) + (W2.T,), W2.ranks, W2.seed)
    tmax = W2.t_init + nsl * W2.t_new
    Gt = G[:-1] + [G[-1][:, :tmax, :]]
    Xt = otr.tr_full(Gt)
    full = synth.gaussian_tensor(tuple(W2.dims) + (W2.T,), W2.seed + 100)[..., :tmax]
    X = Xt + W2.noise * np.linalg.norm(Xt) * full / np.linalg.norm(full)
    rng = np.random.default_rng(W2.seed + 200)
    init = [g + 0.3 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :W2.t_init, :]
    st = ost.str_init(X[..., :W2.t_init], init)
    t = W2.t_init
    for _ in range(a.warmup):
        ost.str_update(st, X[..., t:t + W2.t_new], sweeps=W2.sweeps)
        t += W2.t_new
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        ost.str_update(st, X[..., t:t + W2.t_new], sweeps=W2.sweeps)
        times.append(time.perf_counter() - t0)
        t += W2.t_new
    E = int(np.prod(W2.dims)) * W2.t_new
    value = a.steps * E / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(times) / a.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD_DESC, "entries_per_update": E},
           "cpu_baseline": {"value": value, "unit": "entries/s", "kind": "oracle", "cores": cpu_threads(),
                            "sample": "each step = one STR update of 10 slices (5 sweeps) by the FP64 oracle"},
           "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    args = args_parse()
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)
