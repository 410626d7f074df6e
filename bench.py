#!/usr/bin/env python3
"""Benchmark of the Compton pair-scatter step on GB300.

A step is one pass of the whole hot path over one batch: binning and random
in-cell pairing of both species (compton_bin_pairs) followed by probability,
Bernoulli trial and collision of every pair (compton_scatter_step).  The
workload is the 2D 512 x 512-cell set with log-normal cell fill (64 per
species per cell on average, ~16.8M pairs per step), Maxwell-Juttner theta=1
electrons and Planck kT=1e-2 photons.  Particle state stays resident in HBM
and ping-pongs between two buffers (the sorted output of one step is the
input of the next); it is about 1.3 GB, far above the 129 MB L2.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Compton pair-scatters/s, plain vs MLP on 1 GB300 at stated error; p50/p99 lat"
UNIT = "pairs/s"
L2_NOTE = "inputs larger than L2 (particle state ~1.3 GB resident, 129 MB L2)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled while the timed region runs
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def cpu_oracle_rate(nx_s: int = 256, ny_s: int = 256, ppc: int = 64, seed: int = 2):
    """Pairs/s of the FP64 oracle (one thread) on a sub-grid of the same
    workload: the same distributions on nx_s x ny_s cells."""
    import oracle
    from paper_2206_02937_gb300 import workloads as wl
    w = wl.c2(nx_s, ny_s, ppc, seed)
    oracle.lib()
    t0 = time.perf_counter()
    o = oracle.step(w.n_cells, w.w_over_v, w.dt, w.seed, 0, w.e, w.g)
    dt = time.perf_counter() - t0
    sample = f"one step of a {nx_s}x{ny_s}-cell sub-grid of the same workload ({o['n_pairs']} pairs)"
    return o["n_pairs"] / dt, o["n_pairs"], dt, sample


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    rates = []
    for _ in range(args.warmup):
        cpu_oracle_rate(32, 32, args.ppc)
    t_all = []
    npairs_all = 0
    sample = ""
    for _ in range(args.steps):
        r, npairs, dt, sample = cpu_oracle_rate(96, 96, args.ppc)
        rates.append(r)
        t_all.append(dt)
        npairs_all += npairs
    value = npairs_all / sum(t_all)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(t_all) / len(t_all),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"c2: 2D {args.nx}x{args.ny} cells, log-normal (sigma 0.5) fill, {args.ppc} per species "
                        f"per cell on average, Maxwell-Juttner theta=1 electrons, Planck kT=1e-2 photons, "
                        f"plain analytic probability, dt=0.05, seed 2",
            "mode": "plain", "l2": L2_NOTE, "parallelism": "cells sharded per rank (independent)"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import paper_2206_02937_gb300 as cg
    from paper_2206_02937_gb300 import workloads as wl

    cg.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = wl.c2(args.nx, args.ny, args.ppc, seed=2 + rank)
    dev = torch.device("cuda", local_rank)

    def species(d):
        return cg.Species(torch.from_numpy(d["ux"]).to(dev), torch.from_numpy(d["uy"]).to(dev),
                          torch.from_numpy(d["uz"]).to(dev), torch.from_numpy(d["cell"]).to(dev),
                          torch.from_numpy(d["id"].view(np.int32)).to(dev))

    A = [species(w.e), species(w.g)]
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    nmax = max(w.n_e, w.n_g)
    ctx = cg.compton_init(w.n_cells, nmax, w.w_over_v, w.dt, w.seed, device=local_rank)
    stream = torch.cuda.current_stream(dev)

    def one_step(step, src, dst, ev=None):
        if ev is not None:
            ev[0].record(stream)
        pairs = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], step, stream)
        if ev is not None:
            ev[1].record(stream)
        cg.compton_scatter_step(ctx, dst[0], dst[1], pairs, cg.MODE_PLAIN, step, None, None, stream)
        if ev is not None:
            ev[2].record(stream)
        return pairs

    bufs = [A, B]
    step = 0
    for _ in range(args.warmup):
        one_step(step, bufs[step % 2], bufs[(step + 1) % 2])
        step += 1
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            one_step(step, bufs[step % 2], bufs[(step + 1) % 2], evs[i])
            step += 1
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    stats = cg.compton_get_stats(ctx, reset=True)
    bin_ms = [e[0].elapsed_time(e[1]) for e in evs]
    sc_ms = [e[1].elapsed_time(e[2]) for e in evs]
    pairs = stats["pairs_tested"]
    frac_scat = stats["scatters"] / max(1, pairs)
    pairs_per_step = pairs / args.steps

    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        p = torch.tensor([float(pairs)], device=dev, dtype=torch.float64)
        dist.all_reduce(p)
        pairs_all = float(p.item())
    else:
        pairs_all = float(pairs)
    value = pairs_all / (total_ms * 1e-3)

    # roofline of the scatter kernel (one launch per compton_scatter_step)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    bytes_scatter = pairs_per_step * (24.0 + 24.0 * frac_scat) + w.n_cells * 16.0
    sc_avg = sum(sc_ms) / len(sc_ms)
    achieved_sc = bytes_scatter / (sc_avg * 1e-3) / 1e9
    # binning: per particle 4 (count) + 8 (key+index read) + 8 (record write)
    # + 8 (record read) + 20 (gather) + 20 (write) = 68 B, both species
    bytes_bin = (w.n_e + w.n_g) * 68.0 + w.n_cells * 64.0
    bin_avg = sum(bin_ms) / len(bin_ms)
    achieved_bin = bytes_bin / (bin_avg * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, cg, torch, ctx, w, stream, dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, npairs, dt, sample = cpu_oracle_rate()
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}

    cg.compton_destroy(ctx)
    if rank == 0:
        dominant = "k_scatter" if sc_avg >= bin_avg else "bin_pairs (6 kernels)"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 collision update)", "data": "synthetic",
            "config": workload_config(args),
            "pairs_per_step": pairs_per_step, "scatter_fraction": frac_scat,
            "kernel_ms": {"bin_pairs": bin_avg, "scatter_step": sc_avg},
            "roofline": {"kernel": "k_scatter", "bound": "hbm", "achieved": achieved_sc, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved_sc / hbm_peak, "traffic": None,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bytes_scatter,
                         "note": f"dominant by time: {dominant}"},
            "roofline_bin": {"bound": "hbm", "achieved": achieved_bin, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_bin / hbm_peak, "algorithmic_bytes_per_launch": bytes_bin},
            "gpu_launches": 7 * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "e2e": e2e,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(args, cg, torch, ctx, w, stream, dev):
    """Same metric through the public API with host buffers: every step copies
    the inputs from pinned host memory, runs bin + scatter, and reads the
    updated momenta back into pinned host memory."""
    host_in = []
    for d in (w.e, w.g):
        host_in.append([torch.from_numpy(d[k] if k != "id" else d[k].view(np.int32)).pin_memory()
                        for k in ("ux", "uy", "uz", "cell", "id")])
    dev_in = [cg.Species(*[torch.empty_like(t, device=dev) for t in h]) for h in host_in]
    dev_out = [cg.Species.empty_like(s) for s in dev_in]
    host_out = [[torch.empty_like(h[i]).pin_memory() for i in range(3)] for h in host_in]
    h2d = sum(t.numel() * t.element_size() for h in host_in for t in h)
    d2h = sum(t.numel() * t.element_size() for h in host_out for t in h)
    n_steps = max(3, min(args.steps, 10))

    def step_e2e(step):
        for s, h in zip(dev_in, host_in):
            for t, src in zip((s.ux, s.uy, s.uz, s.cell, s.id), h):
                t.copy_(src, non_blocking=True)
        pairs = cg.compton_bin_pairs(ctx, dev_in[0], dev_in[1], dev_out[0], dev_out[1], step, stream)
        cg.compton_scatter_step(ctx, dev_out[0], dev_out[1], pairs, cg.MODE_PLAIN, step, None, None, stream)
        for s, h in zip(dev_out, host_out):
            for t, dst in zip((s.ux, s.uy, s.uz), h):
                dst.copy_(t, non_blocking=True)

    for i in range(2):
        step_e2e(1000 + i)
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(n_steps):
        step_e2e(2000 + i)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    pairs = cg.compton_get_stats(ctx, reset=True)["pairs_tested"]
    return {"value": pairs / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": n_steps, "ms_per_step": ms / n_steps}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
