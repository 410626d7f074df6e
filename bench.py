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
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Compton pair-scatters/s, plain vs MLP on 1 GB300 at stated error; p50/p99 lat"
UNIT = "pairs/s"
L2_NOTE = "inputs larger than L2 (particle state ~1.3 GB resident, 129 MB L2)"
# DRAM bytes (read + write) per unit from one ncu capture of the kernel as it
# is now, scaled to a launch by its units; the profile file gives the command.
# A kernel changed since its capture must be taken out of this table.
MEASURED_TRAFFIC = {
    "k_sort_gather": ((134.677504e6 + 111.480576e6) / 8372876, "particle",
                      "profiles/k_sort_gather_in_place_256x256.md"),
    "k_count": (34.025472e6 / 8372876, "particle", "profiles/k_count_256x256.md"),
    "k_pair_prob": ((97.137152e6 + 4.566784e6) / 4186438, "pair", "profiles/k_pair_prob_256x256.md"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--ppc", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--train-steps", type=int, default=8000)
    ap.add_argument("--train-balanced", action="store_true")
    ap.add_argument("--train-precision", default="bf16", choices=["bf16", "fp32"],
                    help="training arithmetic of the surrogate: tcgen05 BF16 (default) or FP32 CUDA cores")
    ap.add_argument("--workload", default="c2", choices=["c2", "c5", "ic"],
                    help="c2: the 2D 512x512 step (default); c5: the 3D power-law precision sweep; "
                         "ic: the inverse-Compton benchmark with a transfer-learned surrogate")
    ap.add_argument("--c5-side", type=int, default=256)
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
        # the raw samples: $COMPTON_CLOCKS_DIR if set, else the temporary directory
        d = os.environ.get("COMPTON_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

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


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: its own sub-grid
    (seed offset by the worker index), one oracle step, its own timing."""
    nx_s, ny_s, ppc, seed = job
    r, npairs, dt, _ = cpu_oracle_rate(nx_s, ny_s, ppc, seed)
    return npairs, dt


def cpu_oracle_rate_all_cores(nx_s: int = 128, ny_s: int = 128, ppc: int = 64):
    """Pairs/s of the oracle run as one process per host core, each on its
    own sub-grid of the same distributions (cells are independent, so this
    is the oracle's parallel form); the processes are spawned, not forked."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(n) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(nx_s, ny_s, ppc, 2 + 100 * i) for i in range(n)])
        wall = time.perf_counter() - t0
    npairs = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return {"value": npairs / slowest, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes, each one step of its own {nx_s}x{ny_s}-cell sub-grid of the same workload "
                      f"({npairs} pairs in all); value = all pairs / the slowest process's oracle time",
            "wall_s_including_process_start": wall}


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
            "mode": "plain", "l2": L2_NOTE, "parallelism": "cells sharded per rank (independent)",
            "input_order": "positions fixed: each step bins the previous step's cell-ordered output "
                           "(the first step and kernel_ms.bin_pairs_shuffled_input bin shuffled input)"}


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
    # weak scaling: rank r owns slab r of a grid of world * nx * ny cells
    # (shard_cells), nx x ny cells drawn from the slab's own seed 2 + r; the
    # slabs exchange nothing inside a step
    from paper_2206_02937_gb300.dist import shard_cells
    slab = shard_cells(world * args.nx * args.ny, rank, world)
    w = wl.c2(args.nx, args.ny, args.ppc, seed=2 + rank)
    assert w.n_cells == slab[1] - slab[0]
    dev = torch.device("cuda", local_rank)

    def species(d):
        return cg.Species(torch.from_numpy(d["ux"]).to(dev), torch.from_numpy(d["uy"]).to(dev),
                          torch.from_numpy(d["uz"]).to(dev), torch.from_numpy(d["cell"]).to(dev),
                          torch.from_numpy(d["id"].view(np.int32)).to(dev))

    A = [species(w.e), species(w.g)]
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    nmax = max(w.n_e, w.n_g)
    ctx = cg.compton_init(w.n_cells, nmax, w.w_over_v, w.dt, w.seed, device=local_rank,
                          max_train_batch=8192)
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

    from paper_2206_02937_gb300.dist import reduce_timing
    total_ms, pairs_all = reduce_timing(total_ms, pairs, dev)
    value = pairs_all / (total_ms * 1e-3)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sc_avg = sum(sc_ms) / len(sc_ms)
    bin_avg = sum(bin_ms) / len(bin_ms)

    # per-kernel device times: the same steps once more with the library's
    # event timing on (kept out of the headline region above).  The library
    # keeps the last 64 launches of each kernel slot and the scan slot
    # launches three kernels per step, so 20 steps keep every launch.
    kt_steps = min(args.steps, 20)
    cg.compton_kernel_timing(ctx, True)
    for i in range(kt_steps):
        one_step(step, bufs[step % 2], bufs[(step + 1) % 2])
        step += 1
    torch.cuda.synchronize()
    kt = cg.compton_kernel_times(ctx)
    cg.compton_kernel_timing(ctx, False)
    n_part = w.n_e + w.n_g
    acc_per_step = stats["scatters"] / args.steps
    # algorithmic bytes per launch (input already in cell order)
    algo_bytes = {
        "k_count": 4.0 * n_part,                       # cell indices read
        "k_scan": 48.0 * w.n_cells,                    # counts in, offsets + CellInfo out
        "k_place": 0.0,                                # returns at once on ordered input
        "k_sort_gather": 36.0 * n_part,                # id + momentum read, sorted copy written
        # both momenta of every pair (charged as if read; only the candidates
        # below the probability bound read theirs), the 48-byte accepted-list
        # entry written, the 16-byte CellInfo of every cell
        "k_pair_prob": 24.0 * pairs_per_step + 48.0 * acc_per_step + 16.0 * w.n_cells,
        "k_collide": 72.0 * acc_per_step,              # 48-byte list entry read, both momenta written
    }
    kernels = {}
    for name, v in kt.items():
        if v["launches"] == 0 or name not in algo_bytes:
            continue
        avg = v["ms"] / v["launches"]
        gbs = algo_bytes[name] / (avg * 1e-3) / 1e9
        kernels[name] = {"avg_launch_ms": avg, "launches_per_step": v["launches"] / kt_steps,
                         "algorithmic_bytes_per_launch": algo_bytes[name], "achieved_gbs": gbs,
                         "frac_of_hbm": gbs / hbm_peak}
    dom = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"] * kernels[k]["launches_per_step"])
    D = kernels[dom]
    traffic = None
    if dom in MEASURED_TRAFFIC:
        per_unit, unit_name, src = MEASURED_TRAFFIC[dom]
        traffic = per_unit * (n_part if unit_name == "particle" else pairs_per_step)
    roofline = {"kernel": dom, "bound": "hbm", "achieved": D["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": D["frac_of_hbm"], "traffic": traffic,
                "traffic_source": MEASURED_TRAFFIC[dom][2] if dom in MEASURED_TRAFFIC else None,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": D["algorithmic_bytes_per_launch"],
                "avg_launch_ms": D["avg_launch_ms"],
                "note": "dominant kernel of the step by device time; durations from CUDA events the library "
                        "records on the launch stream around each kernel"}
    # whole binning and scattering calls (events around the C-ABI calls)
    # the two kernels of the call: k_pair_prob's bytes and k_collide's
    bytes_scatter = pairs_per_step * 24.0 + acc_per_step * (48.0 + 72.0) + w.n_cells * 16.0
    achieved_sc = bytes_scatter / (sc_avg * 1e-3) / 1e9
    # binning of input already in cell order (every step after the first: the
    # particles keep their cells): per particle 4 (count) + 4 + 12 (id and
    # momentum read by the sort) + 20 (sorted write) = 40 B, both species
    bytes_bin = (w.n_e + w.n_g) * 40.0 + w.n_cells * 64.0
    achieved_bin = bytes_bin / (bin_avg * 1e-3) / 1e9
    # No-Time-Counter collisions on the same binned particles (Sec. 3.1)
    for _ in range(args.warmup):
        pr = cg.compton_bin_pairs(ctx, bufs[step % 2][0], bufs[step % 2][1], bufs[(step + 1) % 2][0],
                                  bufs[(step + 1) % 2][1], step, stream)
        cg.compton_scatter_step_ntc(ctx, bufs[(step + 1) % 2][0], bufs[(step + 1) % 2][1], pr, step, stream)
        step += 1
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0.record(stream)
    for _ in range(args.steps):
        pr = cg.compton_bin_pairs(ctx, bufs[step % 2][0], bufs[step % 2][1], bufs[(step + 1) % 2][0],
                                  bufs[(step + 1) % 2][1], step, stream)
        cg.compton_scatter_step_ntc(ctx, bufs[(step + 1) % 2][0], bufs[(step + 1) % 2][1], pr, step, stream)
        step += 1
    n1.record(stream)
    torch.cuda.synchronize()
    ntc_ms = n0.elapsed_time(n1) / args.steps
    st_ntc = cg.compton_get_stats(ctx, reset=True)
    # both collision schemes from the same particles, pairing and draws: the
    # source buffer is left unchanged, each scheme bins it afresh
    X, Y = bufs[step % 2], bufs[(step + 1) % 2]
    same = {"ntc": 0, "pairing": 0}
    for rep in range(3):
        for scheme in ("ntc", "pairing"):
            pr = cg.compton_bin_pairs(ctx, X[0], X[1], Y[0], Y[1], 9000 + rep, stream)
            cg.compton_get_stats(ctx, reset=True)
            if scheme == "ntc":
                cg.compton_scatter_step_ntc(ctx, Y[0], Y[1], pr, 9000 + rep, stream)
            else:
                cg.compton_scatter_step(ctx, Y[0], Y[1], pr, cg.MODE_PLAIN, 9000 + rep, None, None, stream)
            same[scheme] += cg.compton_get_stats(ctx, reset=True)["scatters"]
    ntc = {"ms_per_step": ntc_ms, "candidates_per_step": st_ntc["pairs_tested"] / args.steps,
           "candidates_per_s": st_ntc["pairs_tested"] / args.steps / (ntc_ms * 1e-3),
           "collisions_per_step": st_ntc["scatters"] / args.steps,
           "collision_ratio_ntc_to_pairing_same_state": same["ntc"] / max(1, same["pairing"]),
           "note": "bin + NTC candidates per cell (each cell's candidates in order: cells of 32 or more a warp each, the others a lane each from a shared queue); the ratio "
                   "compares both schemes on the same binned particles over 3 draws (NTC uses the linear "
                   "probability, pairing 1 - exp(-a): expected about 1 + n dt <s v>/2)"}

    # binning of shuffled input: 4 (count) + 20 (placement read) + 20 (record
    # write) + 20 (record read) + 20 (sorted write) = 84 B per particle
    S = [species(w.e), species(w.g)]
    Cb = [cg.Species.empty_like(S[0]), cg.Species.empty_like(S[1])]
    for i in range(args.warmup):
        cg.compton_bin_pairs(ctx, S[0], S[1], Cb[0], Cb[1], step + i, stream)
    shuf_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for i in range(args.steps):
        shuf_ev[i][0].record(stream)
        cg.compton_bin_pairs(ctx, S[0], S[1], Cb[0], Cb[1], step + i, stream)
        shuf_ev[i][1].record(stream)
    torch.cuda.synchronize()
    bin_shuf_avg = sum(e[0].elapsed_time(e[1]) for e in shuf_ev) / args.steps
    bytes_bin_shuf = (w.n_e + w.n_g) * 84.0 + w.n_cells * 64.0
    achieved_bin_shuf = bytes_bin_shuf / (bin_shuf_avg * 1e-3) / 1e9
    del S, Cb

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, cg, torch, ctx, w, stream, dev)

    mlp = None
    if not args.no_mlp:
        mlp = run_mlp(args, cg, torch, ctx, w, stream, dev, bufs, step, peaks,
                      with_oracle=rank == 0 and not args.no_cpu_baseline)
        step += 2 * (args.warmup + args.steps) + 2

    serving = None
    if not args.no_serving and rank == 0:
        serving = run_serving(args, cg, torch, ctx, bufs[step % 2], dev)

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu_baseline:
        r, npairs, dt, sample = cpu_oracle_rate()
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        cpu_all = cpu_oracle_rate_all_cores()

    cg.compton_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 collision update)", "data": "synthetic",
            "config": workload_config(args),
            "pairs_per_step": pairs_per_step, "scatter_fraction": frac_scat,
            "kernel_ms": {"bin_pairs": bin_avg, "scatter_step": sc_avg, "bin_pairs_shuffled_input": bin_shuf_avg},
            "roofline": roofline,
            "kernels": kernels,
            "roofline_scatter_step": {"bound": "hbm", "achieved": achieved_sc, "peak": hbm_peak, "unit": "GB/s",
                                      "frac": achieved_sc / hbm_peak, "algorithmic_bytes_per_launch": bytes_scatter,
                                      "calls": "compton_scatter_step (k_pair_prob + k_collide)"},
            "roofline_bin": {"bound": "hbm", "achieved": achieved_bin, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_bin / hbm_peak, "algorithmic_bytes_per_launch": bytes_bin,
                             "input": "cell order of the previous step's output"},
            "roofline_bin_shuffled": {"bound": "hbm", "achieved": achieved_bin_shuf, "peak": hbm_peak,
                                      "unit": "GB/s", "frac": achieved_bin_shuf / hbm_peak,
                                      "algorithmic_bytes_per_launch": bytes_bin_shuf, "input": "shuffled"},
            "gpu_launches": 8 * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e,
            "mlp": mlp,
            "ntc": ntc,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def train_surrogate(cg, torch, ctx, dev, n_samples=10_000_000, steps=8000, batch=8192, lr=1e-2, balanced=False,
                    precision="bf16"):
    """Train the network on the GPU on analytic targets over the surrogate's
    range (gamma log-uniform on [1, 1e3], eps log-uniform on [1e-4, 1]):
    Adam with the learning rate decayed from lr to 0 on a cosine, MAE loss,
    Glorot-uniform weights (seed 0), 10M samples split 80/20 into training
    and held-out sets.  balanced=True weights the loss by the
    data-balancing weights (32 log bins of r on [1e-6, 1]); with the MAE
    loss that pulls the network towards the rare tiny targets and costs
    accuracy everywhere else, so it is off by default.  precision "bf16"
    runs every contraction of the training step on the tcgen05 tensor cores,
    "fp32" on the CUDA cores.  Not timed as part of the step; its own wall
    time is reported."""
    from paper_2206_02937_gb300 import workloads as wl
    rng = np.random.default_rng(0)
    theta = np.zeros(12993, dtype=np.float32)
    at = 0
    for o, i in [(64, 6), (64, 64), (64, 64), (64, 64), (1, 64)]:
        lim = np.sqrt(6.0 / (o + i))
        theta[at:at + o * i] = rng.uniform(-lim, lim, o * i)
        at += o * i + o
    cg.compton_mlp_set_params(ctx, theta)
    cg.compton_mlp_set_train_precision(ctx, cg.MODE_MLP_BF16 if precision == "bf16" else cg.MODE_MLP_FP32)
    u, k = wl.c3(n_samples, seed=30)
    ut, kt = torch.from_numpy(u).to(dev), torch.from_numpy(k).to(dev)
    r = torch.zeros(n_samples, device=dev)
    cg.compton_kn_ratio(ctx, ut, kt, r)
    wts = None
    if balanced:
        wts = torch.zeros(n_samples, device=dev)
        edges = (1e-6 * (1e6) ** (np.arange(33) / 32)).astype(np.float32)
        cg.compton_mlp_balance_weights(ctx, r, edges, wts)
    gen = torch.Generator(device=dev).manual_seed(0)
    n_train = n_samples * 4 // 5
    losses = []
    torch.cuda.synchronize()
    t0 = time.time()
    for it in range(steps):
        idx = torch.randint(0, n_train, (batch,), device=dev, generator=gen)
        lr_it = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        loss = cg.compton_mlp_train_step(ctx, ut[:, idx].contiguous(), kt[:, idx].contiguous(),
                                         r[idx].contiguous(), None if wts is None else wts[idx].contiguous(),
                                         lr_it, want_loss=(it % 500 == 0 or it == steps - 1))
        if loss is not None:
            losses.append(loss)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    cg.compton_mlp_calibrate(ctx, ut[:, :65536].contiguous(), kt[:, :65536].contiguous())
    # held-out 20 %: error of r in FP32 and BF16 inference
    uh, kh, rh = ut[:, n_train:].contiguous(), kt[:, n_train:].contiguous(), r[n_train:]
    held = {}
    for md, name in ((cg.MODE_MLP_FP32, "fp32"), (cg.MODE_MLP_BF16, "bf16")):
        o = torch.empty_like(rh)
        cg.compton_mlp_infer(ctx, uh, kh, md, o)
        err = (o.double() - rh.double()).abs()
        big = rh > 1e-3
        held[name] = {"mae_r": float(err.mean()),
                      "mean_rel_r_above_1e-3": float((err[big] / rh[big].double()).mean()),
                      "max_rel_r_above_1e-3": float((err[big] / rh[big].double()).max())}
    torch.cuda.synchronize()
    return {"precision": precision, "steps": steps, "batch": batch, "lr": f"{lr} cosine-decayed to 0",
            "samples": n_samples,
            "split": "80 % training / 20 % held out",
            "loss": "MAE" + (" weighted by 32 log bins of r" if balanced else ""),
            "loss_first": losses[0], "loss_last": losses[-1], "train_s": train_s, "held_out": held}


TRAIN_FLOPS_PER_SAMPLE = 2.0 * (6 * 64 + 3 * 64 * 64 + 64) * 2 + 2.0 * 3 * 64 * 64
# forward z = a W^T (25,472) + weight gradients delta^T a (25,472) + input
# gradients delta W of the three 64x64 layers (24,576) = 75,520 per sample


def train_throughput(cg, torch, dev, peaks, batch=1 << 20, reps=5):
    """One training step (forward, backward, Adam) on a large batch, both
    precisions, timed with CUDA events: algorithmic FLOPs per second of the
    whole train-step call against the bf16 tensor peak."""
    from paper_2206_02937_gb300 import workloads as wl
    out = {}
    u, k = wl.c3(batch, seed=31)
    ut, kt = torch.from_numpy(u).to(dev), torch.from_numpy(k).to(dev)
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, device=dev.index or 0, max_train_batch=batch)
    try:
        rng = np.random.default_rng(1)
        theta = (rng.uniform(-0.2, 0.2, 12993)).astype(np.float32)
        cg.compton_mlp_set_params(ctx, theta)
        r = torch.zeros(batch, device=dev)
        cg.compton_kn_ratio(ctx, ut, kt, r)
        peak = float(peaks.get("bf16_tflops", 1900.0))
        for prec, mode in (("bf16", cg.MODE_MLP_BF16), ("fp32", cg.MODE_MLP_FP32)):
            cg.compton_mlp_set_train_precision(ctx, mode)
            for _ in range(2):
                cg.compton_mlp_train_step(ctx, ut, kt, r, None, 1e-4, want_loss=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                cg.compton_mlp_train_step(ctx, ut, kt, r, None, 1e-4, want_loss=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tf = TRAIN_FLOPS_PER_SAMPLE * batch / (ms * 1e-3) / 1e12
            out[prec] = {"ms_per_step": ms, "samples_per_s": batch / (ms * 1e-3), "tflops": tf,
                         "frac_of_bf16_peak": tf / peak}
        assert cg.compton_check(ctx) == cg.COMPTON_OK
    finally:
        cg.compton_destroy(ctx)
    out["batch"] = batch
    out["flops_per_sample"] = TRAIN_FLOPS_PER_SAMPLE
    out["note"] = ("whole compton_mlp_train_step call (gradient kernels, Adam, repacking) on one batch; bf16 = "
                   "tcgen05 tensor cores with BF16 operands and FP32 accumulation, fp32 = CUDA cores; peak: "
                   "measured bf16 burst")
    return out


def train_pnet(cg, torch, ctx, dev, w_cell, p_max_cells, n_samples=1 << 20, steps=8000, batch=8192, lr=1e-2):
    """Train the paper's 9-12-9 network on the same analytic targets.  Its
    inputs also carry the weights (w/V of both species) and the cell's P_max;
    each Adam step takes the P_max of a random cell of the workload, so the
    network sees the spread of densities it meets in the step."""
    from paper_2206_02937_gb300 import workloads as wl
    rng = np.random.default_rng(2)
    theta = np.zeros(cg.PNET_PARAMS, dtype=np.float32)
    at = 0
    for o, i in [(9, 9), (12, 9), (9, 12), (1, 9)]:
        lim = np.sqrt(6.0 / (o + i))
        theta[at:at + o * i] = rng.uniform(-lim, lim, o * i)
        at += o * i + o
    cg.compton_pnet_set_params(ctx, theta)
    u, k = wl.c3(n_samples, seed=30)
    ut, kt = torch.from_numpy(u).to(dev), torch.from_numpy(k).to(dev)
    r = torch.zeros(n_samples, device=dev)
    cg.compton_kn_ratio(ctx, ut, kt, r)
    gen = torch.Generator(device=dev).manual_seed(2)
    pm = rng.choice(p_max_cells, steps)
    losses = []
    torch.cuda.synchronize()
    t0 = time.time()
    for it in range(steps):
        idx = torch.randint(0, n_samples, (batch,), device=dev, generator=gen)
        lr_it = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
        loss = cg.compton_pnet_train_step(ctx, ut[:, idx].contiguous(), kt[:, idx].contiguous(), r[idx].contiguous(),
                                          None, w_cell, w_cell, float(pm[it]), lr_it,
                                          want_loss=(it % 500 == 0 or it == steps - 1))
        if loss is not None:
            losses.append(loss)
    torch.cuda.synchronize()
    return {"steps": steps, "batch": batch, "lr": f"{lr} cosine-decayed to 0",
            "samples": n_samples,
            "loss": "MAE", "loss_first": losses[0], "loss_last": losses[-1], "train_s": time.time() - t0,
            "p_max": "per step, that of a random cell of the workload"}


def dev_int32(torch, ptr, n):
    """n int32 values at a raw device pointer, copied to the host."""
    import ctypes
    t = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    path = None
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                path = line.split()[-1]
                break
    rt = ctypes.CDLL(path or "libcudart.so.13")
    rc = rt.cudaMemcpy(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(ptr), ctypes.c_size_t(4 * n), 3)
    if rc != 0:
        raise RuntimeError(f"cudaMemcpy failed: {rc}")
    return t.cpu().numpy()


def run_mlp(args, cg, torch, ctx, w, stream, dev, bufs, step0, peaks, with_oracle=False):
    """The whole step with the surrogate probability (BF16 tensor cores), its
    network kernel alone, and its error against the analytic path on the same
    pairs and draws."""
    train = train_surrogate(cg, torch, ctx, dev, steps=args.train_steps, balanced=args.train_balanced,
                            precision=args.train_precision)
    train["throughput"] = train_throughput(cg, torch, dev, peaks)
    mode = cg.MODE_MLP_BF16
    step = step0

    def one(src, dst, st, md, prob=None):
        pairs = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], st, stream)
        cg.compton_scatter_step(ctx, dst[0], dst[1], pairs, md, st, prob, None, stream)
        return pairs

    # the plain and the surrogate step timed from the same particle state and
    # step numbers (so the same pair lists and draws), with the same events
    snap = [cg.Species(*(t.clone() for t in (sp.ux, sp.uy, sp.uz, sp.cell, sp.id))) for sp in bufs[step % 2]]

    def restore():
        for sp, sn in zip(bufs[step0 % 2], snap):
            for a_, b_ in ((sp.ux, sn.ux), (sp.uy, sn.uy), (sp.uz, sn.uz), (sp.cell, sn.cell), (sp.id, sn.id)):
                a_.copy_(b_)

    def timed(md):
        st_ = step0
        for _ in range(args.warmup):
            one(bufs[st_ % 2], bufs[(st_ + 1) % 2], st_, md)
            st_ += 1
        torch.cuda.synchronize()
        cg.compton_get_stats(ctx, reset=True)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            one(bufs[st_ % 2], bufs[(st_ + 1) % 2], st_, md)
            st_ += 1
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1), cg.compton_get_stats(ctx, reset=True), st_

    ms_plain_same, st_plain_same, _ = timed(cg.MODE_PLAIN)
    restore()
    ms, st, step = timed(mode)
    # network kernel alone on 16.8M samples (electron/photon arrays as pairs)
    src = bufs[step % 2]
    n = min(src[0].n, src[1].n)
    u = torch.stack([src[0].ux[:n], src[0].uy[:n], src[0].uz[:n]])
    k = torch.stack([src[1].ux[:n], src[1].uy[:n], src[1].uz[:n]])
    rr = torch.empty(n, device=dev)
    kern = {}
    for md, name in ((cg.MODE_MLP_BF16, "bf16"), (cg.MODE_MLP_FP8, "fp8"), (cg.MODE_MLP_FP32, "fp32")):
        cg.compton_mlp_infer(ctx, u, k, md, rr, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            cg.compton_mlp_infer(ctx, u, k, md, rr, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        kern[name] = e0.elapsed_time(e1) / 3
    flops = 2.0 * (6 * 64 + 3 * 64 * 64 + 64) * n
    peak_bf16 = float(peaks.get("bf16_tflops", 1900.0))
    achieved = flops / (kern["bf16"] * 1e-3) / 1e12
    # error against the analytic path: same input, same step and draws, on
    # the workload's initial particles (after many scattering steps the
    # photons drift above the network's training range and take the
    # analytic path, which would flatter the comparison)
    a_copy = [cg.Species(*[torch.from_numpy(d[c] if c != "id" else d[c].view(np.int32)).to(dev)
                           for c in ("ux", "uy", "uz", "cell", "id")]) for d in (w.e, w.g)]
    scratch = [cg.Species.empty_like(sp) for sp in a_copy]

    n_sub = 1 << 20  # pairs compared with the FP64 oracle
    sub = {}

    def scattered_spectrum(md, P_out, st=777, name=None):
        pairs = cg.compton_bin_pairs(ctx, a_copy[0], a_copy[1], scratch[0], scratch[1], st, stream)
        torch.cuda.synchronize()
        before_g = torch.stack([scratch[1].ux, scratch[1].uy, scratch[1].uz]).clone()
        if name is not None and "ig" not in sub:
            # the first n_sub pairs of the step: their particles and densities
            off_e = dev_int32(torch, pairs.off_e_dev, w.n_cells + 1).astype(np.int64)
            off_g = dev_int32(torch, pairs.off_g_dev, w.n_cells + 1).astype(np.int64)
            m = np.minimum(np.diff(off_e), np.diff(off_g))
            pair_off = np.concatenate([[0], np.cumsum(m)])
            ns = int(min(n_sub, pair_off[-1]))
            cell = np.searchsorted(pair_off, np.arange(ns), side="right") - 1
            j = np.arange(ns) - pair_off[cell]
            sub["ie"], sub["ig"] = off_e[cell] + j, off_g[cell] + j
            sub["dens"] = (np.maximum(np.diff(off_e), np.diff(off_g))[cell] * w.w_over_v).astype(np.float32)
            ie_t = torch.from_numpy(sub["ie"]).to(dev)
            ig_t = torch.from_numpy(sub["ig"]).to(dev)
            sub["u"] = torch.stack([scratch[0].ux[ie_t], scratch[0].uy[ie_t], scratch[0].uz[ie_t]]).cpu().numpy()
            sub["k"] = before_g[:, ig_t].cpu().numpy()
        cg.compton_scatter_step(ctx, scratch[0], scratch[1], pairs, md, st, P_out, None, stream)
        torch.cuda.synchronize()
        k_after = torch.stack([scratch[1].ux, scratch[1].uy, scratch[1].uz])
        hit = (k_after != before_g).any(dim=0)
        if name is not None:
            ig_t = torch.from_numpy(sub["ig"]).to(dev)
            ns = sub["ig"].shape[0]
            sub[name] = (P_out[:ns].double().cpu().numpy(), k_after[:, ig_t].double().cpu().numpy(),
                         hit[ig_t].cpu().numpy())
        eps = k_after[:, hit].norm(dim=0).double().clamp_min(1e-12)
        h = torch.histc(eps.log10(), bins=64, min=-5.0, max=1.0)
        return h / h.sum().clamp_min(1.0), int(hit.sum())

    P_pl = torch.empty(n, device=dev)
    cg.compton_get_stats(ctx, reset=True)
    h_pl, n_pl = scattered_spectrum(cg.MODE_PLAIN, P_pl, name="plain")
    np_pairs = int(cg.compton_get_stats(ctx, reset=True)["pairs_tested"])
    pl = P_pl[:np_pairs].double()
    err = {}
    for md, name in ((cg.MODE_MLP_BF16, "bf16"), (cg.MODE_MLP_FP8, "fp8"), (cg.MODE_MLP_FP32, "fp32")):
        P_ml = torch.empty(n, device=dev)
        cg.compton_get_stats(ctx, reset=True)
        h_ml, n_ml = scattered_spectrum(md, P_ml, name=name)
        fb_ml = cg.compton_get_stats(ctx, reset=True)["mlp_fallbacks"] / max(1, np_pairs)
        mlv = P_ml[:np_pairs].double()
        rel = ((mlv - pl).abs() / pl.clamp_min(1e-30))
        err[name] = {"mean_abs_P": float((mlv - pl).abs().mean()), "mean_rel_P": float(rel.mean()),
                     "median_rel_P": float(rel.median()), "p99_rel_P": float(rel[::4].float().quantile(0.99)),
                     "collision_rate_ratio": n_ml / max(1, n_pl), "fallback_fraction": fb_ml,
                     "spectrum_L1": float((h_ml - h_pl).abs().sum()),
                     "spectrum_note": "L1 distance of normalised 64-bin log10(eps) histograms of the scattered photons, "
                                      "surrogate vs plain run on the same pairs and draws, the workload's initial "
                                      "particles"}
    err["mean_P_plain"] = float(pl.mean())
    # every path against the FP64 oracle on the first 2^20 pairs of the same
    # step and draws (part of the cpu_baseline leg: the oracle runs on the host)
    vs_oracle = None
    if with_oracle:
        import oracle
        t_or = time.time()
        uo_o, ko_o, P_o, flag_o = oracle.pairs(sub["u"], sub["k"], sub["dens"], w.dt, w.seed, 777)
        t_or = time.time() - t_or
        hit_o = flag_o == 1

        def spec(kk, hh):
            e = np.linalg.norm(kk[:, hh], axis=0)
            h, _ = np.histogram(np.log10(np.maximum(e, 1e-12)), bins=64, range=(-5.0, 1.0))
            return h / max(1, h.sum())

        s_o = spec(ko_o, hit_o)
        vs_oracle = {"pairs": int(P_o.shape[0]), "oracle_seconds_one_core": t_or,
                     "oracle_collisions": int(hit_o.sum()),
                     "note": "the first 2^20 pairs of the workload's initial particles, same pair list, step and "
                             "Philox draws; the oracle is FP64 on the host; flips = decisions that differ from "
                             "the oracle's; spectrum = L1 of normalised 64-bin log10(eps) histograms of the "
                             "scattered photons"}
        for name in ("plain", "fp32", "bf16", "fp8"):
            Pg, kg, hg = sub[name]
            rel_o = np.abs(Pg - P_o) / np.maximum(P_o, 1e-30)
            vs_oracle[name] = {"mean_rel_P": float(rel_o.mean()), "median_rel_P": float(np.median(rel_o)),
                               "p99_rel_P": float(np.quantile(rel_o, 0.99)), "max_rel_P": float(rel_o.max()),
                               "decision_flips": int((hg != hit_o).sum()), "collisions": int(hg.sum()),
                               "spectrum_L1": float(np.abs(spec(kg, hg) - s_o).sum())}
    # sampling noise of the spectrum distance: two plain runs with other draws
    h_pl2, _ = scattered_spectrum(cg.MODE_PLAIN, torch.empty(n, device=dev), st=778)
    err["spectrum_L1_plain_vs_plain_other_draws"] = float((h_pl2 - h_pl).abs().sum())

    # ablation: the same network trained on invariant inputs (ln x, ln v)
    # instead of momenta; the momentum network is restored afterwards
    blob = cg.compton_mlp_save(ctx)
    cg.compton_mlp_set_features(ctx, cg.FEATURES_INVARIANTS)
    train_inv = train_surrogate(cg, torch, ctx, dev, steps=args.train_steps, balanced=args.train_balanced,
                                precision=args.train_precision)
    P_iv = torch.empty(n, device=dev)
    h_iv, n_iv = scattered_spectrum(mode, P_iv)
    iv = P_iv[:np_pairs].double()
    rel_iv = ((iv - pl).abs() / pl.clamp_min(1e-30))
    # timed like the momentum network: same state, steps and draws as the
    # plain steps above
    restore()
    ms_iv, st_iv, step = timed(mode)
    invariant = {"features": "ln(x)/8, ln(v)/8 from the FP32 invariants", "mode": "bf16",
                 "ms_per_step": ms_iv / args.steps, "gain_vs_plain": ms_plain_same / ms_iv,
                 "fallback_fraction": st_iv["mlp_fallbacks"] / max(1, st_iv["pairs_tested"]),
                 "mean_rel_P": float(rel_iv.mean()), "median_rel_P": float(rel_iv.median()),
                 "p99_rel_P": float(rel_iv[::4].float().quantile(0.99)),
                 "collision_rate_ratio": n_iv / max(1, n_pl),
                 "spectrum_L1": float((h_iv - h_pl).abs().sum()), "train": train_inv}
    cg.compton_mlp_load(ctx, blob)

    # the paper's own 9-12-9 ReLU network (FP32, CUDA cores)
    cnt = np.maximum(np.bincount(w.e["cell"], minlength=w.n_cells), np.bincount(w.g["cell"], minlength=w.n_cells))
    p_max_cells = 2.0 * w.dt * w.w_over_v * cnt[cnt > 0].astype(np.float64)
    train_pn = train_pnet(cg, torch, ctx, dev, w.w_over_v, p_max_cells, steps=4 * args.train_steps)
    P_pn = torch.empty(n, device=dev)
    cg.compton_get_stats(ctx, reset=True)
    h_pn, n_pn = scattered_spectrum(cg.MODE_PNET, P_pn)
    fb_pn = cg.compton_get_stats(ctx, reset=True)["mlp_fallbacks"] / max(1, np_pairs)
    pnv = P_pn[:np_pairs].double()
    rel_pn = ((pnv - pl).abs() / pl.clamp_min(1e-30))
    for _ in range(args.warmup):
        one(bufs[step % 2], bufs[(step + 1) % 2], step, cg.MODE_PNET)
        step += 1
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one(bufs[step % 2], bufs[(step + 1) % 2], step, cg.MODE_PNET)
        step += 1
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pn = e0.elapsed_time(e1)
    st_pn = cg.compton_get_stats(ctx, reset=True)
    pm_med = float(np.median(p_max_cells))
    cg.compton_pnet_infer(ctx, u, k, w.w_over_v, w.w_over_v, pm_med, rr, stream)
    e0.record(stream)
    for _ in range(3):
        cg.compton_pnet_infer(ctx, u, k, w.w_over_v, w.w_over_v, pm_med, rr, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    kern_pn = e0.elapsed_time(e1) / 3
    pnet = {"network": "9-12-9 ReLU, sigmoid output, 337 parameters, FP32 on the CUDA cores",
            "value": st_pn["pairs_tested"] / (ms_pn * 1e-3), "unit": UNIT, "ms_per_step": ms_pn / args.steps,
            "network_kernel_ms": kern_pn, "network_samples": n,
            "network_kernel_bytes_per_sample": 28,
            "mean_rel_P": float(rel_pn.mean()), "median_rel_P": float(rel_pn.median()),
            "p99_rel_P": float(rel_pn[::4].float().quantile(0.99)),
            "fallback_fraction": fb_pn,
            "fallback_fraction_timed_steps": st_pn["mlp_fallbacks"] / max(1, st_pn["pairs_tested"]),
            "collision_rate_ratio": n_pn / max(1, n_pl),
            "spectrum_L1": float((h_pn - h_pl).abs().sum()), "train": train_pn}
    return {"mode": "bf16", "metric": METRIC, "value": st["pairs_tested"] / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / args.steps, "fallback_fraction": st["mlp_fallbacks"] / max(1, st["pairs_tested"]),
            "gain_vs_plain": ms_plain_same / ms,
            "gain_vs_plain_note": "plain step time over surrogate step time, both timed over the same steps from "
                                  "the same particle state (same pair lists and draws), after the headline region "
                                  f"(start step {step0}); the surrogate's fallback fraction is fallback_fraction",
            "plain_ms_per_step_same_state": ms_plain_same / args.steps,
            "plain_collisions_same_state": st_plain_same["scatters"], "collisions": st["scatters"],
            "network_kernel_ms": kern, "network_samples": n,
            "roofline": {"kernel": "k_mlp_ta (bf16)", "bound": "tensor", "achieved": achieved, "peak": peak_bf16,
                         "unit": "TFLOP/s", "frac": achieved / peak_bf16,
                         "note": "algorithmic FLOPs 2(6*64+3*64*64+64) per sample; peak: measured bf16 burst"},
            "error_vs_plain": err, "error_vs_oracle": vs_oracle, "train": train, "invariant_features": invariant,
            "paper_network": pnet}


def serve_stream(cg, torch, ctx, dev, u_pool, k_pool, rate, n_req, seed):
    """Drive the serving engine with n_req requests arriving as a Poisson
    stream at `rate` per second, sizes log-uniform in [1e3, 1e7] pairs, each a
    slice of the device-resident particle pool, alternately plain and BF16
    surrogate.  Latency = completion observed by poll - scheduled arrival."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    sizes = np.floor(10 ** rng.uniform(3, 7, n_req)).astype(np.int64)
    n_pool = u_pool.shape[1]
    outs, pending, lat, pairs_done = {}, {}, [], 0
    t_start = time.perf_counter()
    i = 0
    while i < n_req or pending:
        now = time.perf_counter() - t_start
        while i < n_req and arrivals[i] <= now:
            n = int(sizes[i])
            off = int(rng.integers(0, n_pool - n))
            uo = torch.empty((3, n), device=dev)
            ko = torch.empty((3, n), device=dev)
            mode = cg.MODE_PLAIN if i % 2 == 0 else cg.MODE_MLP_BF16
            t = cg.compton_submit(ctx, u_pool[:, off:off + n], k_pool[:, off:off + n], uo, ko, 1.0, 5000 + i, 0, mode)
            pending[t] = (i, n)
            outs[t] = (uo, ko)
            i += 1
        for t in list(pending):
            r = cg.compton_poll(ctx, t)
            if r is not None:
                idx, n = pending.pop(t)
                done = time.perf_counter() - t_start
                lat.append(done - arrivals[idx])
                pairs_done += n
                outs.pop(t)
        time.sleep(0.0002)
    wall = time.perf_counter() - t_start
    lat_ms = np.array(lat) * 1e3
    return {"arrival_rate_per_s": rate, "requests": n_req, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(lat_ms.mean()),
            "pairs": int(pairs_done), "wall_s": wall, "pairs_per_s": pairs_done / wall,
            "offered_pairs_per_s": float(sizes.sum() / arrivals[-1])}


def run_serving(args, cg, torch, ctx, src, dev):
    """Continuous batching: requests arrive as a Poisson stream at 200/s with
    sizes log-uniform in [1e3, 1e7] pairs, each a slice of the device-resident
    sorted particle arrays, half plain and half BF16 surrogate, admitted under
    a 40 GB budget.  Then a saturation sweep: the arrival rate doubles (400
    requests per rate) until the engine no longer keeps up (served below 90 %
    of the offered pairs/s) or p99 exceeds ten times the 200/s p99; the knee
    is the highest rate that still kept up."""
    n_pool = min(src[0].n, src[1].n)
    u_pool = torch.stack([src[0].ux[:n_pool], src[0].uy[:n_pool], src[0].uz[:n_pool]])
    k_pool = torch.stack([src[1].ux[:n_pool], src[1].uy[:n_pool], src[1].uz[:n_pool]])
    budget = 40 << 30
    cg.compton_serve_start(ctx, budget, 1024)
    base = serve_stream(cg, torch, ctx, dev, u_pool, k_pool, 200.0, args.serve_requests, 4)
    sweep, knee = [], None
    if args.serve_requests >= 400:
        rate = 400.0
        while rate <= 51200.0:
            r = serve_stream(cg, torch, ctx, dev, u_pool, k_pool, rate, 400, 40 + len(sweep))
            r["kept_up"] = r["pairs_per_s"] >= 0.9 * r["offered_pairs_per_s"] and r["p99_ms"] <= 10.0 * base["p99_ms"]
            sweep.append(r)
            if not r["kept_up"]:
                break
            knee = r
            rate *= 2.0
    info = cg.compton_serve_info(ctx)
    cg.compton_serve_stop(ctx)
    out = {"requests": base["requests"], "arrival_rate_per_s": 200, "sizes": "log-uniform [1e3, 1e7] pairs",
           "modes": "50/50 plain / bf16 surrogate", "budget_gb": budget / 2**30,
           "peak_pool_gb": info["peak"] / 2**30}
    out.update({k: base[k] for k in ("p50_ms", "p99_ms", "mean_ms", "pairs", "wall_s", "pairs_per_s",
                                     "offered_pairs_per_s")})
    out["saturation"] = {
        "sweep": [{k: r[k] for k in ("arrival_rate_per_s", "offered_pairs_per_s", "pairs_per_s", "p50_ms", "p99_ms",
                                     "kept_up")} for r in sweep],
        "knee_rate_per_s": None if knee is None else knee["arrival_rate_per_s"],
        "knee_pairs_per_s": None if knee is None else knee["pairs_per_s"],
        "max_served_pairs_per_s": max([r["pairs_per_s"] for r in sweep], default=None),
        "rule": "rate doubles from 400/s (400 requests each) until served < 0.9 x offered pairs/s or "
                "p99 > 10 x the 200/s p99; knee = last rate that kept up; requests are driven by one host "
                "thread polling every 0.2 ms"}
    return out


def run_e2e(args, cg, torch, ctx, w, stream, dev):
    """Same metric through the public API with host buffers: every step copies
    the inputs from pinned host memory, runs bin + scatter, and reads the
    updated momenta back into pinned host memory.  The copies run on two copy
    streams (host to device, device to host) with two sets of device
    buffers, so the upload of step i + 1 and the download of step i - 1
    overlap the kernels of step i; events order each buffer's uses."""
    host_in = []
    for d in (w.e, w.g):
        host_in.append([torch.from_numpy(d[k] if k != "id" else d[k].view(np.int32)).pin_memory()
                        for k in ("ux", "uy", "uz", "cell", "id")])
    dev_in = [[cg.Species(*[torch.empty_like(t, device=dev) for t in h]) for h in host_in] for _ in range(2)]
    dev_out = [[cg.Species.empty_like(s) for s in dev_in[0]] for _ in range(2)]
    host_out = [[[torch.empty_like(h[i]).pin_memory() for i in range(3)] for h in host_in] for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for h in host_in for t in h)
    d2h = sum(t.numel() * t.element_size() for h in host_out[0] for t in h)
    n_steps = max(3, min(args.steps, 10))
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def ev():
        return torch.cuda.Event()

    def run(step0, n):
        uploaded = [None, None]
        computed = [None, None]
        downloaded = [None, None]
        for i in range(n):
            b = i % 2
            with torch.cuda.stream(up):
                if computed[b] is not None:
                    up.wait_event(computed[b])  # step i - 2 is done with these inputs
                for s, h in zip(dev_in[b], host_in):
                    for t, src in zip((s.ux, s.uy, s.uz, s.cell, s.id), h):
                        t.copy_(src, non_blocking=True)
                uploaded[b] = ev()
                uploaded[b].record(up)
            stream.wait_event(uploaded[b])
            if downloaded[b] is not None:
                stream.wait_event(downloaded[b])  # step i - 2's results are read out
            pairs = cg.compton_bin_pairs(ctx, dev_in[b][0], dev_in[b][1], dev_out[b][0], dev_out[b][1],
                                         step0 + i, stream)
            cg.compton_scatter_step(ctx, dev_out[b][0], dev_out[b][1], pairs, cg.MODE_PLAIN, step0 + i,
                                    None, None, stream)
            computed[b] = ev()
            computed[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(computed[b])
                for s, h in zip(dev_out[b], host_out[b]):
                    for t, dst in zip((s.ux, s.uy, s.uz), h):
                        dst.copy_(t, non_blocking=True)
                downloaded[b] = ev()
                downloaded[b].record(down)
        return downloaded

    run(1000, 3)
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(up)
    done = run(2000, n_steps)
    for e in done:
        if e is not None:
            stream.wait_event(e)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    pairs = cg.compton_get_stats(ctx, reset=True)["pairs_tested"]

    # the host link's own bound: the same copies of every step, both
    # directions at once, without the kernels
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c0.record(stream)
    up.wait_stream(stream)
    down.wait_stream(stream)
    for i in range(n_steps):
        b = i % 2
        with torch.cuda.stream(up):
            for s, h in zip(dev_in[b], host_in):
                for t, src in zip((s.ux, s.uy, s.uz, s.cell, s.id), h):
                    t.copy_(src, non_blocking=True)
        with torch.cuda.stream(down):
            for s, h in zip(dev_out[b], host_out[b]):
                for t, dst in zip((s.ux, s.uy, s.uz), h):
                    dst.copy_(t, non_blocking=True)
    stream.wait_stream(up)
    stream.wait_stream(down)
    c1.record(stream)
    torch.cuda.synchronize()
    copy_ms = c0.elapsed_time(c1) / n_steps
    return {"value": pairs / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": n_steps, "ms_per_step": ms / n_steps,
            "copies_only_ms_per_step": copy_ms, "link_GBps": (h2d + d2h) / (copy_ms * 1e6),
            "link_bound_frac": copy_ms / (ms / n_steps),
            "note": "uploads, kernels and downloads of consecutive steps overlap on three streams; "
                    "copies_only_ms_per_step times the same copies without the kernels"}


# ---------------------------------------------------------------------------
# 3D precision sweep: power-law electrons on a photon beam
# ---------------------------------------------------------------------------
def log_spectrum(torch, k_after, hit, lo=-5.0, hi=5.0, bins=64):
    eps = k_after[:, hit].norm(dim=0).double().clamp_min(1e-30)
    h = torch.histc(eps.log10(), bins=bins, min=lo, max=hi)
    return h / h.sum().clamp_min(1.0)


def oracle_subsample(u, k, dens, dt, seed, step):
    """The cpu_baseline leg of the sweep: the FP64 oracle on a pre-paired
    subsample (pair i uses counter i, as the GPU's pair list does), timed on
    one host core.  Returns its timing and the photon momenta it produced."""
    import oracle
    t0 = time.time()
    uo, ko, P, flag = oracle.pairs(u, k, dens, dt, seed, step)
    return time.time() - t0, ko, flag


def run_c5(args, rank: int, world: int, local_rank: int):
    import torch
    import paper_2206_02937_gb300 as cg
    from paper_2206_02937_gb300 import workloads as wl

    cg.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    t_gen = time.time()
    w = wl.c5(args.c5_side, 16, seed=5 + rank)
    t_gen = time.time() - t_gen

    def species(d):
        return cg.Species(torch.from_numpy(d["ux"]).to(dev), torch.from_numpy(d["uy"]).to(dev),
                          torch.from_numpy(d["uz"]).to(dev), torch.from_numpy(d["cell"]).to(dev),
                          torch.from_numpy(d["id"].view(np.int32)).to(dev))

    A = [species(w.e), species(w.g)]
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    n = max(w.n_e, w.n_g)
    del w.e, w.g
    ctx = cg.compton_init(w.n_cells, n, w.w_over_v, w.dt, w.seed, device=local_rank, max_train_batch=8192)
    stream = torch.cuda.current_stream(dev)
    bufs = [A, B]
    step = 0

    def one(src, dst, st, md):
        pairs = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], st, stream)
        cg.compton_scatter_step(ctx, dst[0], dst[1], pairs, md, st, None, None, stream)

    for _ in range(args.warmup):
        one(bufs[step % 2], bufs[(step + 1) % 2], step, cg.MODE_PLAIN)
        step += 1
    torch.cuda.synchronize()
    cg.compton_get_stats(ctx, reset=True)
    if dist is not None:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            one(bufs[step % 2], bufs[(step + 1) % 2], step, cg.MODE_PLAIN)
            step += 1
        t1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    stats = cg.compton_get_stats(ctx, reset=True)
    from paper_2206_02937_gb300.dist import reduce_timing
    total_ms, pairs_all = reduce_timing(total_ms, stats["pairs_tested"], dev)
    value = pairs_all / (total_ms * 1e-3)

    train = train_surrogate(cg, torch, ctx, dev, steps=args.train_steps, balanced=args.train_balanced,
                            precision=args.train_precision)

    # the sweep: every mode takes the same state, pairing and draws
    X, Y = bufs[step % 2], bufs[(step + 1) % 2]
    st = step
    n_sub = min(1 << 20, n)
    sweep, spectra_sub, hits = {}, {}, {}
    for md, name in ((cg.MODE_PLAIN, "plain"), (cg.MODE_MLP_FP32, "fp32"), (cg.MODE_MLP_BF16, "bf16"),
                     (cg.MODE_MLP_FP8, "fp8")):
        ms = []
        for rep in range(3):
            pairs = cg.compton_bin_pairs(ctx, X[0], X[1], Y[0], Y[1], st, stream)
            torch.cuda.synchronize()
            k_before = torch.stack([Y[1].ux, Y[1].uy, Y[1].uz]).clone()
            if name == "plain" and rep == 0:
                sub_u = torch.stack([Y[0].ux[:n_sub], Y[0].uy[:n_sub], Y[0].uz[:n_sub]]).cpu().numpy()
                sub_k = k_before[:, :n_sub].cpu().numpy()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cg.compton_get_stats(ctx, reset=True)
            e0.record(stream)
            cg.compton_scatter_step(ctx, Y[0], Y[1], pairs, md, st, None, None, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        stt = cg.compton_get_stats(ctx, reset=True)
        k_after = torch.stack([Y[1].ux, Y[1].uy, Y[1].uz])
        hit = (k_after != k_before).any(dim=0)
        spec = log_spectrum(torch, k_after, hit)
        hits[name] = int(hit.sum())
        spectra_sub[name] = (k_after[:, :n_sub].cpu().numpy(), hit[:n_sub].cpu().numpy())
        sweep[name] = {"scatter_step_ms": statistics.median(ms), "pairs": stt["pairs_tested"],
                       "scatters": stt["scatters"], "fallbacks": stt["mlp_fallbacks"], "spectrum": spec}
        del k_before, k_after, hit
    for name in sweep:
        sweep[name]["spectrum_L1_vs_plain"] = float((sweep[name]["spectrum"] - sweep["plain"]["spectrum"]).abs().sum())
        sweep[name]["collision_rate_ratio"] = hits[name] / max(1, hits["plain"])
    for name in sweep:
        del sweep[name]["spectrum"]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the first 2^20 pairs of the same step (all cells hold 16
        # of each species, so pair p is particle p of both sorted species)
        dens = np.full(n_sub, 16 * w.w_over_v, dtype=np.float32)
        dt_cpu, ko, oflag = oracle_subsample(sub_u, sub_k, dens, w.dt, w.seed, st)
        cpu = {"value": n_sub / dt_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {n_sub} pairs of one step of the same workload"}
        o_hit = oflag == 1
        o_k = torch.from_numpy(ko)
        o_spec = log_spectrum(torch, o_k, torch.from_numpy(o_hit))
        for name, (kg, hg) in spectra_sub.items():
            g_spec = log_spectrum(torch, torch.from_numpy(kg.astype(np.float64)), torch.from_numpy(hg))
            sweep[name]["spectrum_L1_vs_oracle_subsample"] = float((g_spec - o_spec).abs().sum())
            sweep[name]["collisions_subsample"] = int(hg.sum())
        sweep["oracle_subsample_collisions"] = int(o_hit.sum())

    cg.compton_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (f64 above the gamma and gamma-eps thresholds)",
            "data": "synthetic",
            "config": {"workload": f"c5: 3D {args.c5_side}^3 cells x 16 per species, electrons dN/dgamma ~ gamma^-2 "
                                   f"on [1, 1e4], photon beam 1e-2 along +x, dt=0.05, density 1, seed 5",
                       "mode": "plain (headline); sweep of the surrogate in FP32/BF16/FP8",
                       "l2": "inputs larger than L2", "generate_s": t_gen},
            "pairs_per_step": stats["pairs_tested"] / args.steps,
            "clocks": clk.summary(), "cpu_baseline": cpu, "gpu_launches": 8 * args.steps,
            "precision_sweep": sweep, "train": train,
            "spectrum_note": "L1 distance of normalised 64-bin log10(eps) histograms (eps in [1e-5, 1e5]) of the "
                             "photons that scattered; vs plain over all pairs, vs the FP64 oracle over the subsample",
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Inverse-Compton benchmark (Sec. 3.3) with a transfer-learned surrogate
# ---------------------------------------------------------------------------
IC_FS = (1.0, 5.0, 1e-2, 9.3)          # feature scales for momenta up to ~100
IC_RANGE = (100.01, 1e-4, 100.0)       # gamma_max, eps_min, eps_max of the training data


def train_tl(cg, torch, ctx, dev, stages=(25.0, 50.0, 100.0), n_set=1 << 19, steps=(6000, 3000, 3000),
             lr=(3e-3, 1e-3, 1e-3), batch=8192):
    """Three-stage transfer learning (Sec. 3.2): stage s trains on the union of
    the waterbag data sets of radius up to p0_s, starting from the weights of
    the previous stage, with the learning rate decayed on a cosine within each
    stage.  Returns the network saved after each stage."""
    from paper_2206_02937_gb300 import workloads as wl
    rng = np.random.default_rng(0)
    theta = np.zeros(12993, dtype=np.float32)
    at = 0
    for o, i in [(64, 6), (64, 64), (64, 64), (64, 64), (1, 64)]:
        lim = np.sqrt(6.0 / (o + i))
        theta[at:at + o * i] = rng.uniform(-lim, lim, o * i)
        at += o * i + o
    cg.compton_mlp_set_params(ctx, theta, np.array(IC_FS, dtype=np.float32))
    cg.compton_mlp_set_range(ctx, *IC_RANGE)
    us, ks, blobs, info = [], [], [], []
    gen = torch.Generator(device=dev).manual_seed(0)
    for s_i, p0 in enumerate(stages):
        u, k = wl.waterbag_pairs(n_set, p0, seed=25 + s_i)
        us.append(torch.from_numpy(u).to(dev))
        ks.append(torch.from_numpy(k).to(dev))
        ut, kt = torch.cat(us, dim=1), torch.cat(ks, dim=1)
        n = ut.shape[1]
        r = torch.zeros(n, device=dev)
        cg.compton_kn_ratio(ctx, ut, kt, r)
        if s_i == 0:
            # output bias at the logit of the median target: the targets of
            # these sets lie near 1e-3, and from sigmoid(0) Adam drives the
            # output into the flat tail of the sigmoid before it learns
            rm = float(r.median())
            theta[-1] = np.log(rm / (1.0 - rm))
            cg.compton_mlp_set_params(ctx, theta, np.array(IC_FS, dtype=np.float32))
            cg.compton_mlp_set_range(ctx, *IC_RANGE)
        first = last = None
        for it in range(steps[s_i]):
            idx = torch.randint(0, n, (batch,), device=dev, generator=gen)
            lr_it = lr[s_i] * 0.5 * (1.0 + np.cos(np.pi * it / steps[s_i]))
            loss = cg.compton_mlp_train_step(ctx, ut[:, idx].contiguous(), kt[:, idx].contiguous(),
                                             r[idx].contiguous(), None, lr_it,
                                             want_loss=(it == 0 or it == steps[s_i] - 1))
            if loss is not None:
                first = loss if first is None else first
                last = loss
        cg.compton_mlp_calibrate(ctx, ut[:, :65536].contiguous(), kt[:, :65536].contiguous())
        torch.cuda.synchronize()
        blobs.append(cg.compton_mlp_save(ctx))
        info.append({"p0": p0, "samples": n, "steps": steps[s_i], "lr": lr[s_i], "loss_first": first,
                     "loss_last": last})
    return blobs, info


def train_tl_pnet(cg, torch, ctx, dev, w_cell, p_max, stages=(25.0, 50.0, 100.0), n_set=1 << 19,
                  steps=(20000, 8000, 8000), lr=(3e-3, 1e-3, 1e-3), batch=8192, seed=1):
    """The same three transfer-learning stages for the paper's own 9-12-9
    network, whose inputs also carry the macro-particle weights and the
    cell's P_max (here those of the inverse-Compton cells).  Returns the
    parameters after each stage.  seed sets the initial weights and the
    minibatch draws."""
    from paper_2206_02937_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    theta = np.zeros(cg.PNET_PARAMS, dtype=np.float32)
    at = 0
    for o, i in [(9, 9), (12, 9), (9, 12), (1, 9)]:
        lim = np.sqrt(6.0 / (o + i))
        theta[at:at + o * i] = rng.uniform(-lim, lim, o * i)
        at += o * i + o
    g_max, e_min, e_max = IC_RANGE
    cg.compton_pnet_set_params(ctx, theta, np.array(IC_FS, dtype=np.float32), g_max, e_min, e_max)
    us, ks, thetas, info = [], [], [], []
    gen = torch.Generator(device=dev).manual_seed(seed)
    for s_i, p0 in enumerate(stages):
        u, k = wl.waterbag_pairs(n_set, p0, seed=25 + s_i)
        us.append(torch.from_numpy(u).to(dev))
        ks.append(torch.from_numpy(k).to(dev))
        ut, kt = torch.cat(us, dim=1), torch.cat(ks, dim=1)
        n = ut.shape[1]
        r = torch.zeros(n, device=dev)
        cg.compton_kn_ratio(ctx, ut, kt, r)
        if s_i == 0:
            rm = float(r.median())
            theta[-1] = np.log(rm / (1.0 - rm))
            cg.compton_pnet_set_params(ctx, theta, np.array(IC_FS, dtype=np.float32), g_max, e_min, e_max)
        first = last = None
        t0 = time.time()
        for it in range(steps[s_i]):
            idx = torch.randint(0, n, (batch,), device=dev, generator=gen)
            lr_it = lr[s_i] * 0.5 * (1.0 + np.cos(np.pi * it / steps[s_i]))
            loss = cg.compton_pnet_train_step(ctx, ut[:, idx].contiguous(), kt[:, idx].contiguous(),
                                              r[idx].contiguous(), None, w_cell, w_cell, p_max, lr_it,
                                              want_loss=(it == 0 or it == steps[s_i] - 1))
            if loss is not None:
                first = loss if first is None else first
                last = loss
        torch.cuda.synchronize()
        thetas.append(cg.compton_pnet_get_params(ctx)[0])
        info.append({"p0": p0, "samples": n, "steps": steps[s_i], "lr": lr[s_i], "loss_first": first,
                     "loss_last": last, "stage_s": time.time() - t0})
    return thetas, info


def ic_simulation(cg, torch, ctx, w, steps, mode, dev, step0=0):
    """Run `steps` binning + scattering steps of workload w from its initial
    state; returns the photon momenta at the end and the collision count."""
    def sp(d):
        return cg.Species(torch.from_numpy(d["ux"]).to(dev), torch.from_numpy(d["uy"]).to(dev),
                          torch.from_numpy(d["uz"]).to(dev), torch.from_numpy(d["cell"]).to(dev),
                          torch.from_numpy(d["id"].view(np.int32)).to(dev))
    A = [sp(w.e), sp(w.g)]
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    bufs = [A, B]
    cg.compton_get_stats(ctx, reset=True)
    for i in range(steps):
        src, dst = bufs[i % 2], bufs[(i + 1) % 2]
        pr = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], step0 + i)
        cg.compton_scatter_step(ctx, dst[0], dst[1], pr, mode, step0 + i)
    torch.cuda.synchronize()
    out = bufs[steps % 2]
    return torch.stack([out[1].ux, out[1].uy, out[1].uz]).double(), cg.compton_get_stats(ctx, reset=True)


def ic_spectrum(torch, k, eps0, lo=-1.0, hi=2.5, bins=70):
    eps = k.norm(dim=0)
    hit = (eps - eps0).abs() > 1e-4 * eps0
    h = torch.histc(eps[hit].log10(), bins=bins, min=lo, max=hi)
    centers = 10.0 ** (lo + (torch.arange(bins, dtype=torch.float64) + 0.5) * (hi - lo) / bins)
    return h / h.sum().clamp_min(1.0), int(hit.sum()), float(centers[int(torch.argmax(h))])


def run_ic(args, rank: int, world: int, local_rank: int):
    import torch
    import paper_2206_02937_gb300 as cg
    from paper_2206_02937_gb300 import workloads as wl

    cg.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    probe = wl.inverse_compton(25.0)
    ctx = cg.compton_init(probe.n_cells, probe.n_e, probe.w_over_v, probe.dt, probe.seed, device=local_rank,
                          max_train_batch=8192)
    t_train = time.time()
    blobs, tl_info = train_tl(cg, torch, ctx, dev)
    t_train = time.time() - t_train
    ic_p_max = 2.0 * 1.0 * probe.dt  # density 1 in every cell
    # the paper's network, three training runs (initial weights and
    # minibatches from seeds 1, 2, 3; the gradient sums use float atomics, so
    # a run is not bit-reproducible either): its extrapolation to the
    # benchmark's photons varies from run to run, so all three are reported
    t_pnet = time.time()
    pnet_runs = [train_tl_pnet(cg, torch, ctx, dev, probe.w_over_v, ic_p_max, seed=sd) for sd in (1, 2, 3)]
    t_pnet = (time.time() - t_pnet) / len(pnet_runs)
    pnet_info = pnet_runs[0][1]

    def load_pnet(run):
        cg.compton_pnet_set_params(ctx, pnet_runs[run][0][-1], np.array(IC_FS, dtype=np.float32), *IC_RANGE)

    load_pnet(0)

    # head-on sweep (the paper's probability comparison): p_e along +x,
    # photons along -x with log-spaced energy
    sweep = {}
    eps = np.logspace(-3, 2, 501)
    for p_e in (5.0, 25.0, 50.0):
        u = np.zeros((3, eps.size), dtype=np.float32)
        u[0] = p_e
        k = np.zeros((3, eps.size), dtype=np.float32)
        k[0] = -eps
        ut, kt = torch.from_numpy(u).to(dev), torch.from_numpy(k).to(dev)
        ra, rn = torch.zeros(eps.size, device=dev), torch.zeros(eps.size, device=dev)
        cg.compton_kn_ratio(ctx, ut, kt, ra)
        cg.compton_mlp_infer(ctx, ut, kt, cg.MODE_MLP_BF16, rn)
        rel = ((rn.double() - ra.double()).abs() / ra.double()).cpu().numpy()
        rp = torch.zeros(eps.size, device=dev)
        cg.compton_pnet_infer(ctx, ut, kt, probe.w_over_v, probe.w_over_v, ic_p_max, rp)
        rel_p = ((rp.double() - ra.double()).abs() / ra.double()).cpu().numpy()
        sweep[f"p_e={p_e:g}"] = {"max_rel_r": float(rel.max()), "median_rel_r": float(np.median(rel)),
                                 "pnet_max_rel_r": float(rel_p.max()), "pnet_median_rel_r": float(np.median(rel_p)),
                                 "eps_range": [1e-3, 100.0]}

    # held-out pairs of the last stage's distribution: r error of each network
    uv, kv = wl.waterbag_pairs(1 << 18, 100.0, seed=99)
    uvt, kvt = torch.from_numpy(uv).to(dev), torch.from_numpy(kv).to(dev)
    rv = torch.zeros(uv.shape[1], device=dev)
    cg.compton_kn_ratio(ctx, uvt, kvt, rv)
    held_out = {}
    for name, fn in (("mlp_fp32", lambda o: cg.compton_mlp_infer(ctx, uvt, kvt, cg.MODE_MLP_FP32, o)),
                     ("mlp_bf16", lambda o: cg.compton_mlp_infer(ctx, uvt, kvt, cg.MODE_MLP_BF16, o)),
                     ("pnet", lambda o: cg.compton_pnet_infer(ctx, uvt, kvt, probe.w_over_v, probe.w_over_v,
                                                              ic_p_max, o))):
        o = torch.zeros_like(rv)
        fn(o)
        rel = ((o.double() - rv.double()).abs() / rv.double()).cpu().numpy()
        held_out[name] = {"mean_rel_r": float(rel.mean()), "median_rel_r": float(np.median(rel)),
                          "mean_ratio": float((o.double() / rv.double()).mean())}

    results = {}
    pairs_total, ms_total = 0, 0.0
    for p_e in (25.0, 50.0, 100.0):
        w = wl.inverse_compton(p_e)
        # steps for about 30 % of the electrons to collide: P ~ 2 n dt <r>
        u0 = np.stack([w.e[c] for c in ("ux", "uy", "uz")])
        k0 = np.stack([w.g[c] for c in ("ux", "uy", "uz")])
        rr = torch.zeros(w.n_e, device=dev)
        cg.compton_kn_ratio(ctx, torch.from_numpy(u0).to(dev), torch.from_numpy(k0).to(dev), rr)
        n_steps = int(np.ceil(0.3 / (2.0 * 1.0 * w.dt * float(rr.mean()))))
        t0 = time.time()
        k_pl, st_pl = ic_simulation(cg, torch, ctx, w, n_steps, cg.MODE_PLAIN, dev)
        ms_total += (time.time() - t0) * 1e3
        pairs_total += st_pl["pairs_tested"]
        k_pl2, _ = ic_simulation(cg, torch, ctx, w, n_steps, cg.MODE_PLAIN, dev, step0=100000)
        h_pl, n_pl, peak_pl = ic_spectrum(torch, k_pl, 2.5)
        h_pl2, _, _ = ic_spectrum(torch, k_pl2, 2.5)
        entry = {"steps": n_steps, "scattered_photons_plain": n_pl, "peak_eps_plain": peak_pl,
                 "spectrum_L1_plain_vs_plain_other_draws": float((h_pl2 - h_pl).abs().sum())}
        for si, blob in enumerate(blobs):
            if si < len(blobs) - 1 and p_e != 100.0:
                continue
            cg.compton_mlp_load(ctx, blob)
            k_nn, st_nn = ic_simulation(cg, torch, ctx, w, n_steps, cg.MODE_MLP_BF16, dev)
            h_nn, n_nn, peak_nn = ic_spectrum(torch, k_nn, 2.5)
            tag = f"tl_stage_{si + 1}"
            entry[tag] = {"scattered_photons": n_nn, "peak_eps": peak_nn,
                          "spectrum_L1_vs_plain": float((h_nn - h_pl).abs().sum()),
                          "fallbacks": st_nn["mlp_fallbacks"]}
        # the paper's network after the last stage (FP32, CUDA cores), each
        # training run
        runs = []
        for run in range(len(pnet_runs)):
            load_pnet(run)
            k_pn, st_pn = ic_simulation(cg, torch, ctx, w, n_steps, cg.MODE_PNET, dev)
            h_pn, n_pn, peak_pn = ic_spectrum(torch, k_pn, 2.5)
            runs.append({"scattered_photons": n_pn, "peak_eps": peak_pn,
                         "spectrum_L1_vs_plain": float((h_pn - h_pl).abs().sum()),
                         "fallbacks": st_pn["mlp_fallbacks"]})
        entry["pnet_tl_stage_3"] = {"training_runs": runs,
                                    "median_spectrum_L1_vs_plain":
                                        float(np.median([r_["spectrum_L1_vs_plain"] for r_ in runs]))}
        results[f"p_e={p_e:g}"] = entry
    cg.compton_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": pairs_total / (ms_total * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "inverse Compton: beams p_e = 25, 50, 100 along +x through an isotropic photon "
                                   "gas at eps = 2.5, 512 cells x 128 per species, density 1, dt 0.05; value = "
                                   "pairs/s of the plain runs including host launch overheads"},
            "inverse_compton": results, "head_on_sweep": sweep, "transfer_learning": tl_info, "train_s": t_train,
            "transfer_learning_pnet": pnet_info, "train_pnet_s_per_run": t_pnet,
            "held_out_waterbag_p0_100": held_out,
            "note": "spectra: normalised 70-bin log10(eps) histograms of the photons that scattered at least "
                    "once, after the run; tl_stage_k = the surrogate after k transfer-learning stages (BF16); "
                    "pnet_tl_stage_3 = the paper's 9-12-9 network after the three stages (FP32), three training "
                    "runs; the sweep and held-out figures of the paper's network are those of the first run",
        }
        print(json.dumps(line), flush=True)


def spawn_ranks(n: int) -> int:
    """`--gpus N` run without a launcher: start N ranks of this script with
    torch.distributed.run on this node (127.0.0.1, a free port) and return
    its exit status; rank 0 prints the line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args.gpus))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "c5":
        run_c5(args, rank, world, local_rank)
    elif args.workload == "ic":
        run_ic(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
