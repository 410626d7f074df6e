"""Shared helpers of the GPU tests: move seeded inputs to the device, run the
library's step through the C ABI, and compare with the oracle."""
import numpy as np

import oracle


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def to_species(torch, d):
    import paper_2206_02937_gb300 as cg
    dev = "cuda"
    w = d.get("w")
    return cg.Species(torch.from_numpy(d["ux"]).to(dev), torch.from_numpy(d["uy"]).to(dev),
                      torch.from_numpy(d["uz"]).to(dev), torch.from_numpy(d["cell"]).to(dev),
                      torch.from_numpy(d["id"].view(np.int32)).to(dev),
                      None if w is None else torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(dev))


def species_np(s):
    out = dict(ux=s.ux.cpu().numpy(), uy=s.uy.cpu().numpy(), uz=s.uz.cpu().numpy(),
               cell=s.cell.cpu().numpy(), id=s.id.cpu().numpy().view(np.uint32))
    if s.w is not None:
        out["w"] = s.w.cpu().numpy()
    return out


def gpu_step(w, step=0, gamma64=1.0e3, want_prob=True, want_flag=None):
    """bin_pairs + scatter_step of workload w on cuda:0.  Returns host copies
    of the sorted species before and after the scatter, P, flags, offsets.
    want_flag defaults to want_prob; flags without P take the filtered path
    (only pairs below the probability bound are evaluated)."""
    if want_flag is None:
        want_flag = want_prob
    torch = torch_cuda()
    import paper_2206_02937_gb300 as cg
    cg.build()
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed,
                          gamma_fp64_threshold=gamma64)
    try:
        e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, step)
        torch.cuda.synchronize()
        before_e, before_g = species_np(e_out), species_np(g_out)
        mp = max(1, pairs.max_pairs)
        prob = torch.zeros(mp, dtype=torch.float32, device="cuda") if want_prob else None
        flag = torch.zeros(mp, dtype=torch.uint8, device="cuda") if want_flag else None
        cg.compton_scatter_step(ctx, e_out, g_out, pairs, cg.MODE_PLAIN, step, prob, flag)
        torch.cuda.synchronize()
        st = cg.compton_check(ctx)
        stats = cg.compton_get_stats(ctx, reset=True)
        n_pairs = int(stats["pairs_tested"])
        off_e = _dev_array(torch, pairs.off_e_dev, w.n_cells + 1)
        off_g = _dev_array(torch, pairs.off_g_dev, w.n_cells + 1)
        out = dict(before_e=before_e, before_g=before_g, after_e=species_np(e_out), after_g=species_np(g_out),
                   P=prob.cpu().numpy()[:n_pairs] if want_prob else None,
                   flag=flag.cpu().numpy()[:n_pairs] if want_flag else None,
                   off_e=off_e, off_g=off_g, n_pairs=n_pairs, stats=stats, check=st)
    finally:
        cg.compton_destroy(ctx)
    return out


def _cudart():
    """The CUDA runtime library torch has loaded (for raw-pointer copies)."""
    import ctypes
    path = None
    with open("/proc/self/maps") as f:
        for line in f:
            if "libcudart.so" in line:
                path = line.split()[-1]
                break
    return ctypes.CDLL(path or "libcudart.so.13")


def _dev_array(torch, ptr, n):
    """Copy n int32 values from a raw device pointer into a numpy array."""
    import ctypes
    t = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    rc = _cudart().cudaMemcpy(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(ptr), ctypes.c_size_t(4 * n), 3)
    assert rc == 0
    return t.cpu().numpy()


def u0_of_pairs(seed, step, n_pairs):
    """The Bernoulli uniform of every pair, from the oracle's Philox."""
    return np.array([oracle.bernoulli_u0(seed, step, p) for p in range(n_pairs)])


def energy_scale(u, k):
    """gamma + eps per pair from (3, n) arrays."""
    return np.sqrt(1.0 + (u.astype(np.float64) ** 2).sum(0)) + np.sqrt((k.astype(np.float64) ** 2).sum(0))
