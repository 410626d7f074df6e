"""The continuous-batching serving loop: a request's result is the same alone
and in a mix of uneven requests (bit for bit, and equal to the direct
compton_scatter_pairs call with the same seed), admission respects the memory
budget, and errors are reported."""
import time

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _pairs(torch, n, seed):
    u, k = wl.c3(n, seed=seed)
    return torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()


def _wait(cg, ctx, tickets, timeout=60.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = cg.compton_poll(ctx, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.001)
    return out


def _ctx(cg, max_particles=300000):
    ctx = cg.compton_init(1, max_particles, 1.0, 0.05, 1)
    cg.compton_mlp_set_params(ctx, omlp.init_params(3).astype(np.float32))
    return ctx


def test_alone_equals_mixed_equals_direct():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    ctx = _ctx(cg)
    try:
        cg.compton_serve_start(ctx, 1 << 30, 256)
        u0, k0 = _pairs(torch, 50000, 7)
        dens = torch.full((50000,), 30.0, device="cuda")
        results = {}
        for mode in (cg.MODE_PLAIN, cg.MODE_MLP_BF16):
            # direct call
            ud, kd = u0.clone(), k0.clone()
            cg.compton_scatter_pairs(ctx, ud, kd, dens, 99, 5, mode)
            # alone through the engine
            ua, ka = torch.empty_like(u0), torch.empty_like(k0)
            t = cg.compton_submit(ctx, u0, k0, ua, ka, dens, 99, 5, mode)
            ra = _wait(cg, ctx, [t])[t]
            # in a mix of uneven requests of both modes
            rng = np.random.default_rng(int(mode))
            others, tickets = [], []
            for i in range(24):
                n = int(10 ** rng.uniform(3, 5.3))
                ui, ki = _pairs(torch, n, 100 + i)
                uo, ko = torch.empty_like(ui), torch.empty_like(ki)
                others.append((ui, ki, uo, ko))
                m = cg.MODE_PLAIN if i % 2 else cg.MODE_MLP_BF16
                tickets.append(cg.compton_submit(ctx, ui, ki, uo, ko, 20.0, 1000 + i, 1, m))
                if i == 12:
                    ub, kb = torch.empty_like(u0), torch.empty_like(k0)
                    tickets.append(cg.compton_submit(ctx, u0, k0, ub, kb, dens, 99, 5, mode))
                    t_mix = tickets[-1]
            res = _wait(cg, ctx, tickets)
            torch.cuda.synchronize()
            assert torch.equal(ua, ud) and torch.equal(ka, kd)
            assert torch.equal(ub, ua) and torch.equal(kb, ka)
            assert res[t_mix]["scatters"] == ra["scatters"] > 100
            results[mode] = ra
        assert all(r["latency_s"] > 0 for r in results.values())
    finally:
        cg.compton_destroy(ctx)


def test_budget_admission_and_errors():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    ctx = cg.compton_init(1, 1000, 1.0, 0.05, 1)
    try:
        pool = 4 * 28 * 60000  # room for about four requests of 60k pairs
        cg.compton_serve_start(ctx, pool, 64)
        reqs, tickets = [], []
        for i in range(16):
            ui, ki = _pairs(torch, 60000, 200 + i)
            uo, ko = torch.empty_like(ui), torch.empty_like(ki)
            reqs.append((ui, ki, uo, ko))
            tickets.append(cg.compton_submit(ctx, ui, ki, uo, ko, 25.0, 7, i))
        res = _wait(cg, ctx, tickets)
        info = cg.compton_serve_info(ctx)
        assert info["peak"] <= pool and info["in_use"] == 0
        assert max(r["queue_s"] for r in res.values()) > 0  # some had to wait for budget
        # each equals the direct call
        for i, (ui, ki, uo, ko) in enumerate(reqs):
            ud, kd = ui.clone(), ki.clone()
            nd = torch.full((60000,), 25.0, device="cuda")
            cg.compton_scatter_pairs(ctx, ud, kd, nd, 7, i)
            torch.cuda.synchronize()
            assert torch.equal(uo, ud) and torch.equal(ko, kd)
        # a request that can never fit
        big_u, big_k = torch.zeros((3, 400000), device="cuda"), torch.zeros((3, 400000), device="cuda")
        with pytest.raises(cg.ComptonError) as e:
            cg.compton_submit(ctx, big_u, big_k, big_u, big_k, 1.0, 1)
        assert e.value.status == cg.COMPTON_ERANGE
        with pytest.raises(cg.ComptonError) as e:
            cg.compton_poll(ctx, 123456789)
        assert e.value.status == cg.COMPTON_EINVAL
        with pytest.raises(cg.ComptonError) as e:
            cg.compton_submit(ctx, big_u[:, :10], big_k[:, :10], big_u[:, :10], big_k[:, :10], 1.0, 1, 0,
                              cg.MODE_MLP_BF16)
        assert e.value.status == cg.COMPTON_ENOMODEL
    finally:
        cg.compton_destroy(ctx)
