"""Per-kernel event timing: every kernel slot of a binning + scattering step
records its launches, the times are positive and sum to no more than the
step measured around it."""
import pytest

from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import to_species, torch_cuda

pytestmark = pytest.mark.gpu


def test_kernel_times_cover_the_step():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = wl.c2(48, 48, 32, seed=3)
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        with pytest.raises(cg.ComptonError):
            cg.compton_kernel_times(ctx)  # never enabled
        e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        cg.compton_kernel_timing(ctx, True)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for step in range(3):
            src, dst = ((e_in, g_in), (e_out, g_out)) if step % 2 == 0 else ((e_out, g_out), (e_in, g_in))
            pairs = cg.compton_bin_pairs(ctx, src[0], src[1], dst[0], dst[1], step)
            cg.compton_scatter_step(ctx, dst[0], dst[1], pairs, cg.MODE_PLAIN, step)
        t1.record()
        torch.cuda.synchronize()
        kt = cg.compton_kernel_times(ctx)
        cg.compton_kernel_timing(ctx, False)
    finally:
        cg.compton_destroy(ctx)
    for name in ("k_count", "k_scan", "k_place", "k_sort_gather", "k_pair_prob", "k_collide"):
        assert kt[name]["launches"] == 3, (name, kt[name])
        assert kt[name]["ms"] > 0.0
    assert kt["k_mlp"]["launches"] == 0
    assert sum(v["ms"] for v in kt.values()) <= t0.elapsed_time(t1) * 1.01
