"""The allocation-free offsets entry point, for callers that cannot allocate
device memory when they need it (a particle-in-cell code whose memory manager
owns all device memory, or a step loop that must not allocate).  Its output
must equal the offsets the context path (compton_bin_pairs) produces, on two
calls in a row (the shared static scratch is cleared by each call).  This
file is collected last on purpose."""
import numpy as np
import pytest

from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import _dev_array, to_species, torch_cuda

pytestmark = pytest.mark.gpu


def _context_offsets(cg, torch, w):
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        e_in, g_in = to_species(torch, w.e), to_species(torch, w.g)
        e_out, g_out = cg.Species.empty_like(e_in), cg.Species.empty_like(g_in)
        pairs = cg.compton_bin_pairs(ctx, e_in, g_in, e_out, g_out, 0)
        torch.cuda.synchronize()
        return (_dev_array(torch, pairs.off_e_dev, w.n_cells + 1), _dev_array(torch, pairs.off_g_dev, w.n_cells + 1))
    finally:
        cg.compton_destroy(ctx)


def test_noalloc_offsets_match_context_path_twice():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    for call, (nx, seed) in enumerate(((96, 2), (40, 5))):  # two calls in a row, different sizes
        w = wl.c2(nx, nx, 48, seed=seed)
        ref_e, ref_g = _context_offsets(cg, torch, w)
        for sp, ref in ((w.e, ref_e), (w.g, ref_g)):
            cell = torch.from_numpy(sp["cell"]).cuda()
            off = torch.full((w.n_cells + 1,), -7, dtype=torch.int32, device="cuda")
            cg.compton_cell_offsets_noalloc(cell, w.n_cells, off)
            torch.cuda.synchronize()
            assert np.array_equal(off.cpu().numpy(), ref), f"call {call}"


def test_noalloc_rejects_too_many_cells():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    cell = torch.zeros(10, dtype=torch.int32, device="cuda")
    off = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(cg.ComptonError) as e:
        cg.compton_cell_offsets_noalloc(cell, (1 << 20) + 1, off)
    assert e.value.status == cg.COMPTON_ERANGE
