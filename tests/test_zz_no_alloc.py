"""The allocation-free offsets entry point, for callers that cannot allocate
device memory when they need it (a particle-in-cell code whose memory manager
owns all device memory, or a step loop that must not allocate).  Its output
must equal the offsets the context path (compton_bin_pairs) produces, on two
calls in a row (the shared static scratch is cleared by each call), and a
numpy histogram and cumulative sum at the edges: no particles, the largest
accepted cell count, and indices outside [0, n_cells), which are skipped.
This file is collected last on purpose."""
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


def _numpy_offsets(cell, n_cells):
    c = cell[(cell >= 0) & (cell < n_cells)]
    return np.concatenate([[0], np.cumsum(np.bincount(c, minlength=n_cells))]).astype(np.int32)


def _noalloc(cg, torch, cell_np, n_cells):
    cell = torch.from_numpy(np.ascontiguousarray(cell_np, dtype=np.int32)).cuda()
    off = torch.full((n_cells + 1,), -7, dtype=torch.int32, device="cuda")
    cg.compton_cell_offsets_noalloc(cell, n_cells, off)
    torch.cuda.synchronize()
    return off.cpu().numpy()


def test_noalloc_offsets_match_context_path_twice():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    for call, (nx, seed) in enumerate(((96, 2), (40, 5))):  # two calls in a row, different sizes
        w = wl.c2(nx, nx, 48, seed=seed)
        ref_e, ref_g = _context_offsets(cg, torch, w)
        for sp, ref in ((w.e, ref_e), (w.g, ref_g)):
            assert np.array_equal(_noalloc(cg, torch, sp["cell"], w.n_cells), ref), f"call {call}"


def test_noalloc_edges_against_numpy():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    rng = np.random.default_rng(11)
    # no particles at all
    off = _noalloc(cg, torch, np.zeros(0, dtype=np.int32), 1000)
    assert np.array_equal(off, np.zeros(1001, dtype=np.int32))
    # the largest accepted cell count, with a ragged last strip of the scan
    for n_cells in (1 << 20, (1 << 20) - 4093, 4097, 1):
        cell = rng.integers(0, n_cells, 3_000_000, dtype=np.int64).astype(np.int32)
        assert np.array_equal(_noalloc(cg, torch, cell, n_cells), _numpy_offsets(cell, n_cells)), n_cells
    # indices outside [0, n_cells) are skipped; off[n_cells] counts the rest
    n_cells = 70001
    cell = rng.integers(-5000, n_cells + 5000, 1_000_000, dtype=np.int64).astype(np.int32)
    cell[:3] = [-(2 ** 31), 2 ** 31 - 1, n_cells]
    off = _noalloc(cg, torch, cell, n_cells)
    assert np.array_equal(off, _numpy_offsets(cell, n_cells))
    assert off[-1] == int(((cell >= 0) & (cell < n_cells)).sum()) < cell.size


def test_noalloc_rejects_bad_arguments():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    cell = torch.zeros(10, dtype=torch.int32, device="cuda")
    off = torch.zeros(16, dtype=torch.int32, device="cuda")
    big = torch.zeros((1 << 20) + 2, dtype=torch.int32, device="cuda")
    with pytest.raises(cg.ComptonError) as e:
        cg.compton_cell_offsets_noalloc(cell, (1 << 20) + 1, big)
    assert e.value.status == cg.COMPTON_ERANGE
    with pytest.raises(ValueError):   # off_out shorter than n_cells + 1
        cg.compton_cell_offsets_noalloc(cell, 16, off)
    with pytest.raises(ValueError):   # wrong dtype
        cg.compton_cell_offsets_noalloc(cell.to(torch.int64), 8, off)
