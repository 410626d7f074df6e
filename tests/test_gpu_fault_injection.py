"""Error paths of the C ABI under host-side fault injection
(compton_debug_inject): a checked CUDA call or launch is made to report a
failure on the host, with nothing done to the device.  Every entry point must
return the error status (ENOMEM for the device allocations, ECUDA with the
failing call named by compton_last_error for the rest) and leave the context
usable: the same call repeated without injection gives the result of a
context that never failed."""
import numpy as np
import pytest

from paper_2206_02937_gb300 import workloads as wl
from tests.gpu_util import species_np, to_species, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def disarm():
    yield
    import paper_2206_02937_gb300 as cg
    cg.compton_debug_inject(0, 0)


def _step(cg, torch, ctx, w, A, step=3):
    B = [cg.Species.empty_like(A[0]), cg.Species.empty_like(A[1])]
    p = cg.compton_bin_pairs(ctx, A[0], A[1], B[0], B[1], step)
    cg.compton_scatter_step(ctx, B[0], B[1], p, cg.MODE_PLAIN, step)
    torch.cuda.synchronize()
    return species_np(B[0]), species_np(B[1])


def test_init_allocation_failure_reports_enomem():
    import paper_2206_02937_gb300 as cg
    torch_cuda()
    cg.build()
    cg.compton_debug_inject(0, 1)
    with pytest.raises(cg.ComptonError) as e:
        cg.compton_init(1000, 1000, 1.0, 0.05, 1)
    assert e.value.status == cg.COMPTON_ENOMEM
    assert cg.compton_debug_inject(0, 0) == 0  # the failure was consumed
    ctx = cg.compton_init(1000, 1000, 1.0, 0.05, 1)
    cg.compton_destroy(ctx)


def test_every_failure_point_of_a_step_recovers():
    """Fail the k-th checked call of bin_pairs + scatter_step for every k the
    step reaches; after each failure the context gives the clean result."""
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    w = wl.c2(40, 40, 32, seed=9)
    ctx = cg.compton_init(w.n_cells, max(w.n_e, w.n_g), w.w_over_v, w.dt, w.seed)
    try:
        A = [to_species(torch, w.e), to_species(torch, w.g)]
        ref = _step(cg, torch, ctx, w, A)
        failures = 0
        for k in range(200):
            cg.compton_debug_inject(k, 1)
            try:
                _step(cg, torch, ctx, w, A)
                failed = False
            except cg.ComptonError as e:
                failed = True
                assert e.status == cg.COMPTON_ECUDA
                assert b"injected failure" in cg.lib().compton_last_error(ctx)
            pending = cg.compton_debug_inject(0, 0)
            if pending:  # the step made fewer than k + 1 checks: all points covered
                assert not failed
                break
            assert failed
            failures += 1
            torch.cuda.synchronize()
            got = _step(cg, torch, ctx, w, A)
            for s in (0, 1):
                for key in ("ux", "uy", "uz", "id", "cell"):
                    assert np.array_equal(got[s][key], ref[s][key]), (k, key)
        assert failures >= 5
        assert cg.compton_check(ctx) == cg.COMPTON_OK
    finally:
        cg.compton_destroy(ctx)


def test_network_and_training_calls_report_injected_failures():
    import paper_2206_02937_gb300 as cg
    from oracle import mlp as omlp
    torch = torch_cuda()
    cg.build()
    n = 5000
    u, k = wl.c3(n, seed=13)
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1, max_train_batch=n)
    try:
        ut, kt = torch.from_numpy(u).cuda(), torch.from_numpy(k).cuda()
        cg.compton_mlp_set_params(ctx, omlp.init_params(3).astype(np.float32))
        r = torch.zeros(n, device="cuda")
        cg.compton_kn_ratio(ctx, ut, kt, r)
        out0 = torch.zeros(n, device="cuda")
        cg.compton_mlp_infer(ctx, ut, kt, cg.MODE_MLP_BF16, out0)
        torch.cuda.synchronize()
        for call in ("infer", "train", "ratio"):
            cg.compton_debug_inject(0, 1)
            with pytest.raises(cg.ComptonError) as e:
                if call == "infer":
                    cg.compton_mlp_infer(ctx, ut, kt, cg.MODE_MLP_BF16, torch.zeros(n, device="cuda"))
                elif call == "train":
                    cg.compton_mlp_train_step(ctx, ut, kt, r, None, lr=0.0)
                else:
                    cg.compton_kn_ratio(ctx, ut, kt, torch.zeros(n, device="cuda"))
            assert e.value.status == cg.COMPTON_ECUDA, call
            assert cg.compton_debug_inject(0, 0) == 0
        out1 = torch.zeros(n, device="cuda")
        cg.compton_mlp_infer(ctx, ut, kt, cg.MODE_MLP_BF16, out1)
        torch.cuda.synchronize()
        assert torch.equal(out0, out1)
        cg.compton_mlp_train_step(ctx, ut, kt, r, None, lr=1e-3)
        assert cg.compton_check(ctx) == cg.COMPTON_OK
    finally:
        cg.compton_destroy(ctx)


def test_serving_pool_allocation_failure_reports_enomem():
    import paper_2206_02937_gb300 as cg
    torch = torch_cuda()
    cg.build()
    ctx = cg.compton_init(1, 0, 1.0, 0.05, 1)
    try:
        # fail each checked call of the start in turn: the pool allocation
        # reports ENOMEM, the calls before it ECUDA; each failure leaves no
        # engine behind, so the next start is clean
        statuses = []
        for skip in range(8):
            cg.compton_debug_inject(skip, 1)
            try:
                cg.compton_serve_start(ctx, 1 << 26, 16)
            except cg.ComptonError as e:
                statuses.append(e.status)
                assert cg.compton_debug_inject(0, 0) == 0
                continue
            cg.compton_debug_inject(0, 0)
            cg.compton_serve_stop(ctx)
            break
        assert cg.COMPTON_ENOMEM in statuses
        assert set(statuses) <= {cg.COMPTON_ENOMEM, cg.COMPTON_ECUDA}
        cg.compton_serve_start(ctx, 1 << 26, 16)
        u = torch.rand(3, 1000, device="cuda")
        k = torch.rand(3, 1000, device="cuda") * 1e-2
        uo, ko = torch.empty_like(u), torch.empty_like(k)
        t = cg.compton_submit(ctx, u, k, uo, ko, 1.0, 7, 0, cg.MODE_PLAIN)
        import time
        t0 = time.time()
        while cg.compton_poll(ctx, t) is None:
            assert time.time() - t0 < 30
            time.sleep(0.001)
        cg.compton_serve_stop(ctx)
    finally:
        cg.compton_destroy(ctx)
