// api.cu -- the extern "C" entry points of libcompton: argument checking,
// context and arena management, status codes.  The kernels live in
// bin_pairs.cu and scatter.cu.
#include <cmath>
#include <cstdlib>
#include <new>

#include <atomic>
#include <mutex>

#include "ctx.hpp"

using compton::CellInfo;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
    size_t used = 0;
    template <class T>
    size_t take(size_t count)
    {
        size_t at = align_up(used, 256);
        used = at + count * sizeof(T);
        return at;
    }
};

bool species_ok(const compton_species* s)
{
    if (!s || s->n < 0) return false;
    if (s->n == 0) return true;
    return s->ux_dev && s->uy_dev && s->uz_dev && s->cell_dev && s->id_dev;
}

bool overlaps(const void* a, const void* b, int64_t n, size_t elem)
{
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    const size_t bytes = (size_t)n * elem;
    return pa < pb + bytes && pb < pa + bytes;
}

bool species_alias(const compton_species* a, const compton_species* b, int64_t n)
{
    const void* pa[6] = {a->ux_dev, a->uy_dev, a->uz_dev, a->cell_dev, a->id_dev, a->w_dev};
    const void* pb[6] = {b->ux_dev, b->uy_dev, b->uz_dev, b->cell_dev, b->id_dev, b->w_dev};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            if (pa[i] && pb[j] && overlaps(pa[i], pb[j], n, 4)) return true;
    return false;
}

}  // namespace

extern "C" {

const char* compton_strerror(compton_status s)
{
    switch (s) {
    case COMPTON_OK: return "ok";
    case COMPTON_EINVAL: return "invalid argument";
    case COMPTON_ENOMEM: return "out of device memory or over the memory budget";
    case COMPTON_EBUSY: return "no slot or budget free; retry later";
    case COMPTON_ETIMEOUT: return "a bounded device wait timed out";
    case COMPTON_ERANGE: return "input out of range";
    case COMPTON_ENOTREADY: return "not finished";
    case COMPTON_ECUDA: return "CUDA error";
    case COMPTON_ENOMODEL: return "no surrogate network loaded";
    }
    return "unknown status";
}

const char* compton_last_error(const compton_ctx* ctx) { return ctx ? ctx->last_error : ""; }

compton_status compton_init(const compton_config* cfg, compton_ctx** out)
{
    if (!cfg || !out) return COMPTON_EINVAL;
    *out = nullptr;
    if (cfg->n_cells <= 0 || cfg->n_cells >= INT32_MAX - 1) return COMPTON_EINVAL;
    if (cfg->max_particles < 0 || cfg->max_particles >= INT32_MAX - compton::kSortCap) return COMPTON_EINVAL;
    if (!(cfg->dt >= 0.0) || !(cfg->w_over_v >= 0.0) || std::isinf(cfg->dt) || std::isinf(cfg->w_over_v))
        return COMPTON_EINVAL;
    if (!(cfg->gamma_fp64_threshold >= 0.0f) || !(cfg->collide_fp64_threshold >= 0.0f)) return COMPTON_EINVAL;
    compton_ctx* ctx = new (std::nothrow) compton_ctx();
    if (!ctx) return COMPTON_ENOMEM;
    ctx->cfg = *cfg;
    ctx->last_error[0] = '\0';
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
    if (e != cudaSuccess) {
        delete ctx;
        return COMPTON_ECUDA;
    }
    if (ctx->n_sm < 1) ctx->n_sm = 1;
    const int64_t C = cfg->n_cells;
    const int64_t P = cfg->max_particles;
    ctx->max_scan_tiles = (C + compton::kScanTile - 1) / compton::kScanTile;
    ctx->max_sort_tiles = (P + compton::kSortTile - 1) / compton::kSortTile + 1;
    ctx->max_pair_tiles = (P + compton::kPairsPerTile - 1) / compton::kPairsPerTile + 1;

    Carver cv;
    // both histograms and the two order flags in one block, cleared by one
    // memset per binning call; the second histogram starts 256-byte aligned
    const size_t C_pad = align_up((size_t)C, 64);
    const size_t o_count = cv.take<int32_t>(2 * C_pad + 2);
    size_t o_off[2], o_rec[2], o_stile[2];
    for (int s = 0; s < 2; ++s) {
        o_off[s] = cv.take<int32_t>(C + 1);
        o_rec[s] = cv.take<compton::SortRec>(P > 0 ? P : 1);
        o_stile[s] = cv.take<int32_t>(ctx->max_sort_tiles + 1);
    }
    size_t o_bs = cv.take<int64_t>(3 * ctx->max_scan_tiles);
    size_t o_ci = cv.take<CellInfo>(C);
    size_t o_tc = cv.take<int32_t>(ctx->max_pair_tiles + 1);
    size_t o_np = cv.take<int64_t>(1);
    ctx->accepted_cap = P > ((int64_t)1 << 20) ? P : ((int64_t)1 << 20);
    size_t o_acc = cv.take<compton::AcceptedPair>(ctx->accepted_cap);
    size_t o_nacc = cv.take<uint32_t>(1);
    size_t o_wacc = cv.take<uint32_t>(compton::kMaxProbWarps);
    size_t o_cand = cv.take<compton::CandPair>(ctx->accepted_cap);
    size_t o_ncand = cv.take<uint32_t>(1);
    size_t o_st = cv.take<compton::DeviceStats>(1);
    const size_t NP = compton::kMlpParams;
    size_t o_th = cv.take<float>(NP), o_gr = cv.take<float>(NP), o_am = cv.take<float>(NP),
           o_av = cv.take<float>(NP);
    size_t o_wb = cv.take<uint8_t>(4 * 8192), o_w8 = cv.take<uint8_t>(4 * 8192), o_wt = cv.take<float>(4 * 4096);
    size_t o_wh = cv.take<uint8_t>(4 * 8192 + 3 * 2048);
    size_t o_bi = cv.take<float>(256), o_w4 = cv.take<float>(64), o_b4 = cv.take<float>(1);
    size_t o_sw = cv.take<float>(4), o_swi = cv.take<float>(4), o_sai = cv.take<float>(4), o_lo = cv.take<float>(2),
           o_ax = cv.take<float>(4), o_ed = cv.take<float>(257), o_hi = cv.take<int>(256);
    if (cfg->max_train_batch < 0 || cfg->max_train_batch > (int64_t)1 << 31) {
        delete ctx;
        return COMPTON_EINVAL;
    }
    size_t o_tr = cv.take<uint8_t>(cfg->max_train_batch > 0 ? compton::train_scratch_bytes(cfg->max_train_batch) : 1);
    size_t o_rb = cv.take<float>(P > 0 ? P : 1);
    size_t o_pn = cv.take<float>(4 * compton::kPnetParams + 2);
    const size_t total = align_up(cv.used, 256);
    if (cfg->mem_budget_bytes && total > cfg->mem_budget_bytes) {
        delete ctx;
        return COMPTON_ENOMEM;
    }
    e = compton::inject_fault() ? cudaErrorMemoryAllocation : cudaMalloc(&ctx->arena, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return COMPTON_ENOMEM;
    }
    ctx->arena_bytes = total;
    char* base = static_cast<char*>(ctx->arena);
    for (int s = 0; s < 2; ++s) {
        ctx->count[s] = reinterpret_cast<int32_t*>(base + o_count) + s * C_pad;
        ctx->off[s] = reinterpret_cast<int32_t*>(base + o_off[s]);
        ctx->rec[s] = reinterpret_cast<compton::SortRec*>(base + o_rec[s]);
        ctx->stile[s] = reinterpret_cast<int32_t*>(base + o_stile[s]);
    }
    ctx->unsorted = reinterpret_cast<int32_t*>(base + o_count) + 2 * C_pad;
    ctx->block_sums = reinterpret_cast<int64_t*>(base + o_bs);
    ctx->cinfo = reinterpret_cast<CellInfo*>(base + o_ci);
    ctx->tile_cell = reinterpret_cast<int32_t*>(base + o_tc);
    ctx->n_pairs = reinterpret_cast<int64_t*>(base + o_np);
    ctx->accepted = reinterpret_cast<compton::AcceptedPair*>(base + o_acc);
    ctx->n_accepted = reinterpret_cast<uint32_t*>(base + o_nacc);
    ctx->warp_acc = reinterpret_cast<uint32_t*>(base + o_wacc);
    ctx->cand = reinterpret_cast<compton::CandPair*>(base + o_cand);
    ctx->n_cand = reinterpret_cast<uint32_t*>(base + o_ncand);
    ctx->stats = reinterpret_cast<compton::DeviceStats*>(base + o_st);
    compton::MlpDev& m = ctx->mlp;
    m.theta = reinterpret_cast<float*>(base + o_th);
    m.grad = reinterpret_cast<float*>(base + o_gr);
    m.adam_m = reinterpret_cast<float*>(base + o_am);
    m.adam_v = reinterpret_cast<float*>(base + o_av);
    m.wbf16 = base + o_wb;
    m.whalf = base + o_wh;
    m.wfp8 = base + o_w8;
    m.wt32 = reinterpret_cast<float*>(base + o_wt);
    m.bias = reinterpret_cast<float*>(base + o_bi);
    m.w4 = reinterpret_cast<float*>(base + o_w4);
    m.b4 = reinterpret_cast<float*>(base + o_b4);
    m.scale_w = reinterpret_cast<float*>(base + o_sw);
    m.scale_w_inv = reinterpret_cast<float*>(base + o_swi);
    m.scale_a_inv = reinterpret_cast<float*>(base + o_sai);
    m.loss = reinterpret_cast<float*>(base + o_lo);
    m.amax = reinterpret_cast<float*>(base + o_ax);
    m.edges = reinterpret_cast<float*>(base + o_ed);
    m.hist = reinterpret_cast<int*>(base + o_hi);
    ctx->train_scratch = base + o_tr;
    ctx->r_buf = reinterpret_cast<float*>(base + o_rb);
    {
        float* pb = reinterpret_cast<float*>(base + o_pn);
        compton::PnetDev& pn = ctx->pnet;
        pn.theta = pb;
        pn.grad = pb + compton::kPnetParams;
        pn.adam_m = pb + 2 * compton::kPnetParams;
        pn.adam_v = pb + 3 * compton::kPnetParams;
        pn.loss = pb + 4 * compton::kPnetParams;
        pn.fs[0] = 1.0f;
        pn.fs[1] = 7.0f;
        pn.fs[2] = 1e-4f;
        pn.fs[3] = 10.0f;
        pn.range[0] = 1.0e6f;
        pn.range[1] = 1.0e-8f;
        pn.range[2] = 1.0f;
        pn.step = 0;
    }
    m.fs[0] = 1.0f;   // s_u
    m.fs[1] = 7.0f;   // n_u
    m.fs[2] = 1e-4f;  // s_k
    m.fs[3] = 10.0f;  // n_k
    m.feat_mode = COMPTON_FEATURES_MOMENTA;
    m.range_g2max = 1.0e6f;  // gamma <= 1e3
    m.range_e2min = 1.0e-8f; // eps >= 1e-4
    m.range_e2max = 1.0f;    // eps <= 1
    e = cudaMemset(ctx->arena, 0, total);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ctx->arena);
        delete ctx;
        return COMPTON_ECUDA;
    }
    *out = ctx;
    return COMPTON_OK;
}

compton_status compton_destroy(compton_ctx* ctx)
{
    if (!ctx) return COMPTON_OK;
    cudaSetDevice(ctx->cfg.device);
    compton::serve_stop(ctx);
    cudaDeviceSynchronize();
    if (ctx->timing) {
        for (int s = 0; s < compton::kTimedSlots; ++s)
            for (int k = 0; k < compton::kTimingRing; ++k) {
                cudaEventDestroy(ctx->timing->ev[s][k][0]);
                cudaEventDestroy(ctx->timing->ev[s][k][1]);
            }
        delete ctx->timing;
    }
    if (ctx->arena) cudaFree(ctx->arena);
    delete ctx;
    return COMPTON_OK;
}

compton_status compton_kernel_timing(compton_ctx* ctx, int32_t enable)
{
    if (!ctx) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaSetDevice(ctx->cfg.device));
    if (!enable) {
        if (ctx->timing) ctx->timing->on = false;
        return COMPTON_OK;
    }
    if (!ctx->timing) {
        compton::KernelTiming* T = new (std::nothrow) compton::KernelTiming();
        if (!T) return COMPTON_ENOMEM;
        for (int s = 0; s < compton::kTimedSlots; ++s)
            for (int k = 0; k < compton::kTimingRing; ++k)
                for (int j = 0; j < 2; ++j) {
                    const cudaError_t e = cudaEventCreate(&T->ev[s][k][j]);
                    if (e != cudaSuccess) {
                        for (int s2 = 0; s2 <= s; ++s2)
                            for (int k2 = 0; k2 < compton::kTimingRing; ++k2)
                                for (int j2 = 0; j2 < 2; ++j2) {
                                    if (s2 == s && (k2 > k || (k2 == k && j2 >= j))) continue;
                                    cudaEventDestroy(T->ev[s2][k2][j2]);
                                }
                        delete T;
                        return compton::set_cuda_error(ctx, e, "cudaEventCreate");
                    }
                }
        ctx->timing = T;
    }
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    for (int s = 0; s < compton::kTimedSlots; ++s) ctx->timing->n[s] = 0;
    ctx->timing->on = true;
    return COMPTON_OK;
}

compton_status compton_kernel_times(compton_ctx* ctx, double* ms_out, int64_t* launches_out)
{
    if (!ctx || !ms_out || !launches_out) return COMPTON_EINVAL;
    if (!ctx->timing) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaSetDevice(ctx->cfg.device));
    const compton::KernelTiming& T = *ctx->timing;
    for (int s = 0; s < compton::kTimedSlots; ++s) {
        const int64_t kept = T.n[s] < compton::kTimingRing ? T.n[s] : compton::kTimingRing;
        double sum = 0.0;
        for (int64_t k = 0; k < kept; ++k) {
            const int i = (int)((T.n[s] - kept + k) % compton::kTimingRing);
            COMPTON_CUDA_TRY(ctx, cudaEventSynchronize(T.ev[s][i][1]));
            float ms = 0.0f;
            COMPTON_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, T.ev[s][i][0], T.ev[s][i][1]));
            sum += ms;
        }
        ms_out[s] = sum;
        launches_out[s] = kept;
    }
    return COMPTON_OK;
}

compton_status compton_check(compton_ctx* ctx, compton_stream_t stream)
{
    if (!ctx) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    unsigned long long flags = 0;
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(&flags, &ctx->stats->error_flags, sizeof(flags), cudaMemcpyDeviceToHost));
    if (flags) {
        COMPTON_CUDA_TRY(ctx, cudaMemset(&ctx->stats->error_flags, 0, sizeof(flags)));
        return (flags & compton::kErrTimeout) ? COMPTON_ETIMEOUT : COMPTON_ERANGE;
    }
    return COMPTON_OK;
}

compton_status compton_get_stats(compton_ctx* ctx, compton_stats* out, int reset, compton_stream_t stream)
{
    if (!ctx || !out) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    compton::DeviceStats d;
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(&d, ctx->stats, sizeof(d), cudaMemcpyDeviceToHost));
    out->pairs_tested = d.pairs_tested;
    out->scatters = d.scatters;
    out->mlp_fallbacks = d.mlp_fallbacks;
    out->error_flags = d.error_flags;
    if (reset) COMPTON_CUDA_TRY(ctx, cudaMemset(ctx->stats, 0, sizeof(d)));
    return COMPTON_OK;
}

compton_status compton_bin_pairs(compton_ctx* ctx, const compton_species* e_in, const compton_species* g_in,
                                 compton_species* e_out, compton_species* g_out, uint64_t step,
                                 compton_pairs* pairs_out, compton_stream_t stream)
{
    if (!ctx || !pairs_out || !species_ok(e_in) || !species_ok(g_in) || !e_out || !g_out) return COMPTON_EINVAL;
    if (e_in->n > ctx->cfg.max_particles || g_in->n > ctx->cfg.max_particles) return COMPTON_ERANGE;
    e_out->n = e_in->n;
    g_out->n = g_in->n;
    if (!species_ok(e_out) || !species_ok(g_out)) return COMPTON_EINVAL;
    // weights travel with the particles: an output for every weighted input
    if ((e_in->w_dev && e_in->n > 0 && !e_out->w_dev) || (g_in->w_dev && g_in->n > 0 && !g_out->w_dev))
        return COMPTON_EINVAL;
    if (species_alias(e_in, e_out, e_in->n) || species_alias(g_in, g_out, g_in->n)) return COMPTON_EINVAL;
    compton_status st = compton::launch_bin_pairs(ctx, e_in, g_in, e_out, g_out, step, stream);
    if (st != COMPTON_OK) return st;
    ctx->bin_weighted = e_in->w_dev || g_in->w_dev;
    pairs_out->off_e_dev = ctx->off[0];
    pairs_out->off_g_dev = ctx->off[1];
    pairs_out->cell_info_dev = ctx->cinfo;
    pairs_out->tile_cell_dev = ctx->tile_cell;
    pairs_out->n_pairs_dev = ctx->n_pairs;
    pairs_out->max_pairs = e_in->n < g_in->n ? e_in->n : g_in->n;
    pairs_out->n_cells = ctx->cfg.n_cells;
    return COMPTON_OK;
}

compton_status compton_scatter_step(compton_ctx* ctx, compton_species* e, compton_species* g,
                                    const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                    float* prob_out, uint8_t* flag_out, compton_stream_t stream)
{
    if (!ctx || !pairs || !species_ok(e) || !species_ok(g)) return COMPTON_EINVAL;
    if (pairs->cell_info_dev != ctx->cinfo || pairs->n_cells != ctx->cfg.n_cells) return COMPTON_EINVAL;
    if (pairs->max_pairs > (e->n < g->n ? e->n : g->n)) return COMPTON_EINVAL;
    if ((int)mode < 0 || (int)mode > 4) return COMPTON_EINVAL;
    if ((e->w_dev || g->w_dev) != ctx->bin_weighted) return COMPTON_EINVAL;
    if (mode == COMPTON_MODE_PNET ? !ctx->pnet_loaded : (mode != COMPTON_MODE_PLAIN && !ctx->mlp_loaded))
        return COMPTON_ENOMODEL;
    return compton::launch_scatter_binned(ctx, e, g, pairs, mode, step, prob_out, flag_out, stream);
}

compton_status compton_scatter_step_ntc(compton_ctx* ctx, compton_species* e, compton_species* g,
                                        const compton_pairs* pairs, uint64_t step, compton_stream_t stream)
{
    if (!ctx || !pairs || !species_ok(e) || !species_ok(g)) return COMPTON_EINVAL;
    if (pairs->cell_info_dev != ctx->cinfo || pairs->n_cells != ctx->cfg.n_cells) return COMPTON_EINVAL;
    if (e->w_dev || g->w_dev || ctx->bin_weighted) return COMPTON_EINVAL;
    return compton::launch_scatter_ntc(ctx, e, g, pairs, step, stream);
}

compton_status compton_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                     float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                     compton_mode mode, float* prob_out, uint8_t* flag_out,
                                     compton_stream_t stream)
{
    if (!ctx || n < 0 || n > INT32_MAX) return COMPTON_EINVAL;
    if (n == 0) return COMPTON_OK;
    if (!ux || !uy || !uz || !kx || !ky || !kz || !n_dens) return COMPTON_EINVAL;
    if ((int)mode < 0 || (int)mode > 3) return COMPTON_EINVAL;
    if (mode != COMPTON_MODE_PLAIN && !ctx->mlp_loaded) return COMPTON_ENOMODEL;
    return compton::launch_scatter_pairs(ctx, ux, uy, uz, kx, ky, kz, n_dens, n, seed, step, mode, prob_out,
                                         flag_out, stream);
}

compton_status compton_kn_ratio(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                const float* kx, const float* ky, const float* kz, int64_t n, float* r_out,
                                compton_stream_t stream)
{
    if (!ctx || n < 0) return COMPTON_EINVAL;
    if (n == 0) return COMPTON_OK;
    if (!ux || !uy || !uz || !kx || !ky || !kz || !r_out) return COMPTON_EINVAL;
    return compton::launch_kn_ratio(ctx, ux, uy, uz, kx, ky, kz, n, r_out, stream);
}

// ---------------------------------------------------------------------------
// Surrogate network
// ---------------------------------------------------------------------------
compton_status compton_mlp_set_params(compton_ctx* ctx, const float* theta, int64_t n_params,
                                      const float* feature_scales)
{
    if (!ctx || !theta || n_params != compton::kMlpParams) return COMPTON_EINVAL;
    if (feature_scales) {
        for (int i = 0; i < 4; ++i)
            if (!(feature_scales[i] > 0.0f) || std::isinf(feature_scales[i])) return COMPTON_EINVAL;
        for (int i = 0; i < 4; ++i) ctx->mlp.fs[i] = feature_scales[i];
    }
    COMPTON_CUDA_TRY(ctx, cudaSetDevice(ctx->cfg.device));
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(ctx->mlp.theta, theta, sizeof(float) * n_params, cudaMemcpyHostToDevice));
    COMPTON_CUDA_TRY(ctx, cudaMemset(ctx->mlp.adam_m, 0, sizeof(float) * n_params));
    COMPTON_CUDA_TRY(ctx, cudaMemset(ctx->mlp.adam_v, 0, sizeof(float) * n_params));
    ctx->adam_step = 0;
    // default FP8 activation scales until compton_mlp_calibrate: |inputs| <= 4
    const float sai[4] = {112.0f, 112.0f, 112.0f, 112.0f};
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(ctx->mlp.scale_a_inv, sai, sizeof(sai), cudaMemcpyHostToDevice));
    compton_status st = compton::mlp_repack(ctx, nullptr);
    if (st != COMPTON_OK) return st;
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    ctx->mlp_loaded = true;
    return COMPTON_OK;
}

compton_status compton_mlp_get_params(compton_ctx* ctx, float* theta, int64_t n_params)
{
    if (!ctx || !theta || n_params != compton::kMlpParams) return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(theta, ctx->mlp.theta, sizeof(float) * n_params, cudaMemcpyDeviceToHost));
    return COMPTON_OK;
}

compton_status compton_mlp_calibrate(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                     const float* kx, const float* ky, const float* kz, int64_t n,
                                     compton_stream_t stream)
{
    if (!ctx || n <= 0 || !ux || !uy || !uz || !kx || !ky || !kz) return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    return compton::launch_mlp_calibrate(ctx, ux, uy, uz, kx, ky, kz, n, stream);
}

compton_status compton_mlp_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                 const float* kx, const float* ky, const float* kz, int64_t n, compton_mode mode,
                                 float* r_out, compton_stream_t stream)
{
    if (!ctx || n < 0) return COMPTON_EINVAL;
    if (mode != COMPTON_MODE_MLP_FP32 && mode != COMPTON_MODE_MLP_BF16 && mode != COMPTON_MODE_MLP_FP8)
        return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    if (n == 0) return COMPTON_OK;
    if (!ux || !uy || !uz || !kx || !ky || !kz || !r_out) return COMPTON_EINVAL;
    return compton::launch_mlp_infer(ctx, ux, uy, uz, kx, ky, kz, n, mode, r_out, stream);
}

compton_status compton_mlp_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                      const float* kx, const float* ky, const float* kz, const float* y,
                                      const float* w, int64_t n, float lr, float* loss_out,
                                      compton_stream_t stream)
{
    if (!ctx || n <= 0 || !ux || !uy || !uz || !kx || !ky || !kz || !y) return COMPTON_EINVAL;
    if (!(lr >= 0.0f) || std::isinf(lr)) return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    if (n > ctx->cfg.max_train_batch) return COMPTON_ERANGE;
    compton_status st = compton::launch_mlp_train_step(ctx, ux, uy, uz, kx, ky, kz, y, w, n, lr, stream);
    if (st != COMPTON_OK || !loss_out) return st;
    float l[2];
    COMPTON_CUDA_TRY(ctx, cudaMemcpyAsync(l, ctx->mlp.loss, sizeof(l), cudaMemcpyDeviceToHost, stream));
    COMPTON_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    *loss_out = l[1] > 0.0f ? l[0] / l[1] : 0.0f;
    return COMPTON_OK;
}

compton_status compton_mlp_set_train_precision(compton_ctx* ctx, compton_mode mode)
{
    if (!ctx) return COMPTON_EINVAL;
    if (mode != COMPTON_MODE_MLP_FP32 && mode != COMPTON_MODE_MLP_BF16) return COMPTON_EINVAL;
    ctx->train_tc = mode == COMPTON_MODE_MLP_BF16;
    return COMPTON_OK;
}

compton_status compton_mlp_balance_weights(compton_ctx* ctx, const float* r, int64_t n, const float* edges,
                                           int32_t n_bins, float* w_out, compton_stream_t stream)
{
    if (!ctx || !r || !edges || !w_out || n <= 0 || n_bins < 1 || n_bins > 256) return COMPTON_EINVAL;
    for (int i = 0; i < n_bins; ++i)
        if (!(edges[i] < edges[i + 1])) return COMPTON_EINVAL;
    return compton::launch_balance_weights(ctx, r, n, edges, n_bins, w_out, stream);
}

compton_status compton_mlp_get_grad(compton_ctx* ctx, float* grad, int64_t n_params)
{
    if (!ctx || !grad || n_params != compton::kMlpParams) return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    float l[2];
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(l, ctx->mlp.loss, sizeof(l), cudaMemcpyDeviceToHost));
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(grad, ctx->mlp.grad, sizeof(float) * n_params, cudaMemcpyDeviceToHost));
    const float inv = l[1] > 0.0f ? 1.0f / l[1] : 0.0f;
    for (int64_t i = 0; i < n_params; ++i) grad[i] *= inv;
    return COMPTON_OK;
}

namespace {
struct MlpBlobHeaderV1 {
    char magic[4];
    uint32_t version;
    int64_t n_params;
    int64_t adam_step;
    float fs[4];
    float scale_a_inv[4];
};
struct MlpBlobHeader {
    MlpBlobHeaderV1 v1;
    int32_t feat_mode;
    int32_t reserved;
    float range[4];  // version 3: gamma^2 max, eps^2 min, eps^2 max, unused
};
constexpr size_t kBlobHeadV2 = sizeof(MlpBlobHeaderV1) + 2 * sizeof(int32_t);
}  // namespace

compton_status compton_mlp_save(compton_ctx* ctx, void* buf, size_t* len)
{
    if (!ctx || !len) return COMPTON_EINVAL;
    if (!ctx->mlp_loaded) return COMPTON_ENOMODEL;
    const size_t NP = compton::kMlpParams;
    const size_t need = sizeof(MlpBlobHeader) + 3 * NP * sizeof(float);
    if (!buf || *len < need) {
        *len = need;
        return buf ? COMPTON_ERANGE : COMPTON_OK;
    }
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    MlpBlobHeader h;
    std::memcpy(h.v1.magic, "CMLP", 4);
    h.v1.version = 3;
    h.v1.n_params = (int64_t)NP;
    h.v1.adam_step = ctx->adam_step;
    for (int i = 0; i < 4; ++i) h.v1.fs[i] = ctx->mlp.fs[i];
    h.feat_mode = ctx->mlp.feat_mode;
    h.reserved = 0;
    h.range[0] = ctx->mlp.range_g2max;
    h.range[1] = ctx->mlp.range_e2min;
    h.range[2] = ctx->mlp.range_e2max;
    h.range[3] = 0.0f;
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(h.v1.scale_a_inv, ctx->mlp.scale_a_inv, sizeof(h.v1.scale_a_inv),
                                     cudaMemcpyDeviceToHost));
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const float* src[3] = {ctx->mlp.theta, ctx->mlp.adam_m, ctx->mlp.adam_v};
    for (int i = 0; i < 3; ++i) {
        COMPTON_CUDA_TRY(ctx, cudaMemcpy(p, src[i], NP * sizeof(float), cudaMemcpyDeviceToHost));
        p += NP * sizeof(float);
    }
    *len = need;
    return COMPTON_OK;
}

compton_status compton_mlp_load(compton_ctx* ctx, const void* buf, size_t len)
{
    if (!ctx || !buf || len < sizeof(MlpBlobHeaderV1)) return COMPTON_EINVAL;
    MlpBlobHeaderV1 h;
    std::memcpy(&h, buf, sizeof(h));
    const size_t NP = compton::kMlpParams;
    if (std::memcmp(h.magic, "CMLP", 4) != 0 || h.version < 1 || h.version > 3 || h.n_params != (int64_t)NP)
        return COMPTON_EINVAL;
    const size_t head = h.version == 1 ? sizeof(MlpBlobHeaderV1) : (h.version == 2 ? kBlobHeadV2 : sizeof(MlpBlobHeader));
    if (len != head + 3 * NP * sizeof(float)) return COMPTON_EINVAL;
    MlpBlobHeader h3{};
    std::memcpy(&h3, buf, head);
    const int32_t mode = h.version >= 2 ? h3.feat_mode : (int32_t)COMPTON_FEATURES_MOMENTA;
    if (mode != COMPTON_FEATURES_MOMENTA && mode != COMPTON_FEATURES_INVARIANTS) return COMPTON_EINVAL;
    const char* p = static_cast<const char*>(buf) + head;
    compton_status st = compton_mlp_set_params(ctx, reinterpret_cast<const float*>(p), (int64_t)NP, h.fs);
    if (st != COMPTON_OK) return st;
    ctx->mlp.feat_mode = mode;
    if (h.version >= 3) {
        ctx->mlp.range_g2max = h3.range[0];
        ctx->mlp.range_e2min = h3.range[1];
        ctx->mlp.range_e2max = h3.range[2];
    }
    p += NP * sizeof(float);
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(ctx->mlp.adam_m, p, NP * sizeof(float), cudaMemcpyHostToDevice));
    p += NP * sizeof(float);
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(ctx->mlp.adam_v, p, NP * sizeof(float), cudaMemcpyHostToDevice));
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(ctx->mlp.scale_a_inv, h.scale_a_inv, sizeof(h.scale_a_inv),
                                     cudaMemcpyHostToDevice));
    ctx->adam_step = h.adam_step;
    return COMPTON_OK;
}

compton_status compton_mlp_set_range(compton_ctx* ctx, double gamma_max, double eps_min, double eps_max)
{
    if (!ctx) return COMPTON_EINVAL;
    if (!(gamma_max >= 1.0) || !(eps_min >= 0.0) || !(eps_max > eps_min) || std::isinf(eps_max) ||
        std::isinf(gamma_max))
        return COMPTON_EINVAL;
    ctx->mlp.range_g2max = (float)(gamma_max * gamma_max);
    ctx->mlp.range_e2min = (float)(eps_min * eps_min);
    ctx->mlp.range_e2max = (float)(eps_max * eps_max);
    return COMPTON_OK;
}

compton_status compton_pnet_set_params(compton_ctx* ctx, const float* theta_host, int64_t n_params,
                                      const float* feature_scales_host, double gamma_max, double eps_min,
                                      double eps_max)
{
    if (!ctx || !theta_host || n_params != compton::kPnetParams) return COMPTON_EINVAL;
    if (!(gamma_max >= 1.0) || !(eps_min >= 0.0) || !(eps_max > eps_min) || std::isinf(eps_max) ||
        std::isinf(gamma_max))
        return COMPTON_EINVAL;
    compton::PnetDev& pn = ctx->pnet;
    if (feature_scales_host) {
        for (int i = 0; i < 4; ++i)
            if (!(feature_scales_host[i] > 0.0f)) return COMPTON_EINVAL;
        for (int i = 0; i < 4; ++i) pn.fs[i] = feature_scales_host[i];
    }
    pn.range[0] = (float)(gamma_max * gamma_max);
    pn.range[1] = (float)(eps_min * eps_min);
    pn.range[2] = (float)(eps_max * eps_max);
    COMPTON_CUDA_TRY(ctx, cudaSetDevice(ctx->cfg.device));
    COMPTON_CUDA_TRY(ctx, cudaMemcpy(pn.theta, theta_host, sizeof(float) * compton::kPnetParams,
                                     cudaMemcpyHostToDevice));
    COMPTON_CUDA_TRY(ctx, cudaMemset(pn.adam_m, 0, sizeof(float) * 2 * compton::kPnetParams));
    pn.step = 0;
    ctx->pnet_loaded = true;
    return COMPTON_OK;
}

compton_status compton_pnet_get_params(compton_ctx* ctx, float* theta_host, float* grad_host, int64_t n_params)
{
    if (!ctx || n_params != compton::kPnetParams) return COMPTON_EINVAL;
    if (!ctx->pnet_loaded) return COMPTON_ENOMODEL;
    COMPTON_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (theta_host)
        COMPTON_CUDA_TRY(ctx, cudaMemcpy(theta_host, ctx->pnet.theta, sizeof(float) * compton::kPnetParams,
                                         cudaMemcpyDeviceToHost));
    if (grad_host)
        COMPTON_CUDA_TRY(ctx, cudaMemcpy(grad_host, ctx->pnet.grad, sizeof(float) * compton::kPnetParams,
                                         cudaMemcpyDeviceToHost));
    return COMPTON_OK;
}

compton_status compton_pnet_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                  const float* kx, const float* ky, const float* kz, int64_t n, float w_e,
                                  float w_g, float p_max, float* r_out, compton_stream_t stream)
{
    if (!ctx || n < 0 || (n > 0 && (!ux || !uy || !uz || !kx || !ky || !kz || !r_out))) return COMPTON_EINVAL;
    if (!(w_e > 0.0f) || !(w_g > 0.0f) || !(p_max > 0.0f)) return COMPTON_EINVAL;
    if (!ctx->pnet_loaded) return COMPTON_ENOMODEL;
    return compton::launch_pnet_infer(ctx, ux, uy, uz, kx, ky, kz, n, w_e, w_g, p_max, r_out, stream);
}

compton_status compton_pnet_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                       const float* kx, const float* ky, const float* kz, const float* y,
                                       const float* w, int64_t n, float w_e, float w_g, float p_max, float lr,
                                       float* loss_out_host, compton_stream_t stream)
{
    if (!ctx || n <= 0 || !ux || !uy || !uz || !kx || !ky || !kz || !y) return COMPTON_EINVAL;
    if (!(w_e > 0.0f) || !(w_g > 0.0f) || !(p_max > 0.0f) || !(lr >= 0.0f)) return COMPTON_EINVAL;
    if (!ctx->pnet_loaded) return COMPTON_ENOMODEL;
    compton_status st =
        compton::launch_pnet_train_step(ctx, ux, uy, uz, kx, ky, kz, y, w, n, w_e, w_g, p_max, lr, stream);
    if (st != COMPTON_OK || !loss_out_host) return st;
    float l[2];
    COMPTON_CUDA_TRY(ctx, cudaMemcpyAsync(l, ctx->pnet.loss, sizeof(l), cudaMemcpyDeviceToHost, stream));
    COMPTON_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    *loss_out_host = l[1] > 0.0f ? l[0] / l[1] : 0.0f;
    return COMPTON_OK;
}

compton_status compton_mlp_set_features(compton_ctx* ctx, int32_t features)
{
    if (!ctx) return COMPTON_EINVAL;
    if (features != COMPTON_FEATURES_MOMENTA && features != COMPTON_FEATURES_INVARIANTS) return COMPTON_EINVAL;
    ctx->mlp.feat_mode = features;
    return COMPTON_OK;
}

// ---------------------------------------------------------------------------
// Serving
// ---------------------------------------------------------------------------
compton_status compton_serve_start(compton_ctx* ctx, uint64_t pool_bytes, int32_t max_active)
{
    if (!ctx || pool_bytes < 4096 || max_active <= 0 || max_active > 65536) return COMPTON_EINVAL;
    if (ctx->serve) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaSetDevice(ctx->cfg.device));
    return compton::serve_start(ctx, pool_bytes, max_active);
}

compton_status compton_serve_stop(compton_ctx* ctx)
{
    if (!ctx) return COMPTON_EINVAL;
    return compton::serve_stop(ctx);
}

compton_status compton_submit(compton_ctx* ctx, const compton_request* r, uint64_t* ticket)
{
    if (!ctx || !r || !ticket || !ctx->serve) return COMPTON_EINVAL;
    if (r->n <= 0 || r->n > INT32_MAX) return COMPTON_EINVAL;
    if (!r->ux_in_dev || !r->uy_in_dev || !r->uz_in_dev || !r->kx_in_dev || !r->ky_in_dev || !r->kz_in_dev ||
        !r->ux_out_dev || !r->uy_out_dev || !r->uz_out_dev || !r->kx_out_dev || !r->ky_out_dev || !r->kz_out_dev)
        return COMPTON_EINVAL;
    if ((int)r->mode < 0 || (int)r->mode > 3) return COMPTON_EINVAL;
    if (!r->n_dens_dev && !(r->n_dens >= 0.0f)) return COMPTON_EINVAL;
    if (r->mode != COMPTON_MODE_PLAIN && !ctx->mlp_loaded) return COMPTON_ENOMODEL;
    return compton::serve_submit(ctx, r, ticket);
}

compton_status compton_poll(compton_ctx* ctx, uint64_t ticket, compton_result* out)
{
    if (!ctx || !out) return COMPTON_EINVAL;
    return compton::serve_poll(ctx, ticket, out);
}

compton_status compton_serve_info(compton_ctx* ctx, uint64_t* bytes_in_use, uint64_t* peak_bytes,
                                  uint64_t* pool_bytes)
{
    if (!ctx || !bytes_in_use || !peak_bytes || !pool_bytes) return COMPTON_EINVAL;
    return compton::serve_info(ctx, bytes_in_use, peak_bytes, pool_bytes);
}

compton_status compton_selftest_wait(compton_ctx* ctx, uint64_t timeout_ns, compton_stream_t stream)
{
    if (!ctx || timeout_ns == 0 || timeout_ns > 10000000000ull) return COMPTON_EINVAL;
    return compton::launch_selftest_wait(ctx, timeout_ns, stream);
}

compton_status compton_kn_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n,
                                       float* cth_out, float* sth_out, float* ratio_out, compton_stream_t stream)
{
    if (!ctx || n < 0) return COMPTON_EINVAL;
    if (n == 0) return COMPTON_OK;
    if (!x || !r || !cth_out || !sth_out || !ratio_out) return COMPTON_EINVAL;
    return compton::launch_sample_angle(ctx, x, r, n, cth_out, sth_out, ratio_out, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Host-side fault injection (test support).
// ---------------------------------------------------------------------------
namespace compton {
namespace {
std::mutex g_inject_mu;
std::atomic<int64_t> g_inject_fail{0};
int64_t g_inject_skip = 0;
}  // namespace

bool inject_fault()
{
    if (g_inject_fail.load(std::memory_order_relaxed) <= 0) return false;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_fail.load(std::memory_order_relaxed) <= 0) return false;
    if (g_inject_skip > 0) {
        --g_inject_skip;
        return false;
    }
    g_inject_fail.fetch_sub(1, std::memory_order_relaxed);
    return true;
}

void inject_arm(int64_t skip, int64_t fail)
{
    std::lock_guard<std::mutex> lk(g_inject_mu);
    g_inject_skip = skip > 0 ? skip : 0;
    g_inject_fail.store(fail > 0 ? fail : 0, std::memory_order_relaxed);
}
}  // namespace compton

compton_status compton_debug_inject(int64_t skip, int64_t fail, int64_t* pending_out)
{
    if (skip < 0 || fail < 0) return COMPTON_EINVAL;
    if (pending_out) *pending_out = compton::g_inject_fail.load();
    compton::inject_arm(skip, fail);
    return COMPTON_OK;
}
