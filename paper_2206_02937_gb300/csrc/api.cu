// api.cu -- the extern "C" entry points of libcompton: argument checking,
// context and arena management, status codes.  The kernels live in
// bin_pairs.cu and scatter.cu.
#include <cmath>
#include <cstdlib>
#include <new>

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
    const void* pa[5] = {a->ux_dev, a->uy_dev, a->uz_dev, a->cell_dev, a->id_dev};
    const void* pb[5] = {b->ux_dev, b->uy_dev, b->uz_dev, b->cell_dev, b->id_dev};
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j)
            if (overlaps(pa[i], pb[j], n, 4)) return true;
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
    compton_ctx* ctx = new (std::nothrow) compton_ctx();
    if (!ctx) return COMPTON_ENOMEM;
    ctx->cfg = *cfg;
    ctx->last_error[0] = '\0';
    cudaError_t e = cudaSetDevice(cfg->device);
    if (e != cudaSuccess) {
        delete ctx;
        return COMPTON_ECUDA;
    }
    const int64_t C = cfg->n_cells;
    const int64_t P = cfg->max_particles;
    ctx->max_scan_tiles = (C + compton::kScanTile - 1) / compton::kScanTile;
    ctx->max_sort_tiles = (P + compton::kSortTile - 1) / compton::kSortTile + 1;
    ctx->max_pair_tiles = (P + compton::kPairsPerTile - 1) / compton::kPairsPerTile + 1;

    Carver cv;
    size_t o_count[2], o_off[2], o_rec[2], o_stile[2];
    for (int s = 0; s < 2; ++s) {
        o_count[s] = cv.take<int32_t>(C);
        o_off[s] = cv.take<int32_t>(C + 1);
        o_rec[s] = cv.take<uint2>(P > 0 ? P : 1);
        o_stile[s] = cv.take<int32_t>(ctx->max_sort_tiles + 1);
    }
    size_t o_bs = cv.take<int64_t>(3 * ctx->max_scan_tiles);
    size_t o_ci = cv.take<CellInfo>(C);
    size_t o_tc = cv.take<int32_t>(ctx->max_pair_tiles + 1);
    size_t o_np = cv.take<int64_t>(1);
    size_t o_st = cv.take<compton::DeviceStats>(1);
    const size_t total = align_up(cv.used, 256);
    if (cfg->mem_budget_bytes && total > cfg->mem_budget_bytes) {
        delete ctx;
        return COMPTON_ENOMEM;
    }
    e = cudaMalloc(&ctx->arena, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return COMPTON_ENOMEM;
    }
    ctx->arena_bytes = total;
    char* base = static_cast<char*>(ctx->arena);
    for (int s = 0; s < 2; ++s) {
        ctx->count[s] = reinterpret_cast<int32_t*>(base + o_count[s]);
        ctx->off[s] = reinterpret_cast<int32_t*>(base + o_off[s]);
        ctx->rec[s] = reinterpret_cast<uint2*>(base + o_rec[s]);
        ctx->stile[s] = reinterpret_cast<int32_t*>(base + o_stile[s]);
    }
    ctx->block_sums = reinterpret_cast<int64_t*>(base + o_bs);
    ctx->cinfo = reinterpret_cast<CellInfo*>(base + o_ci);
    ctx->tile_cell = reinterpret_cast<int32_t*>(base + o_tc);
    ctx->n_pairs = reinterpret_cast<int64_t*>(base + o_np);
    ctx->stats = reinterpret_cast<compton::DeviceStats*>(base + o_st);
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
    cudaDeviceSynchronize();
    if (ctx->arena) cudaFree(ctx->arena);
    delete ctx;
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
        return COMPTON_ERANGE;
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
    if (species_alias(e_in, e_out, e_in->n) || species_alias(g_in, g_out, g_in->n)) return COMPTON_EINVAL;
    compton_status st = compton::launch_bin_pairs(ctx, e_in, g_in, e_out, g_out, step, stream);
    if (st != COMPTON_OK) return st;
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
    if (mode != COMPTON_MODE_PLAIN) return COMPTON_ENOMODEL;
    return compton::launch_scatter_binned(ctx, e, g, pairs, mode, step, prob_out, flag_out, stream);
}

compton_status compton_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                     float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                     compton_mode mode, float* prob_out, uint8_t* flag_out,
                                     compton_stream_t stream)
{
    if (!ctx || n < 0 || n > INT32_MAX) return COMPTON_EINVAL;
    if (n == 0) return COMPTON_OK;
    if (!ux || !uy || !uz || !kx || !ky || !kz || !n_dens) return COMPTON_EINVAL;
    if (mode != COMPTON_MODE_PLAIN) return COMPTON_ENOMODEL;
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

compton_status compton_kn_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n,
                                       float* cth_out, float* sth_out, float* ratio_out, compton_stream_t stream)
{
    if (!ctx || n < 0) return COMPTON_EINVAL;
    if (n == 0) return COMPTON_OK;
    if (!x || !r || !cth_out || !sth_out || !ratio_out) return COMPTON_EINVAL;
    return compton::launch_sample_angle(ctx, x, r, n, cth_out, sth_out, ratio_out, stream);
}

}  // extern "C"
