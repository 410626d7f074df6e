// scatter.cu -- probability, Bernoulli trial and collision of every pair
// (arXiv 2206.02937, Sec. 3.1: for each pair of the list the probability of
// interaction is computed and compared with a random number, and each pair
// deemed to collide has its kinetic collision resolved and its momenta
// updated; Sec. 3.2: the probability comes from the Klein-Nishina cross
// section in the lepton rest frame, carried back to the simulation frame).
//
// One fused, persistent kernel.  Each CTA walks tiles of 1024 pairs
// (256 threads x 4 pairs):
//   phase 1  every pair of the tile: locate its cell (binary search in the
//            tile's window of CellInfo records staged in shared memory), load
//            both momenta (coalesced: consecutive pairs are consecutive
//            sorted particles), form x and v, sigma_KN, P = 1 - exp(-n dt s v),
//            one Philox block, the Bernoulli decision; accepted pairs are
//            appended to a shared-memory queue that persists across tiles;
//   phase 2  whenever the queue holds at least 256 entries, all 256 threads
//            take one each: inverse-CDF angle in FP32, rest-frame boost and
//            momentum update in FP64, write-back of both momenta in place.
//            The last partial batch is drained after the final tile.
// Accepted pairs are a few percent of all pairs; batching them keeps the
// FP64 branch at full warp width instead of one live lane per warp.
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kScatterThreads = 256;
constexpr int kPairsPerThread = kPairsPerTile / kScatterThreads;
constexpr int kQueueCap = kPairsPerTile + kScatterThreads;

struct ScatterArgs {
    float* u[3];  // electron momenta (sorted species, or explicit pair list)
    float* k[3];  // photon momenta
    const CellInfo* cinfo;
    const int32_t* tile_cell;
    const int64_t* n_pairs;   // binned: device total
    const float* n_dens;      // explicit: density per pair
    int64_t n_explicit;       // explicit: pair count
    float dt;
    uint64_t seed, step;
    float gamma64;
    float collide64_sq;  // (gamma eps)^2 above which the collision runs in FP64
    float* prob_out;
    uint8_t* flag_out;
    DeviceStats* stats;
    const float* r_mlp;  // network output per pair (surrogate modes)
};

struct QEntry {
    int32_t ie, ig;
    float x, F2;
    uint32_t p;  // pair index: counter of its angle draws
    uint32_t pad;
};

__device__ __forceinline__ int find_cell(const CellInfo* win, int nwin, int64_t p)
{
    int lo = 0, hi = nwin - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)win[mid].pair_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void resolve(const ScatterArgs& a, const QEntry& e)
{
    float ux = a.u[0][e.ie], uy = a.u[1][e.ie], uz = a.u[2][e.ie];
    float kx = a.k[0][e.ig], ky = a.k[1][e.ig], kz = a.k[2][e.ig];
    float x = e.x, F2 = e.F2;
    if (x < 0.0f) {  // probability came from the network: the collision needs x and F(x, 2)
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        float v = inv.v;
        x = inv.x;
        if (inv.gamma > a.gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
        F2 = kn_F2(x);
    }
    const Philox4 rnd = draw(a.seed, a.step, kStreamAngle, e.p);
    const Angle ang = kn_sample_angle(x, rnd.r0 >> 8, F2);
    // FP64 where FP32 cancellation would exceed the tolerance (gamma eps large)
    const float ge2 = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, 1.0f))) * fmaf(kx, kx, fmaf(ky, ky, kz * kz));
    if (ge2 > a.collide64_sq) collide_f64(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(rnd.r1));
    else collide_f32(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(rnd.r1));
    a.u[0][e.ie] = ux;
    a.u[1][e.ie] = uy;
    a.u[2][e.ie] = uz;
    a.k[0][e.ig] = kx;
    a.k[1][e.ig] = ky;
    a.k[2][e.ig] = kz;
}

// kMlp: the probability of in-range pairs is P = 1 - exp(-2 n dt r) with r
// from the surrogate network (a.r_mlp, one value per pair); pairs outside the
// network's training range (gamma > 1e3, eps outside [1e-4, 1]) use the
// analytic probability and are counted as fallbacks.
template <bool kBinned, bool kMlp>
__global__ void __launch_bounds__(kScatterThreads, 3) k_scatter(ScatterArgs a)
{
    __shared__ CellInfo win[kCellWindow];
    __shared__ QEntry queue[kQueueCap];
    __shared__ int qn;
    __shared__ unsigned red_pairs, red_scat, red_fb;

    const int tid = threadIdx.x;
    const int64_t total = kBinned ? *a.n_pairs : a.n_explicit;
    const int64_t n_tiles = (total + kPairsPerTile - 1) / kPairsPerTile;
    if (tid == 0) {
        qn = 0;
        red_pairs = 0;
        red_scat = 0;
        red_fb = 0;
    }
    unsigned my_pairs = 0, my_scat = 0, my_fb = 0;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t p0 = tile * kPairsPerTile;
        int c_first = 0, nwin = 0;
        bool use_win = true;
        if (kBinned) {
            c_first = a.tile_cell[tile];
            const int c_last = a.tile_cell[tile + 1];
            nwin = c_last - c_first + 1;
            use_win = nwin <= kCellWindow;
            if (use_win)
                for (int i = tid; i < nwin; i += kScatterThreads) win[i] = a.cinfo[c_first + i];
        }
        __syncthreads();

        // ---------------- phase 1: every pair of the tile ----------------
        // Thread tid takes the 4 consecutive pairs p0 + 4 tid + r: one binary
        // search for the first, a forward step (usually none) for the others.
        int ie[kPairsPerThread], ig[kPairsPerThread];
        float dens[kPairsPerThread];
        bool valid[kPairsPerThread];
        const int64_t pb = p0 + (int64_t)tid * kPairsPerThread;
        const CellInfo* cw = use_win ? win : a.cinfo + c_first;
        int ci_idx = 0;
        if (kBinned && pb < total) ci_idx = find_cell(cw, nwin, pb);
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            const int64_t p = pb + r;
            valid[r] = p < total;
            ie[r] = 0;
            ig[r] = 0;
            dens[r] = 0.0f;
            if (valid[r]) {
                if (kBinned) {
                    while (ci_idx + 1 < nwin && (int64_t)cw[ci_idx + 1].pair_off <= p) ++ci_idx;
                    const CellInfo ci = cw[ci_idx];
                    const int j = (int)(p - ci.pair_off);
                    ie[r] = ci.e_start + j;
                    ig[r] = ci.g_start + j;
                    dens[r] = ci.dens;
                } else {
                    ie[r] = (int)p;
                    ig[r] = (int)p;
                    dens[r] = a.n_dens[p];
                }
            }
        }
        float ux[kPairsPerThread], uy[kPairsPerThread], uz[kPairsPerThread];
        float kx[kPairsPerThread], ky[kPairsPerThread], kz[kPairsPerThread];
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            if (valid[r]) {
                ux[r] = a.u[0][ie[r]];
                uy[r] = a.u[1][ie[r]];
                uz[r] = a.u[2][ie[r]];
                kx[r] = a.k[0][ig[r]];
                ky[r] = a.k[1][ig[r]];
                kz[r] = a.k[2][ig[r]];
            } else {
                ux[r] = uy[r] = uz[r] = kx[r] = ky[r] = kz[r] = 0.0f;
            }
        }
        // the Bernoulli uniforms of the thread's four pairs: one Philox block
        const Philox4 rnd4 = draw(a.seed, a.step, kStreamScatter, (uint32_t)(pb >> 2));
        const uint32_t words[4] = {rnd4.r0, rnd4.r1, rnd4.r2, rnd4.r3};
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            if (!valid[r]) continue;
            const int64_t p = pb + r;
            float x = -1.0f, F2 = 0.0f, P;
            bool analytic = true;
            if (kMlp) {
                const float g2 = fmaf(ux[r], ux[r], fmaf(uy[r], uy[r], fmaf(uz[r], uz[r], 1.0f)));
                const float e2 = fmaf(kx[r], kx[r], fmaf(ky[r], ky[r], kz[r] * kz[r]));
                if (g2 <= 1.0e6f && e2 >= 1.0e-8f && e2 <= 1.0f) {
                    analytic = false;
                    P = one_minus_exp_neg(2.0f * dens[r] * a.dt * a.r_mlp[p]);
                } else {
                    ++my_fb;
                }
            }
            if (analytic) {
                const Invariants inv = invariants_f32(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r]);
                float v = inv.v;
                x = inv.x;
                if (inv.gamma > a.gamma64) invariants_f64(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r], &x, &v);
                F2 = kn_F2(x);
                const float sig = 0.375f * F2;
                P = inv.eps > 0.0f ? one_minus_exp_neg(dens[r] * a.dt * sig * v) : 0.0f;
            }
            const bool hit = u24_closed0(words[r]) < P;
            if (a.prob_out) a.prob_out[p] = P;
            if (a.flag_out) a.flag_out[p] = hit ? 1 : 0;
            ++my_pairs;
            if (hit) {
                ++my_scat;
                const int slot = atomicAdd(&qn, 1);
                queue[slot] = QEntry{ie[r], ig[r], x, F2, (uint32_t)p, 0u};
            }
        }
        __syncthreads();

        // ---------------- phase 2: full batches of accepted pairs ----------------
        int nq = qn;
        while (nq >= kScatterThreads) {
            resolve(a, queue[nq - kScatterThreads + tid]);
            nq -= kScatterThreads;
        }
        __syncthreads();
        if (tid == 0) qn = nq;
    }
    __syncthreads();
    if (tid < qn) resolve(a, queue[tid]);

    // ---------------- counters ----------------
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, d);
        my_scat += __shfl_xor_sync(0xffffffffu, my_scat, d);
        my_fb += __shfl_xor_sync(0xffffffffu, my_fb, d);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&red_pairs, my_pairs);
        atomicAdd(&red_scat, my_scat);
        atomicAdd(&red_fb, my_fb);
    }
    __syncthreads();
    if (tid == 0 && red_pairs) {
        atomicAdd(&a.stats->pairs_tested, (unsigned long long)red_pairs);
        atomicAdd(&a.stats->scatters, (unsigned long long)red_scat);
        if (red_fb) atomicAdd(&a.stats->mlp_fallbacks, (unsigned long long)red_fb);
    }
}

// r = s(x) v / 2 per explicit pair.
__global__ void k_kn_ratio(const float* __restrict__ ux, const float* __restrict__ uy, const float* __restrict__ uz,
                           const float* __restrict__ kx, const float* __restrict__ ky, const float* __restrict__ kz,
                           int64_t n, float gamma64, float* __restrict__ r_out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float a0 = ux[i], a1 = uy[i], a2 = uz[i], b0 = kx[i], b1 = ky[i], b2 = kz[i];
        const Invariants inv = invariants_f32(a0, a1, a2, b0, b1, b2);
        float x = inv.x, v = inv.v;
        if (inv.gamma > gamma64) invariants_f64(a0, a1, a2, b0, b1, b2, &x, &v);
        r_out[i] = inv.eps > 0.0f ? 0.5f * kn_sigma(x) * v : 0.0f;
    }
}

__global__ void k_sample_angle(const float* __restrict__ x, const uint32_t* __restrict__ r, int64_t n,
                               float* __restrict__ cth, float* __restrict__ sth, float* __restrict__ ratio)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float xi = x[i];
        const Angle ang = kn_sample_angle(xi, r[i] >> 8, kn_F2(xi));  // r: a raw angle word
        cth[i] = ang.cth;
        sth[i] = ang.sth;
        ratio[i] = ang.ratio;
    }
}

template <bool kBinned, bool kMlp>
int persistent_grid(int64_t max_pairs)
{
    static int per_sm = 0, n_sm = 0;
    if (per_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<kBinned, kMlp>, kScatterThreads, 0);
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t tiles = (max_pairs + kPairsPerTile - 1) / kPairsPerTile;
    const int64_t full = (int64_t)per_sm * n_sm;
    return (int)(tiles < full ? tiles : full);
}

}  // namespace

compton_status launch_scatter_binned(compton_ctx* ctx, compton_species* e, compton_species* g,
                                     const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                     float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    if (pairs->max_pairs <= 0) return COMPTON_OK;
    const bool mlp = mode != COMPTON_MODE_PLAIN;
    if (mlp) {
        compton_status st = launch_mlp_infer(ctx, e->ux_dev, e->uy_dev, e->uz_dev, g->ux_dev, g->uy_dev, g->uz_dev,
                                             pairs->max_pairs, mode, ctx->r_buf, stream, true);
        if (st != COMPTON_OK) return st;
    }
    ScatterArgs a;
    a.u[0] = e->ux_dev;
    a.u[1] = e->uy_dev;
    a.u[2] = e->uz_dev;
    a.k[0] = g->ux_dev;
    a.k[1] = g->uy_dev;
    a.k[2] = g->uz_dev;
    a.cinfo = ctx->cinfo;
    a.tile_cell = ctx->tile_cell;
    a.n_pairs = ctx->n_pairs;
    a.n_dens = nullptr;
    a.n_explicit = 0;
    a.dt = (float)ctx->cfg.dt;
    a.seed = ctx->cfg.seed;
    a.step = step;
    a.gamma64 = ctx->cfg.gamma_fp64_threshold;
    a.collide64_sq = ctx->cfg.collide_fp64_threshold * ctx->cfg.collide_fp64_threshold;
    a.prob_out = prob_out;
    a.flag_out = flag_out;
    a.stats = ctx->stats;
    a.r_mlp = ctx->r_buf;
    if (mlp) k_scatter<true, true><<<persistent_grid<true, true>(pairs->max_pairs), kScatterThreads, 0, stream>>>(a);
    else k_scatter<true, false><<<persistent_grid<true, false>(pairs->max_pairs), kScatterThreads, 0, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_scatter<binned>");
    return COMPTON_OK;
}

compton_status launch_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                    float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                    compton_mode mode, float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    const bool mlp = mode != COMPTON_MODE_PLAIN;
    if (mlp) {
        if (n > ctx->cfg.max_particles) return COMPTON_ERANGE;
        compton_status st = launch_mlp_infer(ctx, ux, uy, uz, kx, ky, kz, n, mode, ctx->r_buf, stream, false);
        if (st != COMPTON_OK) return st;
    }
    ScatterArgs a;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.cinfo = nullptr;
    a.tile_cell = nullptr;
    a.n_pairs = nullptr;
    a.n_dens = n_dens;
    a.n_explicit = n;
    a.dt = (float)ctx->cfg.dt;
    a.seed = seed;
    a.step = step;
    a.gamma64 = ctx->cfg.gamma_fp64_threshold;
    a.collide64_sq = ctx->cfg.collide_fp64_threshold * ctx->cfg.collide_fp64_threshold;
    a.prob_out = prob_out;
    a.flag_out = flag_out;
    a.stats = ctx->stats;
    a.r_mlp = ctx->r_buf;
    if (mlp) k_scatter<false, true><<<persistent_grid<false, true>(n), kScatterThreads, 0, stream>>>(a);
    else k_scatter<false, false><<<persistent_grid<false, false>(n), kScatterThreads, 0, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_scatter<pairs>");
    return COMPTON_OK;
}

compton_status launch_kn_ratio(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                               const float* kx, const float* ky, const float* kz, int64_t n, float* r_out,
                               cudaStream_t stream)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_kn_ratio<<<(unsigned)blocks, 256, 0, stream>>>(ux, uy, uz, kx, ky, kz, n, ctx->cfg.gamma_fp64_threshold,
                                                     r_out);
    COMPTON_LAUNCH_CHECK(ctx, "k_kn_ratio");
    return COMPTON_OK;
}

compton_status launch_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n, float* cth,
                                   float* sth, float* ratio, cudaStream_t stream)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_sample_angle<<<(unsigned)blocks, 256, 0, stream>>>(x, r, n, cth, sth, ratio);
    COMPTON_LAUNCH_CHECK(ctx, "k_sample_angle");
    return COMPTON_OK;
}

}  // namespace compton
