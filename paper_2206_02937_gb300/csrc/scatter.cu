// scatter.cu -- probability, Bernoulli trial and collision of every pair
// (arXiv 2206.02937, Sec. 3.1: "for each pair in this list, the probability
// of interaction is then calculated and compared against a random number ...
// for each pair deemed to collide, the kinetic collision is resolved and the
// momentum of the particles is updated"; Sec. 3.2: the probability comes from
// the Klein-Nishina cross section in the lepton rest frame, carried back to
// the simulation frame).
//
// One fused kernel, one CTA per tile of 1024 pairs (256 threads x 4 pairs):
//   phase 1  every pair: locate its cell (binary search in the tile's window
//            of CellInfo records staged in shared memory), load the two
//            momenta (coalesced: consecutive pairs are consecutive sorted
//            particles), form x and v, sigma_KN, P = 1 - exp(-n dt s v), one
//            Philox block, the Bernoulli decision; accepted pairs are
//            appended to a shared-memory queue;
//   phase 2  the queue is drained by all threads at full warp occupancy:
//            inverse-CDF angle in FP32, rest-frame boost and momentum update
//            in FP64, write-back of both momenta in place.
// Accepted pairs are a few percent of all pairs, so compacting them keeps the
// expensive branch from running with one live lane per warp.
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kScatterThreads = 256;
constexpr int kPairsPerThread = kPairsPerTile / kScatterThreads;

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
    float* prob_out;
    uint8_t* flag_out;
    DeviceStats* stats;
};

struct QEntry {
    int32_t ie, ig;
    float x, F2, u1, u2;
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

template <bool kBinned>
__global__ void __launch_bounds__(kScatterThreads) k_scatter(ScatterArgs a)
{
    __shared__ CellInfo win[kCellWindow];
    __shared__ QEntry queue[kPairsPerTile];
    __shared__ int qn;
    __shared__ unsigned red_pairs, red_scat;

    const int64_t total = kBinned ? *a.n_pairs : a.n_explicit;
    const int64_t p0 = (int64_t)blockIdx.x * kPairsPerTile;
    if (p0 >= total) return;
    const int tid = threadIdx.x;

    int c_first = 0, nwin = 0;
    bool use_win = true;
    if (kBinned) {
        c_first = a.tile_cell[blockIdx.x];
        const int c_last = a.tile_cell[blockIdx.x + 1];
        nwin = c_last - c_first + 1;
        use_win = nwin <= kCellWindow;
        if (use_win)
            for (int i = tid; i < nwin; i += kScatterThreads) win[i] = a.cinfo[c_first + i];
    }
    if (tid == 0) {
        qn = 0;
        red_pairs = 0;
        red_scat = 0;
    }
    __syncthreads();

    // ---------------- phase 1: every pair ----------------
    int ie[kPairsPerThread], ig[kPairsPerThread];
    float dens[kPairsPerThread];
    bool valid[kPairsPerThread];
#pragma unroll
    for (int r = 0; r < kPairsPerThread; ++r) {
        const int64_t p = p0 + r * kScatterThreads + tid;
        valid[r] = p < total;
        ie[r] = 0;
        ig[r] = 0;
        dens[r] = 0.0f;
        if (valid[r]) {
            if (kBinned) {
                CellInfo ci;
                if (use_win) {
                    ci = win[find_cell(win, nwin, p)];
                } else {
                    ci = a.cinfo[c_first + find_cell(a.cinfo + c_first, nwin, p)];
                }
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
    unsigned my_pairs = 0, my_scat = 0;
#pragma unroll
    for (int r = 0; r < kPairsPerThread; ++r) {
        if (!valid[r]) continue;
        const int64_t p = p0 + r * kScatterThreads + tid;
        const Invariants inv = invariants_f32(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r]);
        float x = inv.x, v = inv.v;
        if (inv.gamma > a.gamma64) invariants_f64(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r], &x, &v);
        const float F2 = kn_F(x, 2.0f);
        const float sig = 0.375f * F2;
        const float P = inv.eps > 0.0f ? -expm1f(-(dens[r] * a.dt * sig * v)) : 0.0f;
        const Philox4 rnd = draw(a.seed, a.step, kStreamScatter, (uint32_t)p);
        const bool hit = u24_closed0(rnd.r0) < P;
        if (a.prob_out) a.prob_out[p] = P;
        if (a.flag_out) a.flag_out[p] = hit ? 1 : 0;
        ++my_pairs;
        if (hit) {
            ++my_scat;
            const int slot = atomicAdd(&qn, 1);
            queue[slot] = QEntry{ie[r], ig[r], x, F2, u24_open(rnd.r1), u24_closed0(rnd.r2)};
        }
    }
    __syncthreads();

    // ---------------- phase 2: accepted pairs only ----------------
    const int nq = qn;
    for (int q = tid; q < nq; q += kScatterThreads) {
        const QEntry e = queue[q];
        float eux = a.u[0][e.ie], euy = a.u[1][e.ie], euz = a.u[2][e.ie];
        float gkx = a.k[0][e.ig], gky = a.k[1][e.ig], gkz = a.k[2][e.ig];
        const float t = kn_sample_t(e.x, e.u1, e.F2);
        collide_f64(eux, euy, euz, gkx, gky, gkz, e.x, t, e.u2);
        a.u[0][e.ie] = eux;
        a.u[1][e.ie] = euy;
        a.u[2][e.ie] = euz;
        a.k[0][e.ig] = gkx;
        a.k[1][e.ig] = gky;
        a.k[2][e.ig] = gkz;
    }

    // ---------------- counters ----------------
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, d);
        my_scat += __shfl_xor_sync(0xffffffffu, my_scat, d);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&red_pairs, my_pairs);
        atomicAdd(&red_scat, my_scat);
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.stats->pairs_tested, (unsigned long long)red_pairs);
        atomicAdd(&a.stats->scatters, (unsigned long long)red_scat);
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

}  // namespace

compton_status launch_scatter_binned(compton_ctx* ctx, compton_species* e, compton_species* g,
                                     const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                     float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    (void)mode;
    if (pairs->max_pairs <= 0) return COMPTON_OK;
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
    a.prob_out = prob_out;
    a.flag_out = flag_out;
    a.stats = ctx->stats;
    const int64_t tiles = (pairs->max_pairs + kPairsPerTile - 1) / kPairsPerTile;
    k_scatter<true><<<(unsigned)tiles, kScatterThreads, 0, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_scatter<binned>");
    return COMPTON_OK;
}

compton_status launch_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                    float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                    compton_mode mode, float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    (void)mode;
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
    a.prob_out = prob_out;
    a.flag_out = flag_out;
    a.stats = ctx->stats;
    const int64_t tiles = (n + kPairsPerTile - 1) / kPairsPerTile;
    k_scatter<false><<<(unsigned)tiles, kScatterThreads, 0, stream>>>(a);
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

}  // namespace compton
