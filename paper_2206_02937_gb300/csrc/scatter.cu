// scatter.cu -- probability, Bernoulli trial and collision of every pair
// (arXiv 2206.02937, Sec. 3.1: for each pair of the list the probability of
// interaction is computed and compared with a random number, and each pair
// deemed to collide has its kinetic collision resolved and its momenta
// updated; Sec. 3.2: the probability comes from the Klein-Nishina cross
// section in the lepton rest frame, carried back to the simulation frame).
//
// One fused, persistent kernel, software-pipelined over the tiles of 1024
// pairs (256 threads x 4 consecutive pairs) that a CTA owns:
//   * while tile t is computed, the particle data of tile t + G (G = grid
//     size) is already in flight to shared memory (cp.async), and so is the
//     window of CellInfo records of tile t + 2G: the loads of a tile never
//     sit on the critical path of its own arithmetic;
//   phase 1  every pair of tile t, from shared memory: x and v, sigma_KN,
//            P = 1 - exp(-n dt s v), one Philox block per four pairs, the
//            Bernoulli decision; accepted pairs are appended to a
//            shared-memory queue that persists across tiles;
//   phase 2  whenever the queue holds at least 256 entries, all 256 threads
//            take one each: inverse-CDF angle, rest-frame boost and momentum
//            update (FP32, or FP64 above the configured gamma eps), write-back
//            of both momenta in place.  The last partial batch is drained
//            after the final tile.
// Accepted pairs are a few percent of all pairs; batching them keeps the
// collision branch at full warp width instead of one live lane per warp.
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kScatterThreads = 256;
constexpr int kPairsPerThread = kPairsPerTile / kScatterThreads;
constexpr int kQueueCap = kPairsPerTile + kScatterThreads;
constexpr int kSlots = 8;  // staged per pair: ux uy uz kx ky kz, density (explicit pairs), network output

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

// A pair accepted in phase 1 and waiting for its collision.  x < 0 marks a
// pair whose probability came from the network (x is then recomputed).
struct QEntry {
    int32_t ie, ig;
    float x;
    uint32_t p;  // pair index: counter of its angle draws
};

struct ScatterSmem {
    float* stage[2];   // [kSlots][kPairsPerTile] each
    CellInfo* win[2];  // [kCellWindow] each
    QEntry* queue;     // [kQueueCap]
};
constexpr size_t kStageBytes = sizeof(float) * kSlots * kPairsPerTile;
constexpr size_t kScatterSmem = 2 * kStageBytes + 2 * sizeof(CellInfo) * kCellWindow + sizeof(QEntry) * kQueueCap;

__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int find_cell(const CellInfo* win, int nwin, int64_t p)
{
    int lo = 0, hi = nwin - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)win[mid].pair_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Where the four pairs of one thread in one tile live.
struct PairLoc {
    int32_t ie[kPairsPerThread], ig[kPairsPerThread];
    float dens[kPairsPerThread];  // binned: the cell's density
};

// First and last cell of a binned tile.
struct TileCells {
    int32_t first, last;
};

__device__ __forceinline__ TileCells tile_cells(const ScatterArgs& a, int64_t tile)
{
    return TileCells{a.tile_cell[tile], a.tile_cell[tile + 1]};
}

// Window of CellInfo records of a tile to shared memory (when it fits).
__device__ __forceinline__ void issue_window(const ScatterArgs& a, CellInfo* win, TileCells tc)
{
    const int nwin = tc.last - tc.first + 1;
    if (nwin > kCellWindow) return;
    for (int i = threadIdx.x; i < nwin; i += kScatterThreads) cp_async16(&win[i], &a.cinfo[tc.first + i]);
}

template <bool kBinned>
__device__ __forceinline__ PairLoc locate(const ScatterArgs& a, const CellInfo* win, TileCells tc, int64_t pb,
                                          int64_t total)
{
    PairLoc L;
    if (!kBinned) {
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            L.ie[r] = (int32_t)(pb + r);
            L.ig[r] = (int32_t)(pb + r);
            L.dens[r] = 0.0f;
        }
        return L;
    }
    const int nwin = tc.last - tc.first + 1;
    const CellInfo* cw = nwin <= kCellWindow ? win : a.cinfo + tc.first;
    int ci_idx = pb < total ? find_cell(cw, nwin, pb) : 0;
#pragma unroll
    for (int r = 0; r < kPairsPerThread; ++r) {
        const int64_t p = pb + r;
        L.ie[r] = 0;
        L.ig[r] = 0;
        L.dens[r] = 0.0f;
        if (p < total) {
            while (ci_idx + 1 < nwin && (int64_t)cw[ci_idx + 1].pair_off <= p) ++ci_idx;
            const CellInfo ci = cw[ci_idx];
            const int j = (int)(p - ci.pair_off);
            L.ie[r] = ci.e_start + j;
            L.ig[r] = ci.g_start + j;
            L.dens[r] = ci.dens;
        }
    }
    return L;
}

// Four values of one array at indices i0..i3 to st[4 tid .. 4 tid + 3]: one
// 16-byte copy when they are consecutive and aligned, else one per value.
__device__ __forceinline__ void stage4(float* st, const float* src, int32_t i0, int32_t i1, int32_t i2, int32_t i3,
                                       int nvalid)
{
    if (nvalid == kPairsPerThread && i3 == i0 + 3 && ((reinterpret_cast<uintptr_t>(src + i0) & 15u) == 0)) {
        cp_async16(st, src + i0);
        return;
    }
    cp_async4(st, src + i0);
    if (nvalid > 1) cp_async4(st + 1, src + i1);
    if (nvalid > 2) cp_async4(st + 2, src + i2);
    if (nvalid > 3) cp_async4(st + 3, src + i3);
}

template <bool kBinned, bool kMlp>
__device__ __forceinline__ void issue_pairs(const ScatterArgs& a, float* stage, const PairLoc& L, int64_t pb,
                                            int64_t total)
{
    const int64_t left = total - pb;
    const int nvalid = left <= 0 ? 0 : (left >= kPairsPerThread ? kPairsPerThread : (int)left);
    if (nvalid == 0) return;
    const int o = kPairsPerThread * threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        stage4(stage + c * kPairsPerTile + o, a.u[c], L.ie[0], L.ie[1], L.ie[2], L.ie[3], nvalid);
        stage4(stage + (3 + c) * kPairsPerTile + o, a.k[c], L.ig[0], L.ig[1], L.ig[2], L.ig[3], nvalid);
    }
    const int32_t p0 = (int32_t)pb;
    if (!kBinned) stage4(stage + 6 * kPairsPerTile + o, a.n_dens, p0, p0 + 1, p0 + 2, p0 + 3, nvalid);
    if (kMlp) stage4(stage + 7 * kPairsPerTile + o, a.r_mlp, p0, p0 + 1, p0 + 2, p0 + 3, nvalid);
}

__device__ __forceinline__ void resolve(const ScatterArgs& a, const QEntry& e)
{
    float ux = a.u[0][e.ie], uy = a.u[1][e.ie], uz = a.u[2][e.ie];
    float kx = a.k[0][e.ig], ky = a.k[1][e.ig], kz = a.k[2][e.ig];
    float x = e.x;
    if (x < 0.0f) {  // probability came from the network: the collision needs x
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        float v = inv.v;
        x = inv.x;
        if (inv.gamma > a.gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
    }
    const float F2 = kn_F2(x);
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
__global__ void __launch_bounds__(kScatterThreads, 2) k_scatter(ScatterArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem sm;
    sm.stage[0] = reinterpret_cast<float*>(smem_raw);
    sm.stage[1] = sm.stage[0] + kSlots * kPairsPerTile;
    sm.win[0] = reinterpret_cast<CellInfo*>(sm.stage[1] + kSlots * kPairsPerTile);
    sm.win[1] = sm.win[0] + kCellWindow;
    sm.queue = reinterpret_cast<QEntry*>(sm.win[1] + kCellWindow);
    __shared__ int qn;
    __shared__ unsigned red_pairs, red_scat, red_fb;

    const int tid = threadIdx.x;
    const int64_t total = kBinned ? *a.n_pairs : a.n_explicit;
    const int64_t n_tiles = (total + kPairsPerTile - 1) / kPairsPerTile;
    const int64_t G = gridDim.x;
    if (tid == 0) {
        qn = 0;
        red_pairs = 0;
        red_scat = 0;
        red_fb = 0;
    }
    unsigned my_pairs = 0, my_scat = 0, my_fb = 0;

    // prologue: window of the first tile, then its pairs and the second window
    int64_t tile = blockIdx.x;
    TileCells tc_next{0, 0}, tc_next2{0, 0};
    PairLoc nx{};
    if (tile < n_tiles) {
        if (kBinned) {
            tc_next = tile_cells(a, tile);
            issue_window(a, sm.win[0], tc_next);
            cp_async_commit();
            cp_async_wait_all();
        }
        __syncthreads();
        const int64_t pb = tile * kPairsPerTile + (int64_t)tid * kPairsPerThread;
        nx = locate<kBinned>(a, sm.win[0], tc_next, pb, total);
        issue_pairs<kBinned, kMlp>(a, sm.stage[0], nx, pb, total);
        if (kBinned && tile + G < n_tiles) {
            tc_next2 = tile_cells(a, tile + G);
            issue_window(a, sm.win[1], tc_next2);
        }
        cp_async_commit();
    }

    for (int buf = 0; tile < n_tiles; tile += G, buf ^= 1) {
        const PairLoc cur = nx;
        const int64_t pb = tile * kPairsPerTile + (int64_t)tid * kPairsPerThread;
        cp_async_wait_all();
        __syncthreads();  // stage[buf] holds this tile, win[buf ^ 1] the next tile's window

        // ---------------- prefetch: next tile's pairs, window after it ----------------
        const int64_t tn = tile + G;
        if (tn < n_tiles) {
            const int64_t pbn = tn * kPairsPerTile + (int64_t)tid * kPairsPerThread;
            nx = locate<kBinned>(a, sm.win[buf ^ 1], tc_next2, pbn, total);
            issue_pairs<kBinned, kMlp>(a, sm.stage[buf ^ 1], nx, pbn, total);
            if (kBinned && tn + G < n_tiles) {
                tc_next2 = tile_cells(a, tn + G);
                issue_window(a, sm.win[buf], tc_next2);
            }
        }
        cp_async_commit();

        // ---------------- phase 1: every pair of the tile ----------------
        const float* st = sm.stage[buf];
        const int o = kPairsPerThread * tid;
        const float4 vux = *reinterpret_cast<const float4*>(st + 0 * kPairsPerTile + o);
        const float4 vuy = *reinterpret_cast<const float4*>(st + 1 * kPairsPerTile + o);
        const float4 vuz = *reinterpret_cast<const float4*>(st + 2 * kPairsPerTile + o);
        const float4 vkx = *reinterpret_cast<const float4*>(st + 3 * kPairsPerTile + o);
        const float4 vky = *reinterpret_cast<const float4*>(st + 4 * kPairsPerTile + o);
        const float4 vkz = *reinterpret_cast<const float4*>(st + 5 * kPairsPerTile + o);
        const float ux[4] = {vux.x, vux.y, vux.z, vux.w}, uy[4] = {vuy.x, vuy.y, vuy.z, vuy.w};
        const float uz[4] = {vuz.x, vuz.y, vuz.z, vuz.w}, kx[4] = {vkx.x, vkx.y, vkx.z, vkx.w};
        const float ky[4] = {vky.x, vky.y, vky.z, vky.w}, kz[4] = {vkz.x, vkz.y, vkz.z, vkz.w};
        // the Bernoulli uniforms of the thread's four pairs: one Philox block
        const Philox4 rnd4 = draw(a.seed, a.step, kStreamScatter, (uint32_t)(pb >> 2));
        const uint32_t words[4] = {rnd4.r0, rnd4.r1, rnd4.r2, rnd4.r3};
        float P[kPairsPerThread], xq[kPairsPerThread];
        if (!kMlp) {
            // common path, straight-line for all four pairs: FP32 invariants,
            // series sigma_KN, probability
            bool rare[kPairsPerThread];
#pragma unroll
            for (int r = 0; r < kPairsPerThread; ++r) {
                const float dens = kBinned ? cur.dens[r] : st[6 * kPairsPerTile + o + r];
                const Invariants inv = invariants_f32(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r]);
                xq[r] = inv.x;
                const float F2 = kn_F2_series(fminf(inv.x, 0.99f));
                const float Pr = one_minus_exp_neg(dens * a.dt * 0.375f * F2 * inv.v);
                P[r] = inv.eps > 0.0f ? Pr : 0.0f;
                rare[r] = (inv.gamma > a.gamma64 || !(inv.x < 0.99f)) && pb + r < total;
            }
            // rare pairs: FP64 invariants above the gamma threshold, closed-form
            // sigma_KN above the series range
#pragma unroll
            for (int r = 0; r < kPairsPerThread; ++r) {
                if (!rare[r]) continue;
                const float dens = kBinned ? cur.dens[r] : st[6 * kPairsPerTile + o + r];
                const Invariants inv = invariants_f32(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r]);
                float x = inv.x, v = inv.v;
                if (inv.gamma > a.gamma64) invariants_f64(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r], &x, &v);
                xq[r] = x;
                P[r] = inv.eps > 0.0f ? one_minus_exp_neg(dens * a.dt * 0.375f * kn_F2(x) * v) : 0.0f;
            }
        } else {
#pragma unroll
            for (int r = 0; r < kPairsPerThread; ++r) {
                if (pb + r >= total) continue;
                const float dens = kBinned ? cur.dens[r] : st[6 * kPairsPerTile + o + r];
                const float g2 = fmaf(ux[r], ux[r], fmaf(uy[r], uy[r], fmaf(uz[r], uz[r], 1.0f)));
                const float e2 = fmaf(kx[r], kx[r], fmaf(ky[r], ky[r], kz[r] * kz[r]));
                if (g2 <= 1.0e6f && e2 >= 1.0e-8f && e2 <= 1.0f) {
                    xq[r] = -1.0f;
                    P[r] = one_minus_exp_neg(2.0f * dens * a.dt * st[7 * kPairsPerTile + o + r]);
                } else {
                    ++my_fb;
                    const Invariants inv = invariants_f32(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r]);
                    float x = inv.x, v = inv.v;
                    if (inv.gamma > a.gamma64) invariants_f64(ux[r], uy[r], uz[r], kx[r], ky[r], kz[r], &x, &v);
                    xq[r] = x;
                    P[r] = inv.eps > 0.0f ? one_minus_exp_neg(dens * a.dt * 0.375f * kn_F2(x) * v) : 0.0f;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            const int64_t p = pb + r;
            if (p >= total) continue;
            const bool hit = u24_closed0(words[r]) < P[r];
            if (a.prob_out) a.prob_out[p] = P[r];
            if (a.flag_out) a.flag_out[p] = hit ? 1 : 0;
            ++my_pairs;
            if (hit) {
                ++my_scat;
                const int slot = atomicAdd(&qn, 1);
                sm.queue[slot] = QEntry{cur.ie[r], cur.ig[r], xq[r], (uint32_t)p};
            }
        }
        __syncthreads();

        // ---------------- phase 2: full batches of accepted pairs ----------------
        int nq = qn;
        while (nq >= kScatterThreads) {
            resolve(a, sm.queue[nq - kScatterThreads + tid]);
            nq -= kScatterThreads;
        }
        __syncthreads();
        if (tid == 0) qn = nq;
    }
    cp_async_wait_all();
    __syncthreads();
    if (tid < qn) resolve(a, sm.queue[tid]);

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

// Persistent grid: every CTA that fits on the SMs at once (the kernel's
// dynamic shared memory is set on each call, so any current device works),
// capped by the tile count.  Returns 0 if the attributes cannot be set.
template <bool kBinned, bool kMlp>
int persistent_grid(int64_t max_pairs)
{
    const void* kern = (const void*)k_scatter<kBinned, kMlp>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return 0;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScatterThreads, kScatterSmem) != cudaSuccess)
        per_sm = 1;
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = (max_pairs + kPairsPerTile - 1) / kPairsPerTile;
    const int64_t full = (int64_t)per_sm * n_sm;
    return (int)(tiles < 1 ? 1 : (tiles < full ? tiles : full));
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
    const int grid = mlp ? persistent_grid<true, true>(pairs->max_pairs) : persistent_grid<true, false>(pairs->max_pairs);
    if (grid == 0) return set_cuda_error(ctx, cudaGetLastError(), "k_scatter<binned> attributes");
    if (mlp) k_scatter<true, true><<<grid, kScatterThreads, kScatterSmem, stream>>>(a);
    else k_scatter<true, false><<<grid, kScatterThreads, kScatterSmem, stream>>>(a);
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
    const int grid = mlp ? persistent_grid<false, true>(n) : persistent_grid<false, false>(n);
    if (grid == 0) return set_cuda_error(ctx, cudaGetLastError(), "k_scatter<pairs> attributes");
    if (mlp) k_scatter<false, true><<<grid, kScatterThreads, kScatterSmem, stream>>>(a);
    else k_scatter<false, false><<<grid, kScatterThreads, kScatterSmem, stream>>>(a);
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
