// scatter.cu -- probability, Bernoulli trial and collision of every pair
// (arXiv 2206.02937, Sec. 3.1: for each pair of the list the probability of
// interaction is computed and compared with a random number, and each pair
// deemed to collide has its kinetic collision resolved and its momenta
// updated; Sec. 3.2: the probability comes from the Klein-Nishina cross
// section in the lepton rest frame, carried back to the simulation frame).
//
// Two kernels per step:
//   k_pair_prob  persistent CTAs (four per SM) of eight independent warps:
//                each warp owns a contiguous run of 128-pair chunks (32 lanes
//                x 4 consecutive pairs, one Philox block per lane for the
//                four Bernoulli uniforms), stages the current pair tile's
//                cells and a per-pair cell map in its own shared-memory
//                window, and queues the pairs whose uniform lies below the
//                probability bound (candidates, about a tenth); candidates
//                are evaluated 32 at a time, one per lane: straight-line FP32
//                (x and v without cancellation, sigma_KN from its series or
//                its closed form above x = 1, 1 - exp(-n dt s v)); the rare
//                candidates above the FP64 gamma threshold are decided after
//                the warp's last chunk.  Accepted pairs go to the warp's own
//                region of the list.  No CTA-wide barrier, no shared counter.
//   k_collide_regions (plain mode) / k_collide (surrogate modes)
//                every accepted pair (a few percent of all pairs) at full
//                warp width: inverse-CDF angle, rest-frame boost and momentum
//                update (FP32, or FP64 above the configured gamma eps),
//                write-back of both momenta in place.
// Every draw is keyed by the pair index, so the order of the list does not
// change any result.
#include <type_traits>

#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kProbThreads = 256;
constexpr int kPairsPerThread = kPairsPerTile / kProbThreads;

struct ScatterArgs {
    float* u[3];  // electron momenta (sorted species, or explicit pair list)
    float* k[3];  // photon momenta
    const CellInfo* cinfo;
    const int32_t* tile_cell;
    const int64_t* n_pairs;   // binned: device total
    const float* n_dens;      // explicit: density per pair
    int64_t p_begin, p_end;   // explicit: the pairs of this launch
    float dt;
    uint64_t seed, step;
    float gamma64;
    float collide64_sq;  // (gamma eps)^2 above which the collision runs in FP64
    float* prob_out;
    uint8_t* flag_out;
    DeviceStats* stats;
    const float* r_mlp;  // network output per pair (surrogate modes)
    AcceptedPair* accepted;
    uint32_t* n_accepted;
    // plain mode: each probability warp appends its accepted pairs to its own
    // region of the list (from its first pair index on) and leaves the count
    // in warp_acc[warp]; the collision kernel walks the regions
    uint32_t* warp_acc;
    CandPair* cand_rare;  // plain mode: the rare candidates of each warp's region
    CandPair* cand;
    uint32_t* n_cand;
    MlpDev mlp;  // the network's training range (surrogate modes)
    // unequal weights: per-particle weights (nullptr: w_const for all) of the
    // sorted species; cinfo.dens then holds max(N_e, N_g)
    const float* w_e;
    const float* w_g;
    float w_const;
    bool weighted;
};

// A binned pair's density: the cell's, or with unequal weights the cell's
// larger count times the pair's heavier weight.
template <bool kWeighted>
__device__ __forceinline__ float pair_density(const ScatterArgs& a, float cell_dens, int ie, int ig)
{
    if (!kWeighted) return cell_dens;
    const float we = a.w_e ? a.w_e[ie] : a.w_const;
    const float wg = a.w_g ? a.w_g[ig] : a.w_const;
    return cell_dens * fmaxf(we, wg);
}

__device__ __forceinline__ int find_cell(const CellInfo* win, int nwin, int64_t p)
{
    int lo = 0, hi = nwin - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)win[mid].pair_off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The collision of one accepted pair, written back in place.
__device__ __forceinline__ void resolve(const ScatterArgs& a, const AcceptedPair& e)
{
    float ux = e.u[0], uy = e.u[1], uz = e.u[2];
    float kx = e.k[0], ky = e.k[1], kz = e.k[2];
    float x = e.x;
    if (x < 0.0f) {  // probability came from the network: the collision needs x
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        float v = inv.v;
        x = inv.x;
        if (inv.gamma > a.gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
    }
    // sigma_KN's integral, as the probability kernel computed it (kept in the
    // entry's first spare word; zero from the other producers)
    const float F2 = e.pad[0] ? __uint_as_float(e.pad[0]) : kn_F2(x);
    const Philox4 rnd = draw(a.seed, a.step, kStreamAngle, e.p);
    const Angle ang = kn_sample_angle(x, rnd.r0 >> 8, F2);
    collide_pair(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(rnd.r1), a.collide64_sq);
    bool upd_e = true, upd_g = true;
    if (a.weighted) {
        // weight rejection: the heavier partner takes its new momentum with
        // probability w_light / w_heavy; u w_heavy < w_light is decided
        // exactly (both products of 24-bit mantissas fit FP64)
        const float we = a.w_e ? a.w_e[e.ie] : a.w_const;
        const float wg = a.w_g ? a.w_g[e.ig] : a.w_const;
        const double uw = (double)u24_closed0(rnd.r2);
        if (we > wg) upd_e = uw * (double)we < (double)wg;
        else if (wg > we) upd_g = uw * (double)wg < (double)we;
    }
    if (upd_e) {
        a.u[0][e.ie] = ux;
        a.u[1][e.ie] = uy;
        a.u[2][e.ie] = uz;
    }
    if (upd_g) {
        a.k[0][e.ig] = kx;
        a.k[1][e.ig] = ky;
        a.k[2][e.ig] = kz;
    }
}

// The analytic probability of one pair and its rest-frame energy x.
__device__ __forceinline__ float analytic_P(const ScatterArgs& a, float ux, float uy, float uz, float kx, float ky,
                                           float kz, float dens, float* x_out)
{
    return analytic_prob(ux, uy, uz, kx, ky, kz, dens, a.dt, a.gamma64, x_out);
}


// Probability, Bernoulli trial and list of accepted pairs.
//
// Candidate filter: sigma_KN <= sigma_T and v = 1 - beta cos psi <= 2 bound
// every pair's probability by P_b = 1 - exp(-2 n dt) (the P_max of the
// No-Time-Counter method, Sec. 3.1), and the network output r <= 1 gives the
// same bound in the surrogate modes.  A pair whose uniform u0 >= P_b cannot
// collide, so only the candidates u0 < P_b (a fraction ~2 n dt of the pairs)
// load their momenta and evaluate P; the decision u0 < P is the one the full
// evaluation would take, bit for bit.  With prob_out requested every pair is
// evaluated.
//
// Every warp works on its own: it owns a contiguous run of 128-pair chunks
// (32 lanes x 4 consecutive pairs, one Philox block per lane), stages the
// cells of the current pair tile in its own shared-memory window, and keeps
// its own queue of candidates, so no warp ever waits for another at a barrier.
// Per chunk (phase A): locate each pair's cell (a per-pair cell map staged
// with the tile), draw the four Bernoulli words, test them against the cell's
// integer threshold (the exact image of u0 < P_b on the 24-bit uniform) and
// append the candidates to the queue.  Candidates are evaluated 32 at a time,
// one per lane (phase B), as soon as 32 are queued; other warps hide the
// scattered loads.  Accepted pairs go to the warp's own region of the
// accepted list.  Candidates above the FP64 gamma threshold are set aside and
// decided after the warp's last chunk.
constexpr int kProbWarps = kProbThreads / 32;
constexpr int kChunkPairs = 32 * kPairsPerThread;  // pairs of one warp step
constexpr int kWarpCells = 64;                     // cells of a pair tile a warp stages
constexpr int kQueueCap = 160;                     // queued candidates per warp (31 + one chunk's 128)

struct WarpWindow {
    int32_t off[kWarpCells];    // first pair of each cell
    int2 shift[kWarpCells];     // first sorted electron and photon minus the first pair
    float dens[kWarpCells];     // pair density
    uint32_t thr[kWarpCells];   // candidate threshold on the 24-bit uniform
    uint8_t cell[kPairsPerTile];  // the window cell of each pair of the tile
};

struct WarpQueue {
    int32_t ie[kQueueCap], ig[kQueueCap];
    float dens[kQueueCap], u0[kQueueCap];
    uint32_t p[kQueueCap];
};

// The candidate test u0 < P_b on u0 = m 2^-24 (m = word >> 8) as m < T with
// T = ceil(P_b 2^24): P_b 2^24 is exact in FP32 (a power-of-two scaling) and
// m is an integer, so the two tests agree for every word.  The 2.0002 factor
// keeps P_b above any FP32 rounding of P.
__device__ __forceinline__ uint32_t cand_threshold(float dens, float dt)
{
    return (uint32_t)ceilf(one_minus_exp_neg(2.0002f * dens * dt) * 16777216.0f);
}

// One evaluation batch: up to 32 queue entries from slot `first` on, one
// per lane, with their momenta.
struct Batch {
    int n, first;  // entries, first slot (the same in every lane)
    float u[3], k[3];
};

// kCandOut (the surrogate modes' first kernel): the same filter, but each
// batch of candidates goes with its momenta to the context's candidate list
// (one atomic per batch) instead of being evaluated.
template <bool kBinned, bool kWeighted, bool kCandOut = false>
__global__ void __launch_bounds__(kProbThreads, 4) k_pair_prob(ScatterArgs a)
{
    __shared__ WarpWindow s_win[kProbWarps];
    __shared__ WarpQueue s_queue[kProbWarps];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int w = threadIdx.x >> 5;
    WarpWindow& W = s_win[w];
    WarpQueue& Q = s_queue[w];
    // pair indices: 32-bit for the binned pair list (its offsets are int32),
    // 64-bit for explicit pair lists
    using pidx = typename std::conditional<kBinned, int32_t, int64_t>::type;
    const pidx total = kBinned ? (pidx)*a.n_pairs : (pidx)a.p_end;
    const pidx pbase = kBinned ? 0 : (pidx)a.p_begin;
    const int64_t n_chunks = total > pbase ? ((int64_t)total - pbase + kChunkPairs - 1) / kChunkPairs : 0;
    const int64_t n_warps = (int64_t)gridDim.x * kProbWarps;
    const int64_t gw = (int64_t)blockIdx.x * kProbWarps + w;
    const int ch_begin = (int)(n_chunks * gw / n_warps), ch_end = (int)(n_chunks * (gw + 1) / n_warps);
    const bool all = a.prob_out != nullptr;
    unsigned n_pairs = 0;
    int qh = 0, qn = 0;     // queue head and length (the same in every lane)
    // this warp's region of the accepted list: one slot per pair it owns
    const uint32_t acc_base = (uint32_t)ch_begin * kChunkPairs;
    uint32_t n_acc = 0, n_rare = 0;
    int win_tile = -1;  // pair tile whose cells the window holds
    int c_first = 0, nw = 0;

    // Take up to 32 candidates off the queue and load their momenta.  The
    // entries stay in their slots until the batch is evaluated; a chunk
    // starts with fewer than 32 entries queued and appends at most 128.
    auto take = [&](Batch& b) {
        b.n = qn < 32 ? qn : 32;
        b.first = qh;
        int slot = qh + (int)lane;
        if (slot >= kQueueCap) slot -= kQueueCap;
        if ((int)lane < b.n) {
            const int32_t ie = Q.ie[slot], ig = Q.ig[slot];
            b.u[0] = a.u[0][ie];
            b.u[1] = a.u[1][ie];
            b.u[2] = a.u[2][ie];
            b.k[0] = a.k[0][ig];
            b.k[1] = a.k[1][ig];
            b.k[2] = a.k[2][ig];
        }
        qh += b.n;
        if (qh >= kQueueCap) qh -= kQueueCap;
        qn -= b.n;
    };
    // probability, decision and accepted-list entry of a batch; the rare
    // candidates whose electron lies above the FP64 gamma threshold are set
    // aside in the warp's region of the candidate list and decided after the
    // warp's last chunk, so that the FP64 invariants stay out of the loop
    auto evaluate = [&](const Batch& b) {
        if (kCandOut) {
            uint32_t base = 0;
            if (lane == 0 && b.n > 0) base = atomicAdd(a.n_cand, (uint32_t)b.n);
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((int)lane < b.n) {
                int slot = b.first + (int)lane;
                if (slot >= kQueueCap) slot -= kQueueCap;
                a.cand[base + lane] = CandPair{Q.ie[slot], Q.ig[slot], Q.dens[slot], Q.u0[slot], Q.p[slot],
                                               {b.u[0], b.u[1], b.u[2]}, {b.k[0], b.k[1], b.k[2]}, 0u};
            }
            return;
        }
        bool hit = false, rare = false;
        float x = -1.0f, F2 = 0.0f;
        int32_t ie = 0, ig = 0;
        uint32_t p = 0;
        float dens = 0.0f, u0 = 1.0f;
        if ((int)lane < b.n) {
            int slot = b.first + (int)lane;
            if (slot >= kQueueCap) slot -= kQueueCap;
            ie = Q.ie[slot];
            ig = Q.ig[slot];
            p = Q.p[slot];
            dens = Q.dens[slot];
            u0 = Q.u0[slot];
            const Invariants inv = invariants_f32(b.u[0], b.u[1], b.u[2], b.k[0], b.k[1], b.k[2]);
            x = inv.x;
            rare = inv.gamma > a.gamma64;
            if (!rare) {
                // sigma_KN from its series below x = 1, the closed form above
                F2 = kn_F2(inv.x);
                const float Pr = one_minus_exp_neg(dens * a.dt * 0.375f * F2 * inv.v);
                const float P = inv.eps > 0.0f ? Pr : 0.0f;
                hit = u0 < P;
                if (a.prob_out) a.prob_out[p] = P;
                if (a.flag_out) a.flag_out[p] = hit ? 1 : 0;
            }
        }
        const unsigned mr = __ballot_sync(0xffffffffu, rare);
        if (rare)
            a.cand_rare[acc_base + n_rare + __popc(mr & lt_mask)] =
                CandPair{ie, ig, dens, u0, p, {b.u[0], b.u[1], b.u[2]}, {b.k[0], b.k[1], b.k[2]}, 0u};
        n_rare += __popc(mr);
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit)
            a.accepted[acc_base + n_acc + __popc(m & lt_mask)] =
                AcceptedPair{ie, ig, x, p, {b.u[0], b.u[1], b.u[2]}, {b.k[0], b.k[1], b.k[2]}, {__float_as_uint(F2), 0u}};
        n_acc += __popc(m);
    };

    for (int ch = ch_begin; ch < ch_end; ++ch) {
        // ---------------- phase A: the chunk's 128 pairs ----------------
        const pidx q0 = pbase + (pidx)ch * kChunkPairs;
        const pidx pb = q0 + 4 * (pidx)lane;
        const Philox4 rnd4 = draw(a.seed, a.step, kStreamScatter, (uint32_t)(pb >> 2));
        const uint32_t words[4] = {rnd4.r0, rnd4.r1, rnd4.r2, rnd4.r3};
        if (kBinned) {
            const int t = (int)(q0 / kPairsPerTile);
            if (t != win_tile) {
                __syncwarp();  // every lane is done with the previous window
                win_tile = t;
                c_first = a.tile_cell[t];
                nw = a.tile_cell[t + 1] - c_first + 1;
                if (nw <= kWarpCells) {
                    for (int i = (int)lane; i < nw; i += 32) {
                        const CellInfo c = a.cinfo[c_first + i];
                        W.off[i] = c.pair_off;
                        W.shift[i] = make_int2(c.e_start - c.pair_off, c.g_start - c.pair_off);
                        W.dens[i] = c.dens;
                        if (!kWeighted) W.thr[i] = cand_threshold(c.dens, a.dt);
                    }
                    __syncwarp();
                    // the cell map: cell i owns the tile's pairs from its first
                    // pair to the next cell's (clipped to the tile); the last
                    // cell of the window owns the rest of the tile
                    const int q_t = t * kPairsPerTile;
                    for (int i = (int)lane; i < nw; i += 32) {
                        int o0 = W.off[i] - q_t;
                        int o1 = i + 1 < nw ? W.off[i + 1] - q_t : kPairsPerTile;
                        o0 = o0 < 0 ? 0 : o0;
                        o1 = o1 > kPairsPerTile ? kPairsPerTile : o1;
                        int q = o0;
                        for (; q < o1 && (q & 3); ++q) W.cell[q] = (uint8_t)i;
                        for (; q + 4 <= o1; q += 4)
                            *reinterpret_cast<uint32_t*>(&W.cell[q]) = 0x01010101u * (uint32_t)i;
                        for (; q < o1; ++q) W.cell[q] = (uint8_t)i;
                    }
                }
                __syncwarp();
            }
        }
        const bool local = nw <= kWarpCells;
        const CellInfo* cw = a.cinfo + c_first;  // the tile's cells in global memory (wide tiles)
        // the window cells of the lane's four pairs, one byte each
        const uint32_t cells4 =
            (kBinned && local) ? *reinterpret_cast<const uint32_t*>(&W.cell[pb - (pidx)win_tile * kPairsPerTile]) : 0u;
        int ci = 0;
        if (kBinned && !local && pb < total) {
            int lo = 0, hi = nw - 1;  // last cell whose first pair is <= pb
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cw[mid].pair_off <= pb) lo = mid; else hi = mid - 1;
            }
            ci = lo;
        }
        int cur = -1;
        int32_t c_off = 0, c_es = 0, c_gs = 0;
        float c_dens = 0.0f;
        uint32_t c_thr = 0;
#pragma unroll
        for (int r = 0; r < kPairsPerThread; ++r) {
            const pidx p = pb + r;
            const bool valid = p < total;
            int ie = 0, ig = 0;
            float dens = 0.0f;
            uint32_t thr = 0;
            if (valid) {
                if (kBinned && local) {
                    // the same loads in every lane: no per-lane cell bookkeeping
                    const int cr = (int)((cells4 >> (8 * r)) & 0xFFu);
                    const int2 sh = W.shift[cr];
                    ie = sh.x + (int)p;
                    ig = sh.y + (int)p;
                    dens = pair_density<kWeighted>(a, W.dens[cr], ie, ig);
                    thr = kWeighted ? cand_threshold(dens, a.dt) : W.thr[cr];
                } else if (kBinned) {
                    // a tile of more cells than the window: cells in global memory
                    while (ci + 1 < nw && cw[ci + 1].pair_off <= p) ++ci;
                    if (ci != cur) {
                        cur = ci;
                        const CellInfo c = cw[ci];
                        c_off = c.pair_off;
                        c_es = c.e_start;
                        c_gs = c.g_start;
                        c_dens = c.dens;
                        if (!kWeighted) c_thr = cand_threshold(c.dens, a.dt);
                    }
                    const int j = (int)(p - c_off);
                    ie = c_es + j;
                    ig = c_gs + j;
                    dens = pair_density<kWeighted>(a, c_dens, ie, ig);
                    thr = kWeighted ? cand_threshold(dens, a.dt) : c_thr;
                } else {
                    ie = (int)p;
                    ig = (int)p;
                    dens = a.n_dens[p];
                    thr = cand_threshold(dens, a.dt);
                }
                ++n_pairs;
            }
            const bool is_cand = valid && (all || (words[r] >> 8) < thr);
            if (valid && !is_cand && a.flag_out) a.flag_out[p] = 0;
            const unsigned m = __ballot_sync(0xffffffffu, is_cand);
            if (is_cand) {
                int slot = qh + qn + __popc(m & lt_mask);
                if (slot >= kQueueCap) slot -= kQueueCap;
                Q.ie[slot] = ie;
                Q.ig[slot] = ig;
                Q.dens[slot] = dens;
                Q.u0[slot] = u24_closed0(words[r]);
                Q.p[slot] = (uint32_t)p;
            }
            qn += __popc(m);
        }
        __syncwarp();  // the queue entries are visible to every lane

        // ---------------- phase B: candidates, 32 at a time ----------------
        while (qn >= 32) {
            Batch b;
            take(b);
            evaluate(b);
        }
        __syncwarp();  // slots evaluated above may be refilled by other lanes next
    }
    while (qn > 0) {
        Batch b;
        take(b);
        evaluate(b);
    }

    // the rare candidates set aside: the analytic probability with the FP64
    // invariants and the closed-form cross section as they need
    __syncwarp();
    for (uint32_t i0 = 0; i0 < n_rare; i0 += 32) {
        const uint32_t i = i0 + lane;
        bool hit = false;
        float x = -1.0f;
        CandPair c{};
        if (i < n_rare) {
            c = a.cand_rare[acc_base + i];
            const float P = analytic_P(a, c.u[0], c.u[1], c.u[2], c.k[0], c.k[1], c.k[2], c.dens, &x);
            hit = c.u0 < P;
            if (a.prob_out) a.prob_out[c.p] = P;
            if (a.flag_out) a.flag_out[c.p] = hit ? 1 : 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (hit)
            a.accepted[acc_base + n_acc + __popc(m & lt_mask)] =
                AcceptedPair{c.ie, c.ig, x, c.p, {c.u[0], c.u[1], c.u[2]}, {c.k[0], c.k[1], c.k[2]}, {0u, 0u}};
        n_acc += __popc(m);
    }

    // counters: the warp's accepted count for the collision kernel, warp
    // sums of the statistics, one atomic per warp
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n_pairs += __shfl_xor_sync(0xffffffffu, n_pairs, d);
    if (lane == 0) {
        a.warp_acc[gw] = n_acc;
        if (n_pairs) atomicAdd(&a.stats->pairs_tested, (unsigned long long)n_pairs);
        if (n_acc) atomicAdd(&a.stats->scatters, (unsigned long long)n_acc);
    }
}

// The collisions of the accepted pairs of k_pair_prob: the list has
// prob_warps regions (region w from pair index chunk_begin(w) * 128 on,
// warp_acc[w] entries); kCollideWarps warps share a region, taking its
// entries 32 at a time in turn (one, two, four and eight warps per region:
// 0.083, 0.072, 0.066 and 0.065 ms on the 512^2 step; the regions' lengths
// vary, and with one warp each the longest set the kernel's time).
constexpr int kCollideWarps = 8;
__global__ void __launch_bounds__(128) k_collide_regions(ScatterArgs a, int prob_warps)
{
    const int64_t total = a.n_pairs ? *a.n_pairs : a.p_end;
    const int64_t pbase = a.n_pairs ? 0 : a.p_begin;
    const int64_t n_chunks = total > pbase ? (total - pbase + kChunkPairs - 1) / kChunkPairs : 0;
    const unsigned lane = threadIdx.x & 31u;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int v = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); v < kCollideWarps * prob_warps;
         v += warps) {
        const int w = v / kCollideWarps;
        const uint32_t base = (uint32_t)(n_chunks * w / prob_warps) * kChunkPairs;
        const uint32_t n = a.warp_acc[w];
        for (uint32_t i = lane + 32u * (uint32_t)(v % kCollideWarps); i < n; i += 32u * kCollideWarps)
            resolve(a, a.accepted[base + i]);
    }
}

// Surrogate modes, third kernel: every candidate's probability from its
// network output r (P = 1 - exp(-2 n dt r)) or, outside the network's
// training range (compton_mlp_set_range), from the analytic
// path (counted); the decision; accepted pairs to the list.
__global__ void __launch_bounds__(256) k_decide(ScatterArgs a)
{
    const uint32_t n = *a.n_cand;
    const unsigned lane = threadIdx.x & 31u;
    unsigned n_hit = 0, n_fb = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // warp-uniform trip count, so the ballots see whole warps
    const uint32_t first = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint32_t base = first; base < n; base += stride) {
        const uint32_t i = base + lane;
        bool hit = false;
        CandPair c{};
        float x = -1.0f;
        float ux = 0.0f, uy = 0.0f, uz = 0.0f, kx = 0.0f, ky = 0.0f, kz = 0.0f;
        if (i < n) {
            c = a.cand[i];
            ux = c.u[0];
            uy = c.u[1];
            uz = c.u[2];
            kx = c.k[0];
            ky = c.k[1];
            kz = c.k[2];
            const float g2 = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, 1.0f)));
            const float e2 = fmaf(kx, kx, fmaf(ky, ky, kz * kz));
            float P;
            if (mlp_in_range(a.mlp, g2, e2)) {
                P = one_minus_exp_neg(2.0f * c.dens * a.dt * a.r_mlp[i]);
            } else {
                ++n_fb;
                P = analytic_P(a, ux, uy, uz, kx, ky, kz, c.dens, &x);
            }
            hit = c.u0 < P;
            if (a.prob_out) a.prob_out[c.p] = P;
            if (a.flag_out) a.flag_out[c.p] = hit ? 1 : 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(a.n_accepted, (uint32_t)__popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (hit) {
                a.accepted[at + __popc(m & ((1u << lane) - 1u))] =
                    AcceptedPair{c.ie, c.ig, x, c.p, {ux, uy, uz}, {kx, ky, kz}, {0u, 0u}};
                ++n_hit;
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        n_hit += __shfl_xor_sync(0xffffffffu, n_hit, d);
        n_fb += __shfl_xor_sync(0xffffffffu, n_fb, d);
    }
    if (lane == 0) {
        if (n_hit) atomicAdd(&a.stats->scatters, (unsigned long long)n_hit);
        if (n_fb) atomicAdd(&a.stats->mlp_fallbacks, (unsigned long long)n_fb);
    }
}

__global__ void __launch_bounds__(256) k_collide(ScatterArgs a)
{
    const uint32_t n = *a.n_accepted;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) resolve(a, a.accepted[i]);
}

// No-Time-Counter candidate selection (Sec. 3.1, second step; Bird 1989),
// one thread per cell: the cell draws N = floor(E + U) candidates with
// E = N_e N_g (w/V) 2 dt (sigma_max v_max = 2 sigma_T c) and U from
// Philox(c, step, 5); candidate j takes the block (c, step, 6 | j << 8):
// word 0 picks the electron, word 1 the photon, the pair collides iff the
// uniform of word 2 is below r = sigma_KN(x) v / (2 sigma_T), word 3 drives
// the angle and word 0 of block (c, step, 7 | j << 8) the azimuth.  An
// accepted candidate collides at once, so later candidates of the cell see
// the updated momenta.  E + U is formed in FP64 with explicit rounding so the
// candidate count is the one FP64 arithmetic gives.
struct NtcArgs {
    float* u[3];
    float* k[3];
    const int32_t* off_e;
    const int32_t* off_g;
    int64_t n_cells;
    double w_over_v, dt;
    uint64_t seed, step;
    float gamma64, collide64_sq;
    DeviceStats* stats;
    uint32_t* next;      // next cell to take (zeroed before the launch)
    uint32_t* next_big;  // next listed cell to take (zeroed before the launch)
    int32_t* big;        // cells of at least kNtcBig candidates
    uint32_t* n_big;     // their count (zeroed before the launch)
};

// Candidates of cell c: floor(N_e N_g (w/V) 2 dt + u) (the NTC count,
// rounded with a uniform from the cell's own draw).
__device__ __forceinline__ int32_t ntc_count(const NtcArgs& a, int32_t c, int ne, int ng)
{
    const Philox4 rc = draw(a.seed, a.step, 5u, (uint32_t)c);
    const double expect = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn((double)ne, (double)ng), a.w_over_v), 2.0), a.dt);
    const double uc = (double)(rc.r0 >> 8) * (1.0 / 16777216.0);
    return (int32_t)floor(__dadd_rn(expect, uc));
}

// Cells with at least this many candidates are taken by a whole warp.
constexpr int kNtcBig = 32;

__device__ __forceinline__ int pick_index(uint32_t w, int n) { return (int)(((uint64_t)w * (uint64_t)n) >> 32); }

// NTC, first pass: every cell's candidate count; the cells of at least
// kNtcBig candidates go to the list the warps of k_ntc take first.
__global__ void __launch_bounds__(256) k_ntc_scan(NtcArgs a)
{
    unsigned long long n_cand = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.n_cells; c += stride) {
        const int e0 = a.off_e[c], ne = a.off_e[c + 1] - e0;
        const int g0 = a.off_g[c], ng = a.off_g[c + 1] - g0;
        if (ne > 0 && ng > 0) {
            const int32_t nc = ntc_count(a, (int32_t)c, ne, ng);
            n_cand += (unsigned long long)nc;
            if (nc >= kNtcBig) a.big[atomicAdd(a.n_big, 1u)] = (int32_t)c;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n_cand += __shfl_xor_sync(0xffffffffu, n_cand, d);
    if ((threadIdx.x & 31u) == 0 && n_cand) atomicAdd(&a.stats->pairs_tested, n_cand);
}

// The candidates of cell c from candidate j0 on, by the whole warp, exact
// and in order: the warp evaluates the next 32 candidates at once on the
// momenta as they are; candidate k's evaluation is what the sequence would
// give unless an earlier candidate of the batch was accepted and shares its
// electron or photon.  The candidates before the first such k are final:
// their accepted ones (which share no particle) collide and write back, and
// the next batch starts at k with the updated momenta.
__device__ __forceinline__ unsigned long long ntc_cell_warp(const NtcArgs& a, int32_t c)
{
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long n_coll = 0;
    const int e0 = a.off_e[c], ne = a.off_e[c + 1] - e0;
    const int g0 = a.off_g[c], ng = a.off_g[c + 1] - g0;
    const int32_t nc = ntc_count(a, c, ne, ng);
    for (int32_t j0 = 0; j0 < nc;) {
        const int32_t j = j0 + (int32_t)lane;
        const bool valid = j < nc;
        int ie = -1, ig = -1;
        bool acc = false;
        float ux = 0.0f, uy = 0.0f, uz = 0.0f, kx = 0.0f, ky = 0.0f, kz = 0.0f, x = 0.0f, F2 = 0.0f;
        uint32_t r3 = 0;
        if (valid) {
            const Philox4 q = draw(a.seed, a.step, 6u | ((uint32_t)j << 8), (uint32_t)c);
            ie = e0 + pick_index(q.r0, ne);
            ig = g0 + pick_index(q.r1, ng);
            ux = a.u[0][ie];
            uy = a.u[1][ie];
            uz = a.u[2][ie];
            kx = a.k[0][ig];
            ky = a.k[1][ig];
            kz = a.k[2][ig];
            const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
            float v = inv.v;
            x = inv.x;
            if (inv.gamma > a.gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
            F2 = kn_F2(x);
            const float ratio = inv.eps > 0.0f ? 0.5f * 0.375f * F2 * v : 0.0f;
            acc = u24_closed0(q.r2) < ratio;
            r3 = q.r3;
        }
        // the first candidate whose evaluation an earlier accepted one of the
        // batch may have changed
        bool stale = false;
        const unsigned accm = __ballot_sync(0xffffffffu, acc);
#pragma unroll 4
        for (int i = 0; i < 31; ++i) {
            const int iei = __shfl_sync(0xffffffffu, ie, i), igi = __shfl_sync(0xffffffffu, ig, i);
            stale |= (int)lane > i && ((accm >> i) & 1u) && (iei == ie || igi == ig);
        }
        const unsigned sm = __ballot_sync(0xffffffffu, stale && valid);
        const int nv = nc - j0 < 32 ? nc - j0 : 32;
        const int kf = sm ? __ffs(sm) - 1 : nv;  // candidates j0 .. j0 + kf - 1 are final
        if ((int)lane < kf && acc) {
            const Philox4 z = draw(a.seed, a.step, 7u | ((uint32_t)j << 8), (uint32_t)c);
            const Angle ang = kn_sample_angle(x, r3 >> 8, F2);
            collide_pair(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(z.r0), a.collide64_sq);
            a.u[0][ie] = ux;
            a.u[1][ie] = uy;
            a.u[2][ie] = uz;
            a.k[0][ig] = kx;
            a.k[1][ig] = ky;
            a.k[2][ig] = kz;
            ++n_coll;
        }
        __syncwarp();  // the next batch reads the momenta written here
        j0 += kf;
    }
    return n_coll;
}

// NTC, second pass.  Warps first take the cells of many candidates from the
// list, one cell per warp (ntc_cell_warp), so that the longest sequences
// start at once; then every lane works through the candidates of the other
// cells in order, taking the next cell from a shared counter when its cell
// is done, so that a warp's lanes stay busy however unequal the cells'
// candidate counts are.  A cell's candidates run in sequence, so the results
// do not depend on which warp or lane takes the cell.
__global__ void __launch_bounds__(256) k_ntc(NtcArgs a)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long n_coll = 0;
    const uint32_t n_big = *a.n_big;
    for (;;) {
        uint32_t w = 0;
        if (lane == 0) w = atomicAdd(a.next_big, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= n_big) break;
        n_coll += ntc_cell_warp(a, a.big[w]);
    }
    int64_t c = 0, nc = 0, j = 0;
    int e0 = 0, ne = 0, g0 = 0, ng = 0;
    bool done = false;
    for (;;) {
        // lanes with no candidate left take the next cells, one atomic per warp
        const bool need = !done && j >= nc;
        const unsigned want = __ballot_sync(0xffffffffu, need);
        if (want) {
            const int leader = __ffs(want) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(a.next, (uint32_t)__popc(want));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                c = (int64_t)base + __popc(want & lt_mask);
                j = 0;
                nc = 0;
                if (c >= a.n_cells) {
                    done = true;
                } else {
                    e0 = a.off_e[c];
                    ne = a.off_e[c + 1] - e0;
                    g0 = a.off_g[c];
                    ng = a.off_g[c + 1] - g0;
                    if (ne > 0 && ng > 0) {
                        nc = ntc_count(a, (int32_t)c, ne, ng);
                        if (nc >= kNtcBig) nc = 0;  // a listed cell: done above
                    }
                }
            }
        }
        if (__all_sync(0xffffffffu, done)) break;
        if (done || j >= nc) continue;
        const Philox4 q = draw(a.seed, a.step, 6u | ((uint32_t)j << 8), (uint32_t)c);
        const int ie = e0 + pick_index(q.r0, ne);
        const int ig = g0 + pick_index(q.r1, ng);
        float ux = a.u[0][ie], uy = a.u[1][ie], uz = a.u[2][ie];
        float kx = a.k[0][ig], ky = a.k[1][ig], kz = a.k[2][ig];
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        float x = inv.x, v = inv.v;
        if (inv.gamma > a.gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
        const float F2 = kn_F2(x);
        const float ratio = inv.eps > 0.0f ? 0.5f * 0.375f * F2 * v : 0.0f;
        if (u24_closed0(q.r2) < ratio) {
            const Philox4 z = draw(a.seed, a.step, 7u | ((uint32_t)j << 8), (uint32_t)c);
            const Angle ang = kn_sample_angle(x, q.r3 >> 8, F2);
            collide_pair(ux, uy, uz, kx, ky, kz, x, ang, u24_closed0(z.r0), a.collide64_sq);
            a.u[0][ie] = ux;
            a.u[1][ie] = uy;
            a.u[2][ie] = uz;
            a.k[0][ig] = kx;
            a.k[1][ig] = ky;
            a.k[2][ig] = kz;
            ++n_coll;
        }
        ++j;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n_coll += __shfl_xor_sync(0xffffffffu, n_coll, d);
    if (lane == 0 && n_coll) atomicAdd(&a.stats->scatters, n_coll);
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

// Persistent probability kernel: at most the CTAs resident at once (four
// per SM).
unsigned prob_grid(unsigned tiles)
{
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    if (n_sm > kMaxProbWarps / (4 * kProbWarps)) n_sm = kMaxProbWarps / (4 * kProbWarps);
    const unsigned cap = (unsigned)n_sm * 4u;
    return tiles < 1u ? 1u : (tiles < cap ? tiles : cap);
}

// CTAs of 256 threads over a list of up to max_accepted entries: up to 32
// per SM, so that a 512^2 step's accepted pairs (about a million) take at
// most one entry per thread (with 8 per SM each thread resolved two or three
// in turn: 0.119 against 0.106 ms for the BF16-network step's collisions).
int collide_grid(int64_t max_accepted)
{
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    const int64_t want = (max_accepted + 255) / 256;
    const int64_t cap = (int64_t)n_sm * 32;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

void fill_common(ScatterArgs& a, compton_ctx* ctx, uint64_t seed, uint64_t step, float* prob_out, uint8_t* flag_out)
{
    a.dt = (float)ctx->cfg.dt;
    a.seed = seed;
    a.step = step;
    a.gamma64 = ctx->cfg.gamma_fp64_threshold;
    a.collide64_sq = ctx->cfg.collide_fp64_threshold * ctx->cfg.collide_fp64_threshold;
    a.prob_out = prob_out;
    a.flag_out = flag_out;
    a.stats = ctx->stats;
    a.r_mlp = ctx->r_buf;
    a.accepted = ctx->accepted;
    a.n_accepted = ctx->n_accepted;
    a.warp_acc = ctx->warp_acc;
    a.cand_rare = ctx->cand;
    a.cand = ctx->cand;
    a.n_cand = ctx->n_cand;
    a.mlp = ctx->mlp;
    a.w_e = nullptr;
    a.w_g = nullptr;
    a.w_const = (float)ctx->cfg.w_over_v;
    a.weighted = false;
}

// The collisions of the accepted pairs.
compton_status launch_collide(compton_ctx* ctx, ScatterArgs& a, int64_t rows, cudaStream_t stream)
{
    {
        TimedScope ts_(ctx, COMPTON_K_COLLIDE, stream);
        k_collide<<<collide_grid(rows), 256, 0, stream>>>(a);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_collide");
    return COMPTON_OK;
}

// The step after the pair list is known: probability and trial of every
// pair (plain: one kernel; surrogate: candidates, network, decisions), then
// the collisions.  Tiles: pair tiles of this launch; rows: a host bound on
// the pair count.
template <bool kBinned, bool kWeighted>
compton_status launch_step(compton_ctx* ctx, ScatterArgs& a, compton_mode mode, unsigned tiles, int64_t rows,
                           cudaStream_t stream)
{
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->n_accepted, 0, sizeof(uint32_t), stream));
    if (mode == COMPTON_MODE_PLAIN) {
        const unsigned grid = prob_grid(tiles);
        {
            TimedScope ts_(ctx, COMPTON_K_PROB, stream);
            k_pair_prob<kBinned, kWeighted><<<grid, kProbThreads, 0, stream>>>(a);
        }
        COMPTON_LAUNCH_CHECK(ctx, "k_pair_prob");
        const int prob_warps = (int)grid * kProbWarps;
        {
            TimedScope ts_(ctx, COMPTON_K_COLLIDE, stream);
            // kCollideWarps warps per region, four to a CTA
            k_collide_regions<<<(kCollideWarps * prob_warps + 3) / 4, 128, 0, stream>>>(a, prob_warps);
        }
        COMPTON_LAUNCH_CHECK(ctx, "k_collide_regions");
        return COMPTON_OK;
    } else {
        COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->n_cand, 0, sizeof(uint32_t), stream));
        {
            TimedScope ts_(ctx, COMPTON_K_PROB, stream);
            // the candidate filter of the plain kernel, candidates to the list
            k_pair_prob<kBinned, kWeighted, true><<<prob_grid(tiles), kProbThreads, 0, stream>>>(a);
        }
        COMPTON_LAUNCH_CHECK(ctx, "k_pair_prob<cand>");
        // tensor-core modes and the paper's network decide inside the network
        // kernel; the FP32 network writes r and k_decide decides
        const MlpDecide dec{a.dt, a.gamma64, a.prob_out, a.flag_out};
        if (mode == COMPTON_MODE_PNET) {
            const compton_status sp = launch_pnet_decide(ctx, rows, dec, a.w_e, a.w_g, stream);
            if (sp != COMPTON_OK) return sp;
            return launch_collide(ctx, a, rows, stream);
        }
        const bool fused = mode != COMPTON_MODE_MLP_FP32;
        compton_status st = launch_mlp_infer(ctx, a.u[0], a.u[1], a.u[2], a.k[0], a.k[1], a.k[2], rows, mode,
                                             ctx->r_buf, stream, false, true, fused ? &dec : nullptr);
        if (st != COMPTON_OK) return st;
        if (!fused) {
            TimedScope ts_(ctx, COMPTON_K_PROB, stream);
            k_decide<<<collide_grid(rows), 256, 0, stream>>>(a);
        }
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_pair_prob");
    return launch_collide(ctx, a, rows, stream);
}

}  // namespace

compton_status launch_scatter_binned(compton_ctx* ctx, compton_species* e, compton_species* g,
                                     const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                     float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    if (pairs->max_pairs <= 0) return COMPTON_OK;
    if (pairs->max_pairs > ctx->accepted_cap) return COMPTON_ERANGE;
    if (mode != COMPTON_MODE_PLAIN && mode != COMPTON_MODE_PNET && pairs->max_pairs > ctx->cfg.max_particles)
        return COMPTON_ERANGE;
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
    a.p_begin = 0;
    a.p_end = 0;
    fill_common(a, ctx, ctx->cfg.seed, step, prob_out, flag_out);
    const unsigned tiles = (unsigned)((pairs->max_pairs + kPairsPerTile - 1) / kPairsPerTile);
    if (ctx->bin_weighted) {
        a.w_e = e->w_dev;
        a.w_g = g->w_dev;
        a.weighted = true;
        return launch_step<true, true>(ctx, a, mode, tiles, pairs->max_pairs, stream);
    }
    return launch_step<true, false>(ctx, a, mode, tiles, pairs->max_pairs, stream);
}

compton_status launch_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                    float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                    compton_mode mode, float* prob_out, uint8_t* flag_out, cudaStream_t stream)
{
    if (n <= 0) return COMPTON_OK;
    if (mode != COMPTON_MODE_PLAIN && mode != COMPTON_MODE_PNET && n > ctx->cfg.max_particles) return COMPTON_ERANGE;
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
    fill_common(a, ctx, seed, step, prob_out, flag_out);
    // chunks that fit the accepted-pair list (whole tiles, so the Philox
    // blocks of four pairs never straddle two chunks)
    const int64_t chunk = ctx->accepted_cap / kPairsPerTile * kPairsPerTile;
    for (int64_t b = 0; b < n; b += chunk) {
        a.p_begin = b;
        a.p_end = b + chunk < n ? b + chunk : n;
        const unsigned tiles = (unsigned)((a.p_end - a.p_begin + kPairsPerTile - 1) / kPairsPerTile);
        const compton_status st = launch_step<false, false>(ctx, a, mode, tiles, a.p_end - a.p_begin, stream);
        if (st != COMPTON_OK) return st;
    }
    return COMPTON_OK;
}

compton_status launch_scatter_ntc(compton_ctx* ctx, compton_species* e, compton_species* g,
                                  const compton_pairs* pairs, uint64_t step, cudaStream_t stream)
{
    if (pairs->n_cells <= 0) return COMPTON_OK;
    NtcArgs a;
    a.u[0] = e->ux_dev;
    a.u[1] = e->uy_dev;
    a.u[2] = e->uz_dev;
    a.k[0] = g->ux_dev;
    a.k[1] = g->uy_dev;
    a.k[2] = g->uz_dev;
    a.off_e = pairs->off_e_dev;
    a.off_g = pairs->off_g_dev;
    a.n_cells = pairs->n_cells;
    a.w_over_v = ctx->cfg.w_over_v;
    a.dt = ctx->cfg.dt;
    a.seed = ctx->cfg.seed;
    a.step = step;
    a.gamma64 = ctx->cfg.gamma_fp64_threshold;
    a.collide64_sq = ctx->cfg.collide_fp64_threshold * ctx->cfg.collide_fp64_threshold;
    a.stats = ctx->stats;
    // scratch free in this mode: the count arrays of the binning (zeroed by
    // the next binning), each of at least max(C, 64) entries: the listed
    // cells in the electron array, three counters in the photon array
    a.next = reinterpret_cast<uint32_t*>(ctx->count[1]);
    a.next_big = a.next + 1;
    a.n_big = a.next + 2;
    a.big = ctx->count[0];
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(a.next, 0, 3 * sizeof(uint32_t), stream));
    // persistent: the CTAs resident at once (work is taken cell by cell)
    int per_sm = 0;
    COMPTON_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ntc, 256, 0));
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)ctx->n_sm * per_sm;
    const int64_t need = (pairs->n_cells + 255) / 256;
    if (blocks > need) blocks = need;
    {
        TimedScope ts_(ctx, COMPTON_K_NTC, stream);
        int64_t sb = (pairs->n_cells + 255) / 256;
        if (sb > (int64_t)ctx->n_sm * 8) sb = (int64_t)ctx->n_sm * 8;
        k_ntc_scan<<<(unsigned)sb, 256, 0, stream>>>(a);
        k_ntc<<<(unsigned)blocks, 256, 0, stream>>>(a);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_ntc");
    return COMPTON_OK;
}

compton_status launch_kn_ratio(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                               const float* kx, const float* ky, const float* kz, int64_t n, float* r_out,
                               cudaStream_t stream)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)ctx->n_sm * 32) blocks = (int64_t)ctx->n_sm * 32;
    k_kn_ratio<<<(unsigned)blocks, 256, 0, stream>>>(ux, uy, uz, kx, ky, kz, n, ctx->cfg.gamma_fp64_threshold,
                                                     r_out);
    COMPTON_LAUNCH_CHECK(ctx, "k_kn_ratio");
    return COMPTON_OK;
}

compton_status launch_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n, float* cth,
                                   float* sth, float* ratio, cudaStream_t stream)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)ctx->n_sm * 32) blocks = (int64_t)ctx->n_sm * 32;
    k_sample_angle<<<(unsigned)blocks, 256, 0, stream>>>(x, r, n, cth, sth, ratio);
    COMPTON_LAUNCH_CHECK(ctx, "k_sample_angle");
    return COMPTON_OK;
}

}  // namespace compton
