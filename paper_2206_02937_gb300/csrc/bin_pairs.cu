// bin_pairs.cu -- binning and random in-cell pairing (arXiv 2206.02937,
// Sec. 3.1, first step: "the simulation space is divided into collision
// cells, in which the particles are binned; from this binning a list of
// colliding leptons and photons is produced for each cell").
//
// Five launches per call, both species in each:
//   k_count        histogram of cell indices (warp-aggregated atomics)
//   k_scan_reduce  per-tile sums of N_e,c, N_g,c and M_c = min(N_e,c, N_g,c)
//   k_scan_blocks  exclusive scan of the tile sums (one CTA)
//   k_scan_final   per-cell offsets, CellInfo, tile maps; resets the cursors
//   k_key_scatter  Philox key per particle, (key, index) record placed in its
//                  cell's segment (arbitrary order inside the segment)
//   k_sort_gather  per-cell sort of the records by (key, id) in shared memory,
//                  then a coalesced gather of the five particle arrays into
//                  sorted order
// The order within a cell depends only on (key, id): the atomics of
// k_key_scatter decide where a record lands inside its segment, and the sort
// removes that freedom.
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kSortThreads = 512;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// ---------------------------------------------------------------------------
// Histogram.  A warp groups lanes with equal cells (__match_any_sync) and one
// lane per group adds the group size: inputs already sorted by cell (every
// step after the first) cost one atomic per run instead of one per particle.
// ---------------------------------------------------------------------------
__global__ void k_count(const int32_t* __restrict__ cell_e, int64_t n_e, const int32_t* __restrict__ cell_g,
                        int64_t n_g, int64_t C, int32_t* __restrict__ count_e, int32_t* __restrict__ count_g,
                        DeviceStats* stats)
{
    const int s = blockIdx.y;
    const int32_t* cell = s == 0 ? cell_e : cell_g;
    const int64_t n = s == 0 ? n_e : n_g;
    int32_t* count = s == 0 ? count_e : count_g;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + 31) / 32 * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        int c = -1;
        if (i < n) {
            const int32_t ci = cell[i];
            if (ci >= 0 && (int64_t)ci < C) c = ci;
            else atomicOr(&stats->error_flags, (unsigned long long)kErrCellRange);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane_id() == (unsigned)(__ffs(peers) - 1)) atomicAdd(&count[c], __popc(peers));
    }
}

// ---------------------------------------------------------------------------
// Scan over cells, in three passes.  Values per cell: N_e, N_g, M = min.
// ---------------------------------------------------------------------------
struct Tri {
    int64_t e, g, m;
};

__device__ __forceinline__ Tri tri_add(Tri a, Tri b) { return {a.e + b.e, a.g + b.g, a.m + b.m}; }

__device__ __forceinline__ Tri warp_incl_scan(Tri v)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t e = __shfl_up_sync(0xffffffffu, v.e, d);
        const int64_t g = __shfl_up_sync(0xffffffffu, v.g, d);
        const int64_t m = __shfl_up_sync(0xffffffffu, v.m, d);
        if (lane_id() >= (unsigned)d) v = {v.e + e, v.g + g, v.m + m};
    }
    return v;
}

// Exclusive scan of one Tri per thread over a block of 256 threads; returns
// the exclusive prefix and writes the block total to *total.
__device__ __forceinline__ Tri block_excl_scan_256(Tri v, Tri* total)
{
    __shared__ Tri warp_tot[8];
    const Tri inc = warp_incl_scan(v);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        Tri t = lane_id() < 8 ? warp_tot[lane_id()] : Tri{0, 0, 0};
        t = warp_incl_scan(t);
        if (lane_id() < 8) warp_tot[lane_id()] = t;
    }
    __syncthreads();
    const Tri before = w > 0 ? warp_tot[w - 1] : Tri{0, 0, 0};
    *total = warp_tot[7];
    __syncthreads();
    return {before.e + inc.e - v.e, before.g + inc.g - v.g, before.m + inc.m - v.m};
}

__global__ void __launch_bounds__(256) k_scan_reduce(const int32_t* __restrict__ count_e,
                                                     const int32_t* __restrict__ count_g, int64_t C,
                                                     int64_t* __restrict__ block_sums, int64_t n_tiles)
{
    const int64_t c0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 8;
    Tri v{0, 0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t c = c0 + j;
        if (c < C) {
            const int64_t a = count_e[c], b = count_g[c];
            v = tri_add(v, Tri{a, b, a < b ? a : b});
        }
    }
    Tri total;
    block_excl_scan_256(v, &total);
    if (threadIdx.x == 0) {
        block_sums[blockIdx.x] = total.e;
        block_sums[n_tiles + blockIdx.x] = total.g;
        block_sums[2 * n_tiles + blockIdx.x] = total.m;
    }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int64_t* __restrict__ block_sums, int64_t n_tiles,
                                                      int64_t* __restrict__ n_pairs)
{
    __shared__ int64_t warp_tot[32];
    for (int s = 0; s < 3; ++s) {
        int64_t* a = block_sums + s * n_tiles;
        int64_t carry = 0;
        for (int64_t base = 0; base < n_tiles; base += 1024) {
            const int64_t i = base + threadIdx.x;
            const int64_t v = i < n_tiles ? a[i] : 0;
            int64_t inc = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane_id() >= (unsigned)d) inc += o;
            }
            const int w = threadIdx.x >> 5;
            if (lane_id() == 31) warp_tot[w] = inc;
            __syncthreads();
            if (w == 0) {
                int64_t t = warp_tot[lane_id()];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int64_t o = __shfl_up_sync(0xffffffffu, t, d);
                    if (lane_id() >= (unsigned)d) t += o;
                }
                warp_tot[lane_id()] = t;
            }
            __syncthreads();
            const int64_t before = w > 0 ? warp_tot[w - 1] : 0;
            const int64_t chunk_total = warp_tot[31];
            if (i < n_tiles) a[i] = carry + before + inc - v;
            carry += chunk_total;
            __syncthreads();
        }
        if (s == 2 && threadIdx.x == 0) *n_pairs = carry;
    }
}

struct ScanFinalArgs {
    int32_t* count_e;
    int32_t* count_g;
    const int64_t* block_sums;
    int64_t n_tiles;
    int64_t C;
    int64_t n_e, n_g;
    int32_t* off_e;
    int32_t* off_g;
    CellInfo* cinfo;
    int32_t* tile_cell;
    int32_t* stile_e;
    int32_t* stile_g;
    int64_t nb_e, nb_g;  // sort tiles per species
    const int64_t* n_pairs;
    double w_over_v;
};

// Sort tiles of a species whose first cell is c+1: every b >= 1 with
// o < b*T <= o+n (the tile boundary lies inside or at the end of cell c).
__device__ __forceinline__ void write_sort_tiles(int32_t* stile, int64_t nb, int64_t o, int64_t n, int64_t c)
{
    if (n <= 0) return;
    const int64_t b_lo = o / kSortTile + 1;
    int64_t b_hi = (o + n) / kSortTile;
    if (b_hi > nb - 1) b_hi = nb - 1;
    for (int64_t b = b_lo; b <= b_hi; ++b) stile[b] = (int32_t)(c + 1);
}

__global__ void __launch_bounds__(256) k_scan_final(ScanFinalArgs a)
{
    const int64_t c0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * 8;
    int32_t ne[8], ng[8];
    Tri v{0, 0, 0};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t c = c0 + j;
        ne[j] = c < a.C ? a.count_e[c] : 0;
        ng[j] = c < a.C ? a.count_g[c] : 0;
        v = tri_add(v, Tri{ne[j], ng[j], ne[j] < ng[j] ? ne[j] : ng[j]});
    }
    Tri total;
    Tri p = block_excl_scan_256(v, &total);
    p.e += a.block_sums[blockIdx.x];
    p.g += a.block_sums[a.n_tiles + blockIdx.x];
    p.m += a.block_sums[2 * a.n_tiles + blockIdx.x];
    const int64_t np_total = *a.n_pairs;
    const int64_t n_pair_tiles = (np_total + kPairsPerTile - 1) / kPairsPerTile;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t c = c0 + j;
        if (c >= a.C) break;
        const int64_t m = ne[j] < ng[j] ? ne[j] : ng[j];
        a.off_e[c] = (int32_t)p.e;
        a.off_g[c] = (int32_t)p.g;
        const int64_t nmax = ne[j] > ng[j] ? ne[j] : ng[j];
        CellInfo ci;
        ci.pair_off = (int32_t)p.m;
        ci.e_start = (int32_t)p.e;
        ci.g_start = (int32_t)p.g;
        ci.dens = (float)((double)nmax * a.w_over_v);
        a.cinfo[c] = ci;
        if (m > 0) {
            // scatter tiles whose first pair lies in [p.m, p.m + m)
            for (int64_t t = (p.m + kPairsPerTile - 1) / kPairsPerTile; t * kPairsPerTile < p.m + m; ++t)
                a.tile_cell[t] = (int32_t)c;
            if (p.m + m == np_total) a.tile_cell[n_pair_tiles] = (int32_t)c;
        }
        write_sort_tiles(a.stile_e, a.nb_e, p.e, ne[j], c);
        write_sort_tiles(a.stile_g, a.nb_g, p.g, ng[j], c);
        a.count_e[c] = 0;  // becomes the insertion cursor of k_key_scatter
        a.count_g[c] = 0;
        if (c == a.C - 1) {
            a.off_e[a.C] = (int32_t)(p.e + ne[j]);
            a.off_g[a.C] = (int32_t)(p.g + ng[j]);
        }
        p.e += ne[j];
        p.g += ng[j];
        p.m += m;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.stile_e[0] = 0;
        a.stile_g[0] = 0;
        a.stile_e[a.nb_e] = (int32_t)a.C;
        a.stile_g[a.nb_g] = (int32_t)a.C;
    }
}

// ---------------------------------------------------------------------------
// Keyed placement: record (key, input index) at off[c] + cursor.
// ---------------------------------------------------------------------------
struct KeyScatterArgs {
    const int32_t* cell[2];
    const uint32_t* id[2];
    int64_t n[2];
    const int32_t* off[2];
    int32_t* cursor[2];
    uint2* rec[2];
    int64_t C;
    uint64_t seed, step;
};

__global__ void k_key_scatter(KeyScatterArgs a)
{
    const bool e = blockIdx.y == 0;
    const int64_t n = e ? a.n[0] : a.n[1];
    const int32_t* __restrict__ cell = e ? a.cell[0] : a.cell[1];
    const uint32_t* __restrict__ id = e ? a.id[0] : a.id[1];
    const int32_t* __restrict__ off = e ? a.off[0] : a.off[1];
    int32_t* __restrict__ cursor = e ? a.cursor[0] : a.cursor[1];
    uint2* __restrict__ rec = e ? a.rec[0] : a.rec[1];
    const uint32_t stream = e ? kStreamPairE : kStreamPairG;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + 31) / 32 * 32;
    const unsigned lane = lane_id();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        int c = -1;
        uint32_t key = 0;
        if (i < n) {
            const int32_t ci = cell[i];
            if (ci >= 0 && (int64_t)ci < a.C) {
                c = ci;
                key = draw(a.seed, a.step, stream, id[i]).r0;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (c >= 0 && lane == (unsigned)leader) base = atomicAdd(&cursor[c], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        if (c >= 0) {
            const int rank = __popc(peers & ((1u << lane) - 1u));
            rec[off[c] + base + rank] = make_uint2(key, (uint32_t)i);
        }
    }
}

// ---------------------------------------------------------------------------
// Per-cell sort by (key, id) and gather into sorted order.
// ---------------------------------------------------------------------------
struct SortGatherArgs {
    const float* in_u[2][3];
    const int32_t* in_cell[2];
    const uint32_t* in_id[2];
    float* out_u[2][3];
    int32_t* out_cell[2];
    uint32_t* out_id[2];
    const uint2* rec[2];
    const int32_t* off[2];
    const int32_t* stile[2];
    int64_t nb_e;
};

// Sort keys are (key << 32 | id) in 64 bits; the shared-memory position j
// breaks ties between equal ids (invalid input), so every order is total and
// every sort yields a permutation.
__device__ __forceinline__ int before64(uint64_t kj, int j, uint64_t ki, int i)
{
    return (kj < ki) | ((kj == ki) & (j < i));
}

// Rank the elements base .. base + 32E - 1 of the segment [a, a+n) against the
// whole segment with one warp: each lane holds E of them in registers and one
// broadcast read of key64[j] serves all E comparisons.  perm[a + rank] = index.
template <int E>
__device__ __forceinline__ void warp_rank_chunk(const uint64_t* key64, int32_t* perm, int a, int n, int base)
{
    const int lane = (int)lane_id();
    uint64_t k[E];
    int idx[E], rank[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        idx[e] = a + base + 32 * e + lane;
        k[e] = base + 32 * e + lane < n ? key64[idx[e]] : 0ull;
        rank[e] = 0;
    }
    for (int j = a; j < a + n; ++j) {
        const uint64_t kj = key64[j];
#pragma unroll
        for (int e = 0; e < E; ++e) rank[e] += before64(kj, j, k[e], idx[e]);
    }
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (base + 32 * e + lane < n) perm[a + rank[e]] = idx[e];
}

// Sort the segment [a, a+n) (n <= 32 E) with one warp: a bitonic network over
// 32 E slots held E per lane (slot i = 32 e + lane), ordered by (key64, index)
// so the order is total and the network always yields a permutation.  Strides
// below 32 exchange through shuffles, larger ones swap registers.
template <int E>
__device__ __forceinline__ void warp_bitonic_segment(uint64_t* key64, int32_t* perm, int a, int n)
{
    const int lane = (int)lane_id();
    uint64_t k[E];
    int32_t p[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        if (i < n) {
            k[e] = key64[a + i];
            p[e] = a + i;
        } else {
            k[e] = ~0ull;
            p[e] = 0x40000000 + i;  // padding sorts last
        }
    }
    constexpr int N = 32 * E;
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & je) == 0) {
                        const int e2 = e | je;
                        const bool asc = ((e * 32 + lane) & kk) == 0;
                        const bool gt = (k[e] > k[e2]) || (k[e] == k[e2] && p[e] > p[e2]);
                        if (gt == asc) {
                            const uint64_t tk = k[e];
                            k[e] = k[e2];
                            k[e2] = tk;
                            const int32_t tp = p[e];
                            p[e] = p[e2];
                            p[e2] = tp;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint64_t ok = __shfl_xor_sync(0xffffffffu, k[e], j);
                    const int32_t op = __shfl_xor_sync(0xffffffffu, p[e], j);
                    const bool take_min = (((lane & j) == 0) == (((e * 32 + lane) & kk) == 0));
                    const bool other_smaller = (ok < k[e]) || (ok == k[e] && op < p[e]);
                    if (take_min == other_smaller) {
                        k[e] = ok;
                        p[e] = op;
                    }
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        if (i < n) {
            perm[a + i] = p[e];
            key64[a + i] = k[e];
        }
    }
    __syncwarp();
}

// Count of sorted keys in key64[b .. b+m) below k (strict) or not above k.
__device__ __forceinline__ int count_below(const uint64_t* key64, int b, int m, uint64_t k, bool or_equal)
{
    int pos = 0;
#pragma unroll
    for (int step = 64; step > 0; step >>= 1) {  // m <= 64: all of a full chunk can count
        if (pos + step <= m) {
            const uint64_t v = key64[b + pos + step - 1];
            if (v < k || (or_equal && v == k)) pos += step;
        }
    }
    return pos;
}

// Segments of 65..256: each 64-element chunk sorted by the bitonic network
// (keys written back in sorted order, source indices in perm), then every
// element's final rank = its rank in its chunk + the number of elements
// before it in each other sorted chunk (binary search; ties go to the lower
// chunk, so ranks stay unique).  Results are written after all ranks are
// known.
__device__ __forceinline__ void warp_chunk_merge_segment(uint64_t* key64, int32_t* perm, int a, int n)
{
    const int lane = (int)lane_id();
    const int nc = (n + 63) >> 6;
    for (int c = 0; c < nc; ++c) {
        const int cn = n - 64 * c < 64 ? n - 64 * c : 64;
        warp_bitonic_segment<2>(key64, perm, a + 64 * c, cn);
    }
    uint64_t kk[8];
    int32_t pp[8];
    int rank[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int idx = lane + 32 * t;
        rank[t] = -1;
        if (idx < n) {
            const int c = idx >> 6;
            kk[t] = key64[a + idx];
            pp[t] = perm[a + idx];
            int r = idx & 63;
            for (int c2 = 0; c2 < nc; ++c2) {
                if (c2 == c) continue;
                const int cn2 = n - 64 * c2 < 64 ? n - 64 * c2 : 64;
                r += count_below(key64, a + 64 * c2, cn2, kk[t], c2 < c);
            }
            rank[t] = r;
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (rank[t] >= 0) {
            key64[a + rank[t]] = kk[t];
            perm[a + rank[t]] = pp[t];
        }
    }
    __syncwarp();
}

// Cells of up to 64 particles: bitonic network in registers; up to 256:
// sorted 64-element chunks merged by rank; larger: register-held ranking
// against the whole cell.  Only perm is meaningful afterwards (key64 may hold
// keys in sorted or in original order, depending on the path).
__device__ __forceinline__ void sort_segment(uint64_t* key64, int32_t* perm, int a, int n)
{
    if (n <= 32) warp_bitonic_segment<1>(key64, perm, a, n);
    else if (n <= 64) warp_bitonic_segment<2>(key64, perm, a, n);
    else if (n <= 256) warp_chunk_merge_segment(key64, perm, a, n);
    else
        for (int base = 0; base < n; base += 256) warp_rank_chunk<8>(key64, perm, a, n, base);
}

__device__ __forceinline__ void gather_out(const SortGatherArgs& g, int s, const uint32_t* src, const int32_t* perm,
                                           int64_t o0, int R)
{
    const uint32_t* __restrict__ iid = g.in_id[s];
    const float* __restrict__ iu0 = g.in_u[s][0];
    const float* __restrict__ iu1 = g.in_u[s][1];
    const float* __restrict__ iu2 = g.in_u[s][2];
    const int32_t* __restrict__ icell = g.in_cell[s];
    for (int p = threadIdx.x; p < R; p += blockDim.x) {
        const int i = perm[p];
        const uint32_t sidx = src[i];
        g.out_u[s][0][o0 + p] = iu0[sidx];
        g.out_u[s][1][o0 + p] = iu1[sidx];
        g.out_u[s][2][o0 + p] = iu2[sidx];
        g.out_cell[s][o0 + p] = icell[sidx];
        g.out_id[s][o0 + p] = iid[sidx];
    }
}

__global__ void __launch_bounds__(kSortThreads, 2) k_sort_gather(SortGatherArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* key64 = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* src = reinterpret_cast<uint32_t*>(key64 + kSortCap);
    int32_t* perm = reinterpret_cast<int32_t*>(src + kSortCap);
    __shared__ int next_cell;

    const int s = (int64_t)blockIdx.x < g.nb_e ? 0 : 1;
    const int64_t b = s == 0 ? blockIdx.x : blockIdx.x - g.nb_e;
    const int32_t* __restrict__ off = g.off[s];
    const uint2* __restrict__ rec = g.rec[s];
    const uint32_t* __restrict__ in_id = g.in_id[s];
    const int64_t c0 = g.stile[s][b];
    const int64_t c1 = g.stile[s][b + 1];
    if (c1 <= c0) return;
    const int64_t o0 = off[c0];
    const int64_t R = (int64_t)off[c1] - o0;
    if (R <= 0) return;

    if (R <= kSortCap) {
        for (int i = threadIdx.x; i < R; i += blockDim.x) {
            const uint2 r = rec[o0 + i];
            key64[i] = ((uint64_t)r.x << 32) | in_id[r.y];
            src[i] = r.y;
        }
        if (threadIdx.x == 0) next_cell = 0;
        __syncthreads();
        // warps take cells in order as they finish (balances uneven cell sizes)
        for (;;) {
            int c = 0;
            if (lane_id() == 0) c = atomicAdd(&next_cell, 1);
            c = __shfl_sync(0xffffffffu, c, 0) + (int)c0;
            if (c >= c1) break;
            const int a = off[c] - (int32_t)o0;
            const int n = off[c + 1] - off[c];
            if (n > 0) sort_segment(key64, perm, a, n);
        }
        __syncthreads();
        gather_out(g, s, src, perm, o0, (int)R);
        return;
    }

    // A cell range larger than shared memory: cell by cell.
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t o = off[c];
        const int64_t n = (int64_t)off[c + 1] - o;
        if (n <= 0) continue;
        if (n <= kSortCap) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const uint2 r = rec[o + i];
                key64[i] = ((uint64_t)r.x << 32) | in_id[r.y];
                src[i] = r.y;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const uint64_t ki = key64[i];
                int rank = 0;
                for (int j = 0; j < n; ++j) rank += before64(key64[j], j, ki, i);
                perm[rank] = i;
            }
            __syncthreads();
            gather_out(g, s, src, perm, o, (int)n);
            __syncthreads();
        } else {
            // Oversized cell: rank against the records in global memory.
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint2 ri = rec[o + i];
                const uint32_t di = in_id[ri.y];
                int64_t rank = 0;
                for (int64_t j = 0; j < n; ++j) {
                    const uint2 rj = rec[o + j];
                    const uint32_t dj = in_id[rj.y];
                    rank += (rj.x < ri.x) | ((rj.x == ri.x) & ((dj < di) | ((dj == di) & (j < i))));
                }
                const int64_t p = o + rank;
                g.out_u[s][0][p] = g.in_u[s][0][ri.y];
                g.out_u[s][1][p] = g.in_u[s][1][ri.y];
                g.out_u[s][2][p] = g.in_u[s][2][ri.y];
                g.out_cell[s][p] = g.in_cell[s][ri.y];
                g.out_id[s][p] = di;
            }
        }
    }
}

int grid_for(int64_t n, int threads, int max_blocks)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace

compton_status launch_bin_pairs(compton_ctx* ctx, const compton_species* e_in, const compton_species* g_in,
                                compton_species* e_out, compton_species* g_out, uint64_t step,
                                cudaStream_t stream)
{
    const int64_t C = ctx->cfg.n_cells;
    const int64_t ne = e_in->n, ng = g_in->n;
    const int64_t n_tiles = (C + kScanTile - 1) / kScanTile;
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->count[0], 0, sizeof(int32_t) * C, stream));
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->count[1], 0, sizeof(int32_t) * C, stream));

    const int64_t nmax = ne > ng ? ne : ng;
    const dim3 pgrid(grid_for(nmax, 256, 152 * 16), 2);
    k_count<<<pgrid, 256, 0, stream>>>(e_in->cell_dev, ne, g_in->cell_dev, ng, C, ctx->count[0], ctx->count[1],
                                       ctx->stats);
    COMPTON_LAUNCH_CHECK(ctx, "k_count");
    k_scan_reduce<<<(unsigned)n_tiles, 256, 0, stream>>>(ctx->count[0], ctx->count[1], C, ctx->block_sums,
                                                         n_tiles);
    COMPTON_LAUNCH_CHECK(ctx, "k_scan_reduce");
    k_scan_blocks<<<1, 1024, 0, stream>>>(ctx->block_sums, n_tiles, ctx->n_pairs);
    COMPTON_LAUNCH_CHECK(ctx, "k_scan_blocks");

    const int64_t nb_e = (ne + kSortTile - 1) / kSortTile;
    const int64_t nb_g = (ng + kSortTile - 1) / kSortTile;
    ScanFinalArgs sf;
    sf.count_e = ctx->count[0];
    sf.count_g = ctx->count[1];
    sf.block_sums = ctx->block_sums;
    sf.n_tiles = n_tiles;
    sf.C = C;
    sf.n_e = ne;
    sf.n_g = ng;
    sf.off_e = ctx->off[0];
    sf.off_g = ctx->off[1];
    sf.cinfo = ctx->cinfo;
    sf.tile_cell = ctx->tile_cell;
    sf.stile_e = ctx->stile[0];
    sf.stile_g = ctx->stile[1];
    sf.nb_e = nb_e;
    sf.nb_g = nb_g;
    sf.n_pairs = ctx->n_pairs;
    sf.w_over_v = ctx->cfg.w_over_v;
    k_scan_final<<<(unsigned)n_tiles, 256, 0, stream>>>(sf);
    COMPTON_LAUNCH_CHECK(ctx, "k_scan_final");

    KeyScatterArgs ks;
    ks.cell[0] = e_in->cell_dev;
    ks.cell[1] = g_in->cell_dev;
    ks.id[0] = e_in->id_dev;
    ks.id[1] = g_in->id_dev;
    ks.n[0] = ne;
    ks.n[1] = ng;
    for (int s = 0; s < 2; ++s) {
        ks.off[s] = ctx->off[s];
        ks.cursor[s] = ctx->count[s];
        ks.rec[s] = ctx->rec[s];
    }
    ks.C = C;
    ks.seed = ctx->cfg.seed;
    ks.step = step;
    k_key_scatter<<<pgrid, 256, 0, stream>>>(ks);
    COMPTON_LAUNCH_CHECK(ctx, "k_key_scatter");

    if (nb_e + nb_g > 0) {
        SortGatherArgs sg;
        const compton_species* ins[2] = {e_in, g_in};
        compton_species* outs[2] = {e_out, g_out};
        for (int s = 0; s < 2; ++s) {
            sg.in_u[s][0] = ins[s]->ux_dev;
            sg.in_u[s][1] = ins[s]->uy_dev;
            sg.in_u[s][2] = ins[s]->uz_dev;
            sg.in_cell[s] = ins[s]->cell_dev;
            sg.in_id[s] = ins[s]->id_dev;
            sg.out_u[s][0] = outs[s]->ux_dev;
            sg.out_u[s][1] = outs[s]->uy_dev;
            sg.out_u[s][2] = outs[s]->uz_dev;
            sg.out_cell[s] = outs[s]->cell_dev;
            sg.out_id[s] = outs[s]->id_dev;
            sg.rec[s] = ctx->rec[s];
            sg.off[s] = ctx->off[s];
            sg.stile[s] = ctx->stile[s];
        }
        sg.nb_e = nb_e;
        const int smem = kSortCap * 16;
        COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sort_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem));
        k_sort_gather<<<(unsigned)(nb_e + nb_g), kSortThreads, smem, stream>>>(sg);
        COMPTON_LAUNCH_CHECK(ctx, "k_sort_gather");
    }
    return COMPTON_OK;
}

}  // namespace compton
