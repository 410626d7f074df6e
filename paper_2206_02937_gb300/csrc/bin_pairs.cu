// bin_pairs.cu -- binning and random in-cell pairing (arXiv 2206.02937,
// Sec. 3.1, first step: "the simulation space is divided into collision
// cells, in which the particles are binned; from this binning a list of
// colliding leptons and photons is produced for each cell").
//
// Six launches per call, both species in each:
//   k_count        histogram of cell indices by run boundaries, order check
//   k_scan_reduce  per-tile sums of N_e,c, N_g,c and M_c = min(N_e,c, N_g,c)
//   k_scan_blocks  exclusive scan of the tile sums (one CTA)
//   k_scan_final   per-cell offsets, CellInfo, tile maps; resets the cursors
//   k_place        input not in cell order only: Philox key per particle,
//                  (key, id, momentum) record placed in its cell's segment
//                  (arbitrary order inside the segment)
//   k_sort_gather  per-cell sort by (key, id) in shared memory (a bucket
//                  sort of each tile of whole cells), each particle written
//                  to its sorted position
// The order within a cell depends only on (key, id): the atomics of k_place
// decide where a record lands inside its segment, and the sort removes that
// freedom.
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {
namespace {

constexpr int kSortThreads = 128;
constexpr int kPlaceThreads = 1024;  // threads per placement CTA
constexpr int kCountThreads = 1024;  // threads per histogram CTA (256, 512: 1 us slower)

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// ---------------------------------------------------------------------------
// Histogram and order check.  Every maximal run of equal in-range cell
// indices at positions [i_s, i_e] adds i_e + 1 - i_s to its cell: the first
// element adds -i_s, the last i_e + 1 (one atomic when they coincide).  This
// counts any input exactly (a cell's runs sum to its size; int32 wrap-around
// cancels), costs one atomic per element of shuffled input and two per run
// of input in cell order.  Each thread takes four consecutive positions with
// one vector load; the neighbours across threads come by shuffle.
// unsorted[s] is set if a cell index descends or lies outside [0, C): only
// then does the placement run.
// ---------------------------------------------------------------------------
template <typename Idx>
__device__ __forceinline__ int4 load_cells4(const int32_t* __restrict__ cell, Idx i, Idx n, bool vec)
{
    if (vec && i + 3 < n) return *reinterpret_cast<const int4*>(cell + i);  // 16-byte aligned: i % 4 == 0
    int4 v = make_int4(-1, -1, -1, -1);
    if (i < n) v.x = cell[i];
    if (i + 1 < n) v.y = cell[i + 1];
    if (i + 2 < n) v.z = cell[i + 2];
    if (i + 3 < n) v.w = cell[i + 3];
    return v;
}

// Positions in Idx: 32-bit when every position the grid visits fits (the
// launch checks), else 64-bit.
template <typename Idx>
__global__ void __launch_bounds__(kCountThreads) k_count(const int32_t* __restrict__ cell_e, int64_t n_e,
                                                        const int32_t* __restrict__ cell_g, int64_t n_g, int64_t C,
                                                        int32_t* __restrict__ count_e, int32_t* __restrict__ count_g,
                                                        int32_t* __restrict__ unsorted, DeviceStats* stats)
{
    const int s = blockIdx.y;
    const int32_t* __restrict__ cell = s == 0 ? cell_e : cell_g;
    const Idx n = (Idx)(s == 0 ? n_e : n_g);
    int32_t* __restrict__ count = s == 0 ? count_e : count_g;
    const unsigned lane = lane_id();
    const Idx stride = (Idx)gridDim.x * (Idx)blockDim.x * 4;
    const Idx n_round = (n + 127) / 128 * 128;  // whole warps in every iteration
    const bool vec = (reinterpret_cast<uintptr_t>(cell) & 15u) == 0;
    // cell indices are int32, so C above 2^31 admits every non-negative one
    const uint32_t C32 = C > 0x80000000ll ? 0x80000000u : (uint32_t)C;
    bool disorder = false, bad = false;
    // the next group's loads are issued before this group is processed, so
    // two groups per thread are in flight
    auto edge = [&](Idx j0) -> int32_t {
        if (lane == 0) return (j0 > 0 && j0 - 1 < n) ? cell[j0 - 1] : -1;
        if (lane == 31) return j0 + 4 < n ? cell[j0 + 4] : -1;
        return -1;
    };
    Idx i0 = ((Idx)blockIdx.x * (Idx)blockDim.x + (Idx)threadIdx.x) * 4;
    int4 q = make_int4(-1, -1, -1, -1);
    int32_t e = -1;
    if (i0 < n_round) {
        q = load_cells4(cell, i0, n, vec);
        e = edge(i0);
    }
    for (; i0 < n_round; i0 += stride) {
        int4 qn = make_int4(-1, -1, -1, -1);
        int32_t en = -1;
        if (i0 + stride < n_round) {
            qn = load_cells4(cell, i0 + stride, n, vec);
            en = edge(i0 + stride);
        }
        const int32_t v[4] = {q.x, q.y, q.z, q.w};
        int32_t prev = __shfl_up_sync(0xffffffffu, v[3], 1);
        int32_t next = __shfl_down_sync(0xffffffffu, v[0], 1);
        if (lane == 0) prev = e;
        if (lane == 31) next = e;
        q = qn;
        e = en;
        if (i0 > 0 && i0 + 4 < n) {
            // interior group: no end of the array in reach, 32-bit positions
            // (the counts wrap in int32 as in the general path)
            const int32_t base = (int32_t)i0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int32_t c = v[j];
                const int32_t pc = j == 0 ? prev : v[j - 1];
                const int32_t nc = j == 3 ? next : v[j + 1];
                const bool ok = (uint32_t)c < C32;
                bad |= !ok;
                disorder |= pc > c;
                const bool first = pc != c, last = nc != c;
                if (ok && (first || last))
                    atomicAdd(&count[c], (last ? base + j + 1 : 0) - (first ? base + j : 0));
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const Idx i = i0 + j;
            if (i >= n) break;
            const int32_t c = v[j];
            const int32_t pc = j == 0 ? prev : v[j - 1];
            const int32_t nc = j == 3 ? next : v[j + 1];
            const bool ok = c >= 0 && (int64_t)c < C;
            bad |= !ok;
            disorder |= i > 0 && pc > c;
            const bool first = ok && (i == 0 || pc != c);
            const bool last = ok && (i + 1 == n || nc != c);
            if (first || last)
                atomicAdd(&count[c], (last ? (int32_t)(i + 1) : 0) - (first ? (int32_t)i : 0));
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&stats->error_flags, (unsigned long long)kErrCellRange);
    if (__any_sync(0xffffffffu, disorder || bad) && lane == 0) atomicOr(&unsorted[s], 1);
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
    const int64_t c0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    Tri v{0, 0, 0};
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
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
    const int64_t c0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int32_t ne[kScanPer], ng[kScanPer];
    Tri v{0, 0, 0};
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
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
    for (int j = 0; j < kScanPer; ++j) {
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
        a.count_e[c] = 0;  // becomes the insertion cursor of k_place
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
// Keyed placement of input not yet in cell order: each particle's record
// (Philox key, id, momentum, weight if any) goes to off[c] + cursor.  A record fills one
// aligned 32-byte sector, written as two 16-byte stores, so the scattered
// writes never leave partly written sectors behind.  Input already in cell
// order (k_count found no descent and no bad index) skips this kernel: the
// sort then reads the input arrays in place.
// ---------------------------------------------------------------------------
struct PlaceArgs {
    const int32_t* cell[2];
    const uint32_t* id[2];
    const float* u[2][3];
    const float* w[2];  // per-particle weights, or nullptr
    int64_t n[2];
    const int32_t* off[2];
    int32_t* cursor[2];
    const int32_t* unsorted;
    SortRec* rec[2];
    int64_t C;
    uint64_t seed, step;
};

__device__ __forceinline__ void store_rec(SortRec* r, uint32_t key, uint32_t pid, float ux, float uy, float uz,
                                          float w)
{
    uint4* q = reinterpret_cast<uint4*>(r);
    q[0] = make_uint4(key, pid, __float_as_uint(ux), __float_as_uint(uy));
    q[1] = make_uint4(__float_as_uint(uz), __float_as_uint(w), 0u, 0u);
}

// The weight a record carries (its first padding word).
__device__ __forceinline__ float rec_weight(const SortRec* r) { return __uint_as_float(r->pad[0]); }

__global__ void __launch_bounds__(kPlaceThreads) k_place(PlaceArgs a)
{
    const int s = blockIdx.y;
    if (a.unsorted[s] == 0) return;
    const int64_t n = a.n[s];
    const int32_t* __restrict__ cell = a.cell[s];
    const uint32_t* __restrict__ id = a.id[s];
    const float* __restrict__ u0 = a.u[s][0];
    const float* __restrict__ u1 = a.u[s][1];
    const float* __restrict__ u2 = a.u[s][2];
    const float* __restrict__ wt = a.w[s];
    const int32_t* __restrict__ off = a.off[s];
    int32_t* __restrict__ cursor = a.cursor[s];
    SortRec* __restrict__ rec = a.rec[s];
    const uint32_t stream = s == 0 ? kStreamPairE : kStreamPairG;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + 31) / 32 * 32;
    const unsigned lane = lane_id();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        int c = -1;
        uint32_t key = 0, pid = 0;
        if (i < n) {
            const int32_t ci = cell[i];
            if (ci >= 0 && (int64_t)ci < a.C) {
                c = ci;
                pid = id[i];
                key = draw(a.seed, a.step, stream, pid).r0;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (c >= 0 && lane == (unsigned)leader) base = atomicAdd(&cursor[c], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        if (c >= 0) {
            const int64_t slot = (int64_t)off[c] + base + __popc(peers & ((1u << lane) - 1u));
            store_rec(rec + slot, key, pid, u0[i], u1[i], u2[i], wt ? wt[i] : 0.0f);
        }
    }
}

// ---------------------------------------------------------------------------
// Per-cell sort by (key, id) and copy into sorted order.
//
// Keys are uniform 32-bit Philox words, so within a cell of n particles the
// bucket floor(key * n / 2^32) is monotone in the key and holds about one
// particle.  A sort tile (whole cells, at most kSortCap particles) gives cell
// c the buckets [a_c, a_c + n_c) at its own positions in the tile, so one
// counting sort over all buckets of the tile sorts every cell at once: a
// histogram in shared memory, one block-wide exclusive scan (its value at the
// start of a cell's buckets is a_c), placement by bucket, and an exact rank
// by (key, id) inside each bucket, after which each element is written to its
// sorted position (entries of neighbouring threads lie in neighbouring
// buckets, so a warp's writes stay within a few sectors).  O(1) work per
// particle, every lane busy whatever the cell sizes.
// ---------------------------------------------------------------------------
struct SortGatherArgs {
    const float* in_u[2][3];
    const uint32_t* in_id[2];
    const float* in_w[2];  // per-particle weights, or nullptr
    float* out_w[2];
    float* out_u[2][3];
    int32_t* out_cell[2];
    uint32_t* out_id[2];
    SortRec* rec[2];
    const int32_t* off[2];
    const int32_t* stile[2];
    const int32_t* unsorted;
    int64_t nb_e;
    uint64_t seed, step;
};

// Where a species' particles are read from: the placed records, or (input in
// cell order) the input arrays, with keys drawn from the ids.
struct SortSrc {
    const SortRec* rec;  // nullptr: read the input arrays in place
    const uint32_t* id;
    const float* u[3];
    const float* w;      // weights (in place), or nullptr
    uint64_t seed, step;
    uint32_t stream;
};

// The order inside a cell is by (key, id), with the tile slot breaking ties
// between equal ids (invalid input), so the order is total and every sort
// yields a permutation.

__device__ __forceinline__ int bucket_of(uint32_t key, int n) { return (int)__umulhi(key, (uint32_t)n); }

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct SortSmem {
    uint32_t* id;     // [cap] particle id of each tile slot
    int32_t* cnt;     // [kBucketsPerSlot * cap] bucket counts, then starts, then ends
    uint32_t* cmap;   // [cap] a_c | n_c << 16 of the slot's cell; after the
                      // histogram, the keys in bucket order
    uint16_t* ptmp;   // [cap] tile slots grouped by bucket
    uint16_t* pbk;    // [cap] their buckets
    float* us[3];     // [cap] momenta staged from global memory
};

// Placed record gi to tile slot i: momentum and id into shared memory; the
// key is returned.
__device__ __forceinline__ uint32_t fetch_rec(const SortSrc& t, const SortSmem& m, int64_t gi, int i)
{
    const uint4* q = reinterpret_cast<const uint4*>(t.rec + gi);
    const uint4 r0 = q[0], r1 = q[1];
    m.us[0][i] = __uint_as_float(r0.z);
    m.us[1][i] = __uint_as_float(r0.w);
    m.us[2][i] = __uint_as_float(r1.x);
    m.id[i] = r0.y;
    return r0.x;
}

// Buckets per tile slot: a cell of n particles takes kBucketsPerSlot * n
// buckets, so a bucket holds Poisson(1 / kBucketsPerSlot) particles.
constexpr int kBucketsPerSlot = 1;

// Block-wide exclusive scan of cnt[0 .. R) in place (R <= kBucketsPerSlot *
// kSortCap).
__device__ __forceinline__ void block_scan_counts(int32_t* cnt, int R)
{
    constexpr int kPer = (kBucketsPerSlot * kSortCap + kSortThreads - 1) / kSortThreads;
    __shared__ int32_t warp_tot[kSortThreads / 32];
    const int tid = threadIdx.x, lane = (int)lane_id(), w = tid >> 5;
    const int b0 = tid * kPer;
    int v[kPer];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = b0 + k < R ? cnt[b0 + k] : 0;
        sum += v[k];
    }
    int inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < kSortThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += o;
        }
        if (lane < kSortThreads / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int run = (w > 0 ? warp_tot[w - 1] : 0) + inc - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (b0 + k < R) cnt[b0 + k] = run;
        run += v[k];
    }
}

// Sort the tile of cells [c0, c1) (positions o0 .. o0 + R of species s) with
// the whole block.
__device__ __forceinline__ void sort_tile_block(const SortGatherArgs& g, int s, const SortSrc& t, const SortSmem& m,
                                                int64_t c0, int64_t c1, int64_t o0, int R)
{
    const int tid = threadIdx.x, lane = (int)lane_id(), w = tid >> 5;
    const int32_t* __restrict__ off = g.off[s];
    constexpr int kPer = (kSortCap + kSortThreads - 1) / kSortThreads;
    uint32_t key[kPer], pid[kPer];
    // input in cell order: issue the tile's loads first, so they are in
    // flight while the cell map is built
    if (!t.rec) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kSortThreads;
            if (i < R) {
                cp_async4(&m.us[0][i], t.u[0] + o0 + i);
                cp_async4(&m.us[1][i], t.u[1] + o0 + i);
                cp_async4(&m.us[2][i], t.u[2] + o0 + i);
                pid[k] = t.id[o0 + i];
            }
        }
    }
    // the tile's cell offsets, staged once (in the placement buffers, unused
    // until later) when they fit; the bucket counters cleared
    const int n_cells = (int)(c1 - c0);
    int32_t* offs = reinterpret_cast<int32_t*>(m.ptmp);
    const bool staged = n_cells < kSortCap;
    if (staged)
        for (int i = tid; i <= n_cells; i += kSortThreads) offs[i] = off[c0 + i] - (int32_t)o0;
    for (int i = tid; i < kBucketsPerSlot * R; i += kSortThreads) m.cnt[i] = 0;
    __syncthreads();
    // cell of every position (warp per cell) and the output cell indices
    for (int64_t c = c0 + w; c < c1; c += kSortThreads / 32) {
        const int a = staged ? offs[c - c0] : off[c] - (int32_t)o0;
        const int n = (staged ? offs[c - c0 + 1] : off[c + 1] - (int32_t)o0) - a;
        for (int j = lane; j < n; j += 32) {
            m.cmap[a + j] = (uint32_t)a | ((uint32_t)n << 16);
            g.out_cell[s][o0 + a + j] = (int32_t)c;
        }
    }
    // keys (and, from placed records, momenta)
    if (t.rec) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kSortThreads;
            if (i < R) key[k] = fetch_rec(t, m, o0 + i, i);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = tid + k * kSortThreads;
            if (i < R) {
                key[k] = draw(t.seed, t.step, t.stream, pid[k]).r0;
                m.id[i] = pid[k];
            }
        }
    }
    __syncthreads();
    // bucket histogram; the slots' buckets stay in registers, two 16-bit
    // buckets to a register
    uint32_t bk2[(kPer + 1) / 2];
#pragma unroll
    for (int k = 0; k < (kPer + 1) / 2; ++k) bk2[k] = 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = tid + k * kSortThreads;
        if (i < R) {
            const uint32_t cm = m.cmap[i];
            const uint32_t b = kBucketsPerSlot * (cm & 0xffffu) +
                               (uint32_t)bucket_of(key[k], kBucketsPerSlot * (int)(cm >> 16));
            bk2[k >> 1] |= b << ((k & 1) * 16);
            atomicAdd(&m.cnt[b], 1);
        }
    }
    __syncthreads();
    block_scan_counts(m.cnt, kBucketsPerSlot * R);
    __syncthreads();
    // slots, keys and buckets grouped by bucket (the cell map is no longer
    // needed); afterwards cnt[b] = end of bucket b
    uint32_t* pkey = m.cmap;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = tid + k * kSortThreads;
        if (i < R) {
            const uint32_t b = (bk2[k >> 1] >> ((k & 1) * 16)) & 0xffffu;
            const int pos = atomicAdd(&m.cnt[b], 1);
            m.ptmp[pos] = (uint16_t)i;
            m.pbk[pos] = (uint16_t)b;
            pkey[pos] = key[k];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // exact rank inside each bucket, one thread per entry of the grouped list
    // (the end of bucket b - 1 is the start of bucket b, also across cells):
    // neighbouring threads read the same or neighbouring buckets, so a
    // bucket's keys reach them by broadcast; only a key that occurs twice
    // needs the ids (and, for equal ids, the slots) to break the tie
    for (int q = tid; q < R; q += kSortThreads) {
        const int b = m.pbk[q];
        const int lo = b == 0 ? 0 : m.cnt[b - 1];
        const int hi = m.cnt[b];
        const int i = m.ptmp[q];
        int fin = lo;
        if (hi - lo > 1) {
            const uint32_t ki = pkey[q];
            int less = 0, eq = 0;
            if (hi - lo <= 4) {
                // buckets hold Poisson(1) keys: up to four, a fixed unrolled
                // pass (no loop control, the same instructions in every lane)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (lo + r < hi) {
                        const uint32_t kr = pkey[lo + r];
                        less += kr < ki;
                        eq += kr == ki;
                    }
                }
            } else {
                for (int r = lo; r < hi; ++r) {
                    const uint32_t kr = pkey[r];
                    less += kr < ki;
                    eq += kr == ki;
                }
            }
            if (eq == 1) {
                fin = lo + less;
            } else {
                const uint32_t di = m.id[i];
                for (int r = lo; r < hi; ++r) {
                    const uint32_t kr = pkey[r];
                    const int jj = m.ptmp[r];
                    const uint32_t dj = m.id[jj];
                    fin += (kr < ki) | ((kr == ki) & ((dj < di) | ((dj == di) & (jj < i))));
                }
            }
        }
        // the element goes straight to its sorted position: neighbouring
        // threads hold neighbouring buckets, so the writes stay close
        const int64_t go = o0 + fin;
        g.out_u[s][0][go] = m.us[0][i];
        g.out_u[s][1][go] = m.us[1][i];
        g.out_u[s][2][go] = m.us[2][i];
        g.out_id[s][go] = m.id[i];
        // the weight is not staged: read once more where the tile came from
        // (a sector this block has just read)
        if (g.out_w[s]) g.out_w[s][go] = t.rec ? rec_weight(t.rec + o0 + i) : t.w[o0 + i];
    }
}

// A cell larger than the shared-memory capacity: records in global memory
// (materialised from the input first when the placement was skipped), each
// particle ranked against the whole cell by the block.
__device__ void sort_giant_cell(const SortGatherArgs& g, int s, const SortSrc& t, int64_t o, int64_t n, int32_t c)
{
    SortRec* rec = g.rec[s];
    if (!t.rec) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t pid = t.id[o + i];
            store_rec(rec + o + i, draw(t.seed, t.step, t.stream, pid).r0, pid, t.u[0][o + i], t.u[1][o + i],
                      t.u[2][o + i], t.w ? t.w[o + i] : 0.0f);
        }
        __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const SortRec ri = rec[o + i];
        int64_t rank = 0;
        for (int64_t j = 0; j < n; ++j) {
            const uint32_t kj = rec[o + j].key, dj = rec[o + j].id;
            rank += (kj < ri.key) | ((kj == ri.key) & ((dj < ri.id) | ((dj == ri.id) & (j < i))));
        }
        const int64_t p = o + rank;
        g.out_u[s][0][p] = ri.ux;
        g.out_u[s][1][p] = ri.uy;
        g.out_u[s][2][p] = ri.uz;
        g.out_cell[s][p] = c;
        g.out_id[s][p] = ri.id;
        if (g.out_w[s]) g.out_w[s][p] = rec_weight(&ri);
    }
    __syncthreads();
}

constexpr size_t kSortSmem = (size_t)kSortCap * (4 + 4 * kBucketsPerSlot + 4 + 12 + 2 + 2);

__global__ void __launch_bounds__(kSortThreads, 10) k_sort_gather(SortGatherArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem m;
    m.id = reinterpret_cast<uint32_t*>(smem_raw);
    m.cnt = reinterpret_cast<int32_t*>(m.id + kSortCap);
    m.cmap = reinterpret_cast<uint32_t*>(m.cnt + kBucketsPerSlot * kSortCap);
    m.us[0] = reinterpret_cast<float*>(m.cmap + kSortCap);
    m.us[1] = m.us[0] + kSortCap;
    m.us[2] = m.us[1] + kSortCap;
    m.ptmp = reinterpret_cast<uint16_t*>(m.us[2] + kSortCap);
    m.pbk = m.ptmp + kSortCap;

    const int s = (int64_t)blockIdx.x < g.nb_e ? 0 : 1;
    const int64_t b = s == 0 ? blockIdx.x : blockIdx.x - g.nb_e;
    const int32_t* __restrict__ off = g.off[s];
    const int64_t c0 = g.stile[s][b];
    const int64_t c1 = g.stile[s][b + 1];
    if (c1 <= c0) return;
    const int64_t o0 = off[c0];
    const int64_t R = (int64_t)off[c1] - o0;
    if (R <= 0) return;

    SortSrc t;
    const bool placed = g.unsorted[s] != 0;
    t.rec = placed ? g.rec[s] : nullptr;
    t.id = g.in_id[s];
    for (int k = 0; k < 3; ++k) t.u[k] = g.in_u[s][k];
    t.w = g.in_w[s];
    t.seed = g.seed;
    t.step = g.step;
    t.stream = s == 0 ? kStreamPairE : kStreamPairG;

    if (R <= kSortCap) {
        sort_tile_block(g, s, t, m, c0, c1, o0, (int)R);
        return;
    }
    // A cell range larger than shared memory: runs of whole cells that fit
    // are sorted block-wide one after another; a cell above the capacity
    // alone is ranked in global memory.
    for (int64_t c = c0; c < c1;) {
        const int64_t o = off[c];
        if ((int64_t)off[c + 1] - o > kSortCap) {
            __syncthreads();
            sort_giant_cell(g, s, t, o, (int64_t)off[c + 1] - o, (int32_t)c);
            ++c;
            continue;
        }
        int64_t e = c + 1;
        while (e < c1 && (int64_t)off[e + 1] - o <= kSortCap) ++e;
        __syncthreads();
        sort_tile_block(g, s, t, m, c, e, o, (int)((int64_t)off[e] - o));
        c = e;
    }
}

// CTAs per SM and species of the grid-stride histogram and placement (the
// launches' second grid dimension takes the two species).  The histogram
// runs in one wave of 1024-thread CTAs: 0.0394 ms on the 512^2 step against
// 0.0404 with four and 0.0435 with eight.  The placement keeps four: with
// two, binning shuffled input took 1.46 against 1.28 ms.
constexpr int kCountCtasPerSm = 2;
constexpr int kPlaceCtasPerSm = 4;

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
    // count[0], count[1] and unsorted lie in one block of the workspace
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->count[0], 0, sizeof(int32_t) * (ctx->unsorted + 2 - ctx->count[0]),
                                          stream));

    const int64_t nmax = ne > ng ? ne : ng;
    // grid-stride kernels: CTAs per SM of the histogram and the placement,
    // both in 1024-thread CTAs (the placement: as many threads as sixteen
    // 256-thread CTAs per SM, whose placement of shuffled input one wave of
    // fewer threads made 0.3 ms longer, in a quarter of the CTAs, so its
    // early exit for input in cell order is shorter)
    const dim3 cgrid(grid_for((nmax + 3) / 4, kCountThreads, ctx->n_sm * kCountCtasPerSm), 2);  // four per thread
    {
        TimedScope ts_(ctx, COMPTON_K_COUNT, stream);
        // 32-bit positions when the grid's last visited position fits
        const int64_t span = (nmax + 127) / 128 * 128 + (int64_t)cgrid.x * kCountThreads * 4;
        if (span < ((int64_t)1 << 31))
            k_count<int32_t><<<cgrid, kCountThreads, 0, stream>>>(e_in->cell_dev, ne, g_in->cell_dev, ng, C,
                                                                  ctx->count[0], ctx->count[1], ctx->unsorted,
                                                                  ctx->stats);
        else
            k_count<int64_t><<<cgrid, kCountThreads, 0, stream>>>(e_in->cell_dev, ne, g_in->cell_dev, ng, C,
                                                                  ctx->count[0], ctx->count[1], ctx->unsorted,
                                                                  ctx->stats);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_count");
    TimedScope scan_scope(ctx, COMPTON_K_SCAN, stream);
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
    // with per-particle weights a cell's density is its larger count; each
    // pair scales it by its own heavier weight
    const bool weighted = e_in->w_dev || g_in->w_dev;
    sf.w_over_v = weighted ? 1.0 : ctx->cfg.w_over_v;
    k_scan_final<<<(unsigned)n_tiles, 256, 0, stream>>>(sf);
    scan_scope.end();
    COMPTON_LAUNCH_CHECK(ctx, "k_scan_final");

    const dim3 pgrid(grid_for(nmax, kPlaceThreads, ctx->n_sm * kPlaceCtasPerSm), 2);
    PlaceArgs pa;
    const compton_species* ins[2] = {e_in, g_in};
    compton_species* outs[2] = {e_out, g_out};
    for (int s = 0; s < 2; ++s) {
        pa.cell[s] = ins[s]->cell_dev;
        pa.id[s] = ins[s]->id_dev;
        pa.u[s][0] = ins[s]->ux_dev;
        pa.u[s][1] = ins[s]->uy_dev;
        pa.u[s][2] = ins[s]->uz_dev;
        pa.w[s] = ins[s]->w_dev;
        pa.n[s] = ins[s]->n;
        pa.off[s] = ctx->off[s];
        pa.cursor[s] = ctx->count[s];
        pa.rec[s] = ctx->rec[s];
    }
    pa.unsorted = ctx->unsorted;
    pa.C = C;
    pa.seed = ctx->cfg.seed;
    pa.step = step;
    {
        TimedScope ts_(ctx, COMPTON_K_PLACE, stream);
        k_place<<<pgrid, kPlaceThreads, 0, stream>>>(pa);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_place");

    if (nb_e + nb_g > 0) {
        SortGatherArgs sg;
        for (int s = 0; s < 2; ++s) {
            sg.in_u[s][0] = ins[s]->ux_dev;
            sg.in_u[s][1] = ins[s]->uy_dev;
            sg.in_u[s][2] = ins[s]->uz_dev;
            sg.in_id[s] = ins[s]->id_dev;
            sg.in_w[s] = ins[s]->w_dev;
            sg.out_w[s] = ins[s]->w_dev ? outs[s]->w_dev : nullptr;
            sg.out_u[s][0] = outs[s]->ux_dev;
            sg.out_u[s][1] = outs[s]->uy_dev;
            sg.out_u[s][2] = outs[s]->uz_dev;
            sg.out_cell[s] = outs[s]->cell_dev;
            sg.out_id[s] = outs[s]->id_dev;
            sg.rec[s] = ctx->rec[s];
            sg.off[s] = ctx->off[s];
            sg.stile[s] = ctx->stile[s];
        }
        sg.unsorted = ctx->unsorted;
        sg.seed = ctx->cfg.seed;
        sg.step = step;
        sg.nb_e = nb_e;
        const int smem = (int)kSortSmem;
        COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_sort_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   smem));
        TimedScope ts_(ctx, COMPTON_K_SORT, stream);
        k_sort_gather<<<(unsigned)(nb_e + nb_g), kSortThreads, smem, stream>>>(sg);
        COMPTON_LAUNCH_CHECK(ctx, "k_sort_gather");
    }
    return COMPTON_OK;
}

}  // namespace compton
