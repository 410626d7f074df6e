// noalloc.cu -- per-cell offsets of one species without any device allocation.
//
// The binning of compton_bin_pairs histograms the cell indices and scans the
// counts into per-cell offsets, in scratch memory that compton_init allocates.
// Some callers cannot allocate device memory at the point where they need the
// offsets: a particle-in-cell code whose memory manager owns every byte of
// device memory up front, or a time-step loop that must not allocate (an
// allocation can synchronise the device or fail midway through a run).  This
// file gives them compton_cell_offsets_noalloc, which keeps its counts in a
// file-scope device array instead:
//   * the array holds kStaticMaxCells int32 counts and one partial sum per
//     strip of 4096 cells (4 MiB + 1 KiB); every GPU that loads the library
//     keeps it until the process exits;
//   * host code must not pass the array's name to a kernel (in host code it is
//     a host-side stand-in, not a device address): its device address is
//     obtained once per device with cudaGetSymbolAddress, with that device
//     current, on the first call made on that device -- so make that first call
//     before any stream capture.  A cudaDeviceReset unloads the library's
//     device code and makes the address kept for that device stale, so the
//     entry point must not be called after a reset in the same process;
//   * every call shares the array: the counts are cleared at the start of each
//     call, and calls whose work overlaps on the GPU (different streams,
//     threads or devices sharing a context) race on it and must be ordered by
//     the caller.
#include <mutex>

#include "ctx.hpp"

namespace compton {
namespace {

constexpr int64_t kStaticMaxCells = int64_t(1) << 20;
// The scan works on strips of 4096 counts (1024 threads x 4 consecutive
// counts each); one partial sum per strip follows the counts in the array.
constexpr int kStripThreads = 1024;
constexpr int kStrip = 4 * kStripThreads;
constexpr int64_t kMaxStrips = kStaticMaxCells / kStrip;
static __device__ __align__(256) int32_t g_cell_counts[kStaticMaxCells + kMaxStrips];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t* g_counts_addr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};

// Histogram with warp-aggregated atomics; indices outside [0, n_cells) are skipped.
__global__ void k_count_static(const int32_t* __restrict__ cell, int64_t n, int64_t n_cells, int32_t* count)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + 31) / 32 * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        int c = -1;
        if (i < n) {
            const int32_t ci = cell[i];
            if (ci >= 0 && (int64_t)ci < n_cells) c = ci;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && (threadIdx.x & 31u) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&count[c], __popc(peers));
    }
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_tot, int32_t* total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t inc = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t t = warp_tot[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += o;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    *total = warp_tot[31];
    return (warp > 0 ? warp_tot[warp - 1] : 0) + inc - v;
}

// Four consecutive counts of this thread in strip blockIdx.x (zero past n_cells):
// neighbouring threads read neighbouring 16 bytes, so a warp's loads coalesce.
__device__ __forceinline__ void load4(const int32_t* __restrict__ count, int64_t n_cells, int32_t v[4])
{
    const int64_t c0 = (int64_t)blockIdx.x * kStrip + 4 * (int64_t)threadIdx.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = c0 + j < n_cells ? count[c0 + j] : 0;
}

// Pass 1: the sum of each strip's counts.
__global__ void __launch_bounds__(kStripThreads) k_strip_sum(const int32_t* __restrict__ count, int64_t n_cells,
                                                             int32_t* __restrict__ strip_sum)
{
    __shared__ int32_t warp_tot[32];
    int32_t v[4];
    load4(count, n_cells, v);
    int32_t total;
    block_exclusive_scan(v[0] + v[1] + v[2] + v[3], warp_tot, &total);
    if (threadIdx.x == 0) strip_sum[blockIdx.x] = total;
}

// Pass 2 (one CTA): exclusive scan of the strip sums in place; off[n_cells] = total.
__global__ void __launch_bounds__(kStripThreads) k_strip_scan(int32_t* __restrict__ strip_sum, int64_t n_strips,
                                                              int64_t n_cells, int32_t* __restrict__ off)
{
    __shared__ int32_t warp_tot[32];
    const int tid = threadIdx.x;
    const int32_t v = tid < n_strips ? strip_sum[tid] : 0;
    int32_t total;
    const int32_t ex = block_exclusive_scan(v, warp_tot, &total);
    if (tid < n_strips) strip_sum[tid] = ex;
    if (tid == 0) off[n_cells] = total;
}

// Pass 3: each strip's running offsets, from its prefix and a block scan.
__global__ void __launch_bounds__(kStripThreads) k_strip_final(const int32_t* __restrict__ count, int64_t n_cells,
                                                               const int32_t* __restrict__ strip_prefix,
                                                               int32_t* __restrict__ off)
{
    __shared__ int32_t warp_tot[32];
    int32_t v[4];
    load4(count, n_cells, v);
    int32_t total;
    int32_t run = strip_prefix[blockIdx.x] + block_exclusive_scan(v[0] + v[1] + v[2] + v[3], warp_tot, &total);
    const int64_t c0 = (int64_t)blockIdx.x * kStrip + 4 * (int64_t)threadIdx.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (c0 + j < n_cells) off[c0 + j] = run;
        run += v[j];
    }
}

}  // namespace
}  // namespace compton

extern "C" compton_status compton_cell_offsets_noalloc(const int32_t* cell_dev, int64_t n, int64_t n_cells,
                                                       int32_t* off_out_dev, compton_stream_t stream)
{
    using namespace compton;
    if (n < 0 || n > INT32_MAX || n_cells <= 0 || !off_out_dev || (n > 0 && !cell_dev)) return COMPTON_EINVAL;
    if (n_cells > kStaticMaxCells) return COMPTON_ERANGE;  // beyond the static array
    // an error left by the caller's own earlier work is not this call's: it
    // is cleared here so that the check after the launches sees only ours
    cudaGetLastError();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return COMPTON_ECUDA;
    }
    int32_t* counts = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_counts_addr[dev]) {
            void* p = nullptr;
            int m = 0;
            if (cudaGetSymbolAddress(&p, g_cell_counts) != cudaSuccess || !p ||
                cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m <= 0) {
                cudaGetLastError();
                return COMPTON_ECUDA;
            }
            g_counts_addr[dev] = static_cast<int32_t*>(p);
            g_sm_count[dev] = m;
        }
        counts = g_counts_addr[dev];
        sms = g_sm_count[dev];
    }
    int32_t* strip_sum = counts + kStaticMaxCells;
    const int64_t n_strips = (n_cells + kStrip - 1) / kStrip;
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_cells, stream) != cudaSuccess) {
        cudaGetLastError();
        return COMPTON_ECUDA;
    }
    if (n > 0) {
        int64_t blocks = (n + 255) / 256;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;  // 8 CTAs of 256 per SM, grid-stride
        k_count_static<<<(unsigned)blocks, 256, 0, stream>>>(cell_dev, n, n_cells, counts);
    }
    k_strip_sum<<<(unsigned)n_strips, kStripThreads, 0, stream>>>(counts, n_cells, strip_sum);
    k_strip_scan<<<1, kStripThreads, 0, stream>>>(strip_sum, n_strips, n_cells, off_out_dev);
    k_strip_final<<<(unsigned)n_strips, kStripThreads, 0, stream>>>(counts, n_cells, strip_sum, off_out_dev);
    if (cudaGetLastError() != cudaSuccess) return COMPTON_ECUDA;
    return COMPTON_OK;
}
