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
//   * the array holds kStaticMaxCells int32 counts (4 MiB); every GPU that
//     loads the library keeps it until the process exits;
//   * host code must not pass the array's name to a kernel (in host code it is
//     a host-side stand-in, not a device address): its device address is
//     obtained once per device with cudaGetSymbolAddress, with that device
//     current, on the first call made on that device -- so make that first call
//     before any stream capture;
//   * every call shares the array: the counts are cleared at the start of each
//     call, and calls whose work overlaps on the GPU (different streams,
//     threads or devices sharing a context) race on it and must be ordered by
//     the caller.
#include <mutex>

#include "ctx.hpp"

namespace compton {
namespace {

constexpr int64_t kStaticMaxCells = int64_t(1) << 20;
static __device__ __align__(256) int32_t g_cell_counts[kStaticMaxCells];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
int32_t* g_counts_addr[kMaxDevices] = {nullptr};

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

// Exclusive scan of the counts by one CTA of 1024 threads: each thread sums a
// contiguous chunk, the chunk sums are scanned across the block, then each
// thread writes its chunk's running offsets.  off[n_cells] = total.
__global__ void __launch_bounds__(1024) k_scan_static(const int32_t* __restrict__ count, int64_t n_cells,
                                                      int32_t* __restrict__ off)
{
    __shared__ int64_t warp_tot[32];
    const int tid = threadIdx.x;
    const int64_t chunk = (n_cells + 1023) / 1024;
    const int64_t c0 = tid * chunk;
    const int64_t c1 = c0 + chunk < n_cells ? c0 + chunk : n_cells;
    int64_t sum = 0;
    for (int64_t c = c0; c < c1; ++c) sum += count[c];
    int64_t inc = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if ((tid & 31) >= d) inc += o;
    }
    if ((tid & 31) == 31) warp_tot[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
        int64_t t = warp_tot[tid];
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(0xffffffffu, t, d);
            if (tid >= d) t += o;
        }
        warp_tot[tid] = t;
    }
    __syncthreads();
    int64_t run = (tid >= 32 ? warp_tot[(tid >> 5) - 1] : 0) + inc - sum;
    for (int64_t c = c0; c < c1; ++c) {
        off[c] = (int32_t)run;
        run += count[c];
    }
    if (tid == 1023) off[n_cells] = (int32_t)(warp_tot[31]);
}

}  // namespace
}  // namespace compton

extern "C" compton_status compton_cell_offsets_noalloc(const int32_t* cell_dev, int64_t n, int64_t n_cells,
                                                       int32_t* off_out_dev, compton_stream_t stream)
{
    using namespace compton;
    if (n < 0 || n > INT32_MAX || n_cells <= 0 || !off_out_dev || (n > 0 && !cell_dev)) return COMPTON_EINVAL;
    if (n_cells > kStaticMaxCells) return COMPTON_ERANGE;  // beyond the static array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return COMPTON_ECUDA;
    }
    int32_t* counts = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_counts_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_cell_counts) != cudaSuccess || !p) {
                cudaGetLastError();
                return COMPTON_ECUDA;
            }
            g_counts_addr[dev] = static_cast<int32_t*>(p);
        }
        counts = g_counts_addr[dev];
    }
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_cells, stream) != cudaSuccess) {
        cudaGetLastError();
        return COMPTON_ECUDA;
    }
    if (n > 0) {
        int64_t blocks = (n + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_count_static<<<(unsigned)blocks, 256, 0, stream>>>(cell_dev, n, n_cells, counts);
    }
    k_scan_static<<<1, 1024, 0, stream>>>(counts, n_cells, off_out_dev);
    if (cudaGetLastError() != cudaSuccess) return COMPTON_ECUDA;
    return COMPTON_OK;
}
