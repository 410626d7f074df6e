// ctx.hpp -- host-side context of libcompton and the launch helpers shared by
// the .cu files of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>

#include "../../include/compton.h"

namespace compton {

// Tiling constants shared by the binning and scattering kernels.
constexpr int kScanTile = 2048;       // cells per scan tile (256 threads x 8)
constexpr int kSortTile = 4096;       // particles per sort tile (by cell start offsets)
constexpr int kSortCap = 6144;        // particles a sort CTA holds in shared memory
constexpr int kPairsPerTile = 1024;   // pairs per scatter CTA (256 threads x 4)
constexpr int kCellWindow = 512;      // cells of a scatter tile staged in shared memory

// Per-cell record written by the scan and read by the scatter kernel.
struct __align__(16) CellInfo {
    int32_t pair_off;  // first pair of the cell
    int32_t e_start;   // first sorted electron
    int32_t g_start;   // first sorted photon
    float dens;        // pair density n_c = max(N_e, N_g) * w_over_v
};

enum : unsigned { kErrCellRange = 1u, kErrCapacity = 2u };

struct DeviceStats {
    unsigned long long pairs_tested, scatters, mlp_fallbacks, error_flags;
};

}  // namespace compton

struct compton_ctx {
    compton_config cfg;
    char last_error[256];
    // single device allocation carved into the buffers below
    void* arena = nullptr;
    size_t arena_bytes = 0;
    // binning scratch (index 0 = electrons, 1 = photons)
    int32_t* count[2] = {nullptr, nullptr};      // [C] histogram, then insertion cursor
    int32_t* off[2] = {nullptr, nullptr};        // [C+1]
    uint2* rec[2] = {nullptr, nullptr};          // [max_particles] (key, source index)
    int32_t* stile[2] = {nullptr, nullptr};      // [max_sort_tiles+1] first cell of each sort tile
    int64_t* block_sums = nullptr;               // [3 * max_scan_tiles]
    compton::CellInfo* cinfo = nullptr;          // [C]
    int32_t* tile_cell = nullptr;                // [max_pair_tiles+1]
    int64_t* n_pairs = nullptr;                  // device scalar
    compton::DeviceStats* stats = nullptr;       // device counters
    int64_t max_scan_tiles = 0, max_sort_tiles = 0, max_pair_tiles = 0;
};

namespace compton {

inline compton_status set_cuda_error(compton_ctx* ctx, cudaError_t e, const char* where)
{
    if (ctx) {
        std::snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where, cudaGetErrorString(e));
    }
    return COMPTON_ECUDA;
}

#define COMPTON_CUDA_TRY(ctx, expr)                                  \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return compton::set_cuda_error((ctx), _e, #expr); \
    } while (0)

// Launch-error check after a kernel launch.
#define COMPTON_LAUNCH_CHECK(ctx, name)                              \
    do {                                                             \
        cudaError_t _e = cudaGetLastError();                         \
        if (_e != cudaSuccess) return compton::set_cuda_error((ctx), _e, name); \
    } while (0)

// Entry points implemented in the kernel files.
compton_status launch_bin_pairs(compton_ctx* ctx, const compton_species* e_in, const compton_species* g_in,
                                compton_species* e_out, compton_species* g_out, uint64_t step,
                                cudaStream_t stream);
compton_status launch_scatter_binned(compton_ctx* ctx, compton_species* e, compton_species* g,
                                     const compton_pairs* pairs, compton_mode mode, uint64_t step,
                                     float* prob_out, uint8_t* flag_out, cudaStream_t stream);
compton_status launch_scatter_pairs(compton_ctx* ctx, float* ux, float* uy, float* uz, float* kx, float* ky,
                                    float* kz, const float* n_dens, int64_t n, uint64_t seed, uint64_t step,
                                    compton_mode mode, float* prob_out, uint8_t* flag_out, cudaStream_t stream);
compton_status launch_kn_ratio(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                               const float* kx, const float* ky, const float* kz, int64_t n, float* r_out,
                               cudaStream_t stream);
compton_status launch_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n, float* cth,
                                   float* sth, float* ratio, cudaStream_t stream);

}  // namespace compton
