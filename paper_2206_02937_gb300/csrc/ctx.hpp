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
constexpr int kScanTile = 1024;       // cells per scan tile (256 threads x kScanPer; 2048 cells per
                                      // tile: the three scan kernels 25 us on 2^18 cells, 1024: 21 us)
constexpr int kScanPer = kScanTile / 256;
constexpr int kSortTile = 512;        // particles per sort tile (by cell start offsets)
constexpr int kSortCap = 640;         // particles a sort CTA holds in shared memory
constexpr int kPairsPerTile = 1024;   // pairs per scatter CTA (256 threads x 4)
constexpr int kCellWindow = 512;      // cells of a scatter tile staged in shared memory
constexpr int kMaxProbWarps = 8192;   // warps of the probability kernel (their accepted counts)

// Per-cell record written by the scan and read by the scatter kernel.
struct __align__(16) CellInfo {
    int32_t pair_off;  // first pair of the cell
    int32_t e_start;   // first sorted electron
    int32_t g_start;   // first sorted photon
    float dens;        // pair density n_c = max(N_e, N_g) * w_over_v; with per-particle
                       // weights max(N_e, N_g) alone (the pair takes max(w_e, w_g))
};

// A particle placed in its cell's segment by the binning: Philox key, id,
// momentum, padded to one aligned 32-byte sector.
struct __align__(32) SortRec {
    uint32_t key, id;
    float ux, uy, uz;
    uint32_t pad[3];
};

// A pair that passed its Bernoulli trial, waiting for its collision: sorted
// electron and photon index, rest-frame photon energy (negative when the
// probability came from the network), pair index (counter of its draws), and
// both momenta as they were read (so the collision kernel reads the list
// sequentially instead of the particle arrays at random); pad[0] holds the
// bits of F(x, 2) (sigma_KN's integral, which the angle sampler needs) when
// the producer computed it, else 0.
struct __align__(16) AcceptedPair {
    int32_t ie, ig;
    float x;
    uint32_t p;
    float u[3], k[3];
    uint32_t pad[2];
};

// A pair whose uniform passed the probability bound P_b = 1 - exp(-2 n dt)
// and whose probability must be evaluated: sorted electron and photon index,
// pair density, its uniform u0, pair index, and both momenta (read once,
// while the pair's tile is being filtered, so the later kernels read the
// list sequentially).
struct __align__(16) CandPair {
    int32_t ie, ig;
    float dens, u0;
    uint32_t p;
    float u[3], k[3];
    uint32_t pad;
};

// The Bernoulli decision made inside the network kernel (surrogate modes on
// tensor cores): time step, FP64 threshold of the analytic fallback, optional
// per-pair outputs.
struct MlpDecide {
    float dt, gamma64;
    float* prob_out;
    uint8_t* flag_out;
};

enum : unsigned { kErrCellRange = 1u, kErrCapacity = 2u, kErrTimeout = 4u };

struct DeviceStats {
    unsigned long long pairs_tested, scatters, mlp_fallbacks, error_flags;
};

// Surrogate network: 6 -> 64 -> 64 -> 64 -> 64 -> 1, parameter vector of
// 12993 floats (W0 64x6, b0, W1 64x64, b1, W2, b2, W3, b3, W4 1x64, b4).
constexpr int kMlpParams = 12993;
__host__ __device__ constexpr int mlp_off_w(int l)
{
    return l == 0 ? 0 : l == 1 ? 448 : l == 2 ? 4608 : l == 3 ? 8768 : 12928;
}
__host__ __device__ constexpr int mlp_off_b(int l)
{
    return l == 0 ? 384 : l == 1 ? 4544 : l == 2 ? 8704 : l == 3 ? 12864 : 12992;
}

// Device-side network state (all pointers into one context allocation).
struct MlpDev {
    float* theta;        // [kMlpParams] FP32 master parameters
    float* grad;         // [kMlpParams]
    float* adam_m;       // [kMlpParams]
    float* adam_v;       // [kMlpParams]
    void* wbf16;         // 4 x 8 KB BF16 tiles, 128-byte swizzled K-major
    void* whalf;         // inference image: 4 x 8 KB BF16 tiles of W / 2 (layer 0 with b / 2 as
                         // hi + lo in K columns 6, 7), then 3 x 2 KB blocks of b / 2 (hi, lo in K
                         // columns 0, 1) of layers 1-3, 32-byte swizzled K-major
    void* wfp8;          // 4 x 8 KB E4M3 tiles (K padded to 128)
    float* wt32;         // 4 x 64 x 64 transposed FP32 weights
    float* bias;         // 4 x 64
    float* w4;           // 64
    float* b4;           // 1
    float* scale_w;      // 4 per-tensor FP8 weight scales
    float* scale_w_inv;  // 4
    float* scale_a_inv;  // 4: 1 / FP8 activation scale of each layer input
    float* loss;         // [2] weighted |error| sum and weight sum of the last step
    float* amax;         // [4] calibration: max |input| of each hidden layer
    float* edges;        // [257] data-balancing bin edges
    int* hist;           // [256] data-balancing counts
    float fs[4];         // feature scales s_u, n_u, s_k, n_k
    int32_t feat_mode;   // compton_features: momenta or invariants
    // training range: pairs outside it take the analytic probability
    float range_g2max;   // gamma^2 at most
    float range_e2min;   // eps^2 at least
    float range_e2max;   // eps^2 at most
};

// Whether a pair lies in the network's training range (gamma^2 = g2, eps^2 = e2).
__host__ __device__ inline bool mlp_in_range(const MlpDev& m, float g2, float e2)
{
    return g2 <= m.range_g2max && e2 >= m.range_e2min && e2 <= m.range_e2max;
}

// The paper's own network (9-12-9 ReLU, sigmoid): 337 parameters.
constexpr int kPnetParams = 337;
struct PnetDev {
    float* theta;   // [kPnetParams]
    float* grad;    // [kPnetParams], divided by the weight sum after a step
    float* adam_m;  // [kPnetParams]
    float* adam_v;  // [kPnetParams]
    float* loss;    // [2] weighted |error| sum, weight sum of the last step
    float fs[4];    // feature scales s_u, n_u, s_k, n_k
    float range[3]; // training range: gamma^2 max, eps^2 min, eps^2 max
    int64_t step;   // Adam steps taken
};

struct ServeEngine;

// Optional per-kernel timing (compton_kernel_timing): every launch of a slot
// records a CUDA event pair on its stream into a ring of kTimingRing pairs.
constexpr int kTimedSlots = COMPTON_N_TIMED;
constexpr int kTimingRing = 64;
struct KernelTiming {
    bool on = false;
    cudaEvent_t ev[kTimedSlots][kTimingRing][2];
    int64_t n[kTimedSlots];
};

}  // namespace compton

struct compton_ctx {
    compton_config cfg;
    char last_error[256];
    int n_sm = 1;  // multiprocessors of the context's device (grid sizes)
    // single device allocation carved into the buffers below
    void* arena = nullptr;
    size_t arena_bytes = 0;
    // binning scratch (index 0 = electrons, 1 = photons)
    int32_t* count[2] = {nullptr, nullptr};      // [C] histogram, then insertion cursor
    int32_t* off[2] = {nullptr, nullptr};        // [C+1]
    compton::SortRec* rec[2] = {nullptr, nullptr};  // [max_particles] placed records
    int32_t* unsorted = nullptr;                 // [2] set when a species' input is not in cell order
    int32_t* stile[2] = {nullptr, nullptr};      // [max_sort_tiles+1] first cell of each sort tile
    int64_t* block_sums = nullptr;               // [3 * max_scan_tiles]
    compton::CellInfo* cinfo = nullptr;          // [C]
    int32_t* tile_cell = nullptr;                // [max_pair_tiles+1]
    int64_t* n_pairs = nullptr;                  // device scalar
    compton::AcceptedPair* accepted = nullptr;   // [accepted_cap] pairs that passed their trial
    uint32_t* n_accepted = nullptr;              // device scalar
    uint32_t* warp_acc = nullptr;                // [kMaxProbWarps] accepted pairs per probability region
    int64_t accepted_cap = 0;                    // max(max_particles, 2^20)
    compton::CandPair* cand = nullptr;           // [accepted_cap] candidates of the surrogate modes
    uint32_t* n_cand = nullptr;                  // device scalar
    compton::DeviceStats* stats = nullptr;       // device counters
    int64_t max_scan_tiles = 0, max_sort_tiles = 0, max_pair_tiles = 0;
    // surrogate network
    compton::MlpDev mlp{};
    bool mlp_loaded = false;
    int64_t adam_step = 0;
    void* train_scratch = nullptr;  // inside the arena, sized by cfg.max_train_batch
    float* r_buf = nullptr;         // [max_particles] network output per pair (surrogate modes)
    compton::ServeEngine* serve = nullptr;  // continuous-batching engine (compton_serve_start)
    compton::KernelTiming* timing = nullptr;  // per-kernel event pairs (compton_kernel_timing)
    bool bin_weighted = false;                // the last binning carried per-particle weights
    bool train_tc = false;                    // training contractions on the tensor cores (BF16)
    compton::PnetDev pnet{};                  // the paper's 9-12-9 network
    bool pnet_loaded = false;
};

namespace compton {

// Host-side fault injection (compton_debug_inject, test support): while a
// fault is pending, the CUDA checks of the library count down `skip` passes
// and then report `fail` failures without making the failing call (an
// allocation reports cudaErrorMemoryAllocation, any other call
// cudaErrorLaunchFailure).  Nothing is done to the device.
bool inject_fault();
void inject_arm(int64_t skip, int64_t fail);

inline compton_status set_injected_error(compton_ctx* ctx, const char* where)
{
    if (ctx) std::snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: injected failure", where);
    return COMPTON_ECUDA;
}

inline compton_status set_cuda_error(compton_ctx* ctx, cudaError_t e, const char* where)
{
    if (ctx) {
        std::snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where, cudaGetErrorString(e));
    }
    return COMPTON_ECUDA;
}

#define COMPTON_CUDA_TRY(ctx, expr)                                  \
    do {                                                             \
        if (compton::inject_fault()) return compton::set_injected_error((ctx), #expr); \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return compton::set_cuda_error((ctx), _e, #expr); \
    } while (0)

// Launch-error check after a kernel launch.
#define COMPTON_LAUNCH_CHECK(ctx, name)                              \
    do {                                                             \
        cudaError_t _e = cudaGetLastError();                         \
        if (_e == cudaSuccess && compton::inject_fault()) return compton::set_injected_error((ctx), name); \
        if (_e != cudaSuccess) return compton::set_cuda_error((ctx), _e, name); \
    } while (0)

// Records an event pair around the launches made in its scope when kernel
// timing is on (start now, stop when the scope ends).
struct TimedScope {
    cudaStream_t stream;
    cudaEvent_t stop = nullptr;
    TimedScope(compton_ctx* ctx, int slot, cudaStream_t s) : stream(s)
    {
        if (!ctx->timing || !ctx->timing->on) return;
        KernelTiming& T = *ctx->timing;
        const int k = (int)(T.n[slot] % kTimingRing);
        if (cudaEventRecord(T.ev[slot][k][0], s) != cudaSuccess) return;
        stop = T.ev[slot][k][1];
        ++T.n[slot];
    }
    void end()
    {
        if (stop) cudaEventRecord(stop, stream);
        stop = nullptr;
    }
    ~TimedScope() { end(); }
};

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
compton_status launch_pnet_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                 const float* kx, const float* ky, const float* kz, int64_t n, float w_e, float w_g,
                                 float p_max, float* r_out, cudaStream_t stream);
compton_status launch_pnet_decide(compton_ctx* ctx, int64_t rows, const MlpDecide& dec, const float* w_e,
                                  const float* w_g, cudaStream_t stream);
compton_status launch_pnet_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                      const float* kx, const float* ky, const float* kz, const float* y,
                                      const float* w, int64_t n, float w_e, float w_g, float p_max, float lr,
                                      cudaStream_t stream);
compton_status launch_scatter_ntc(compton_ctx* ctx, compton_species* e, compton_species* g,
                                  const compton_pairs* pairs, uint64_t step, cudaStream_t stream);
compton_status launch_kn_ratio(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                               const float* kx, const float* ky, const float* kz, int64_t n, float* r_out,
                               cudaStream_t stream);
compton_status launch_sample_angle(compton_ctx* ctx, const float* x, const uint32_t* r, int64_t n, float* cth,
                                   float* sth, float* ratio, cudaStream_t stream);
compton_status mlp_repack(compton_ctx* ctx, cudaStream_t stream);
compton_status launch_mlp_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                const float* kx, const float* ky, const float* kz, int64_t n, compton_mode mode,
                                float* r_out, cudaStream_t stream, bool binned = false, bool candidates = false,
                                const MlpDecide* decide = nullptr);
size_t train_scratch_bytes(int64_t max_batch);
compton_status launch_balance_weights(compton_ctx* ctx, const float* r, int64_t n, const float* edges_host,
                                      int n_bins, float* w_out, cudaStream_t stream);
compton_status launch_mlp_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                     const float* kx, const float* ky, const float* kz, const float* y,
                                     const float* w, int64_t n, float lr, cudaStream_t stream);
compton_status launch_mlp_grad_tc(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                  const float* kx, const float* ky, const float* kz, const float* y, const float* w,
                                  int64_t n, cudaStream_t stream);
compton_status launch_mlp_calibrate(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                    const float* kx, const float* ky, const float* kz, int64_t n,
                                    cudaStream_t stream);
compton_status launch_selftest_wait(compton_ctx* ctx, uint64_t timeout_ns, cudaStream_t stream);
compton_status serve_start(compton_ctx* ctx, uint64_t pool_bytes, int32_t max_active);
compton_status serve_stop(compton_ctx* ctx);
compton_status serve_submit(compton_ctx* ctx, const compton_request* r, uint64_t* ticket);
compton_status serve_poll(compton_ctx* ctx, uint64_t ticket, compton_result* out);
compton_status serve_info(compton_ctx* ctx, uint64_t* in_use, uint64_t* peak, uint64_t* pool);

}  // namespace compton
