// mlp_train_tc.cu -- one training step of the surrogate network with every
// contraction on the tcgen05 tensor cores (BF16 operands, FP32 accumulation
// in tensor memory): arXiv 2206.02937, Sec. 3.2 (the network is trained
// against the analytic probability with the mean absolute error loss and
// Adam).
//
// Notation: h = the six input features (zero-padded to 64), z_l = a_{l-1}
// W_l^T (a_{-1} = h), a_l = SiLU(z_l + b_l) for the four hidden layers,
// y' = sigmoid(a_3 . w_4 + b_4); with the weighted MAE subgradient
// g = w sign(y' - y), d_out = g y'(1 - y'), the backward pass is
//   delta_3 = d_out w_4 * SiLU'(z_3 + b_3),
//   delta_{l-1} = (delta_l W_l) * SiLU'(z_{l-1} + b_{l-1}),
//   dW_l = delta_l^T a_{l-1},  db_l = sum over samples of delta_l,
//   dw_4 = sum d_out a_3,  db_4 = sum d_out.
//
// k_train_tc: persistent CTAs of 128 threads (one sample row per thread),
// one 128-row tile at a time.  Per tile, with one thread issuing the MMAs:
//   forward   z_l (128 x 64) = A_l W_l^T: A_l is the activation tile in the
//             128-byte-swizzled K-major layout (row = sample), W_l the
//             inference weight tile; z_l stays in tensor memory (columns
//             64 l .. 64 l + 63) for the backward pass, the epilogue writes
//             a_l as the next layer's A tile;
//   backward  delta_l is written as a tile of the same row layout, then
//             dX: delta_l (K-major, K = output units) times the same weight
//                 tile read as an MN-major operand (N = input units), so no
//                 transposed weight copy is needed; the result reuses the
//                 columns of z_l, which the epilogue has consumed;
//             dW: delta_l^T a_{l-1} with both tiles read as MN-major operands
//                 (M = output units, N = input units, K = the tile's samples),
//                 accumulated over every tile of the CTA in tensor memory
//                 (columns 256 + 64 l); the MMA has M = 128, its rows 64..127
//                 read a padding region and are never used.
// Bias gradients, the output layer and the loss run on the CUDA cores (warp
// reduce-scatters of the per-row values).  At the end each CTA adds its
// gradient sums to the context's gradient with one atomic per entry; Adam and
// the repacking of the inference images follow as in the FP32 path.
// Every wait is bounded by %globaltimer (ETIMEOUT recorded, TMEM freed).
#include <cuda_bf16.h>

#include "ctx.hpp"
#include "device_math.cuh"
#include "features.cuh"
#include "tc_ptx.cuh"

namespace compton {
namespace {

constexpr int kTT = 128;                     // threads = rows per tile
constexpr uint32_t kTileBytes = 16384;       // 128 rows x 128 B
constexpr uint32_t kWBytes = 8192;           // 64 rows x 128 B
// shared memory (base aligned to 1024 B)
constexpr uint32_t kOffW = 0;                             // W_0..W_3 tiles
constexpr uint32_t kOffAct = kOffW + 4 * kWBytes;         // h, a_0, a_1, a_2 tiles
constexpr uint32_t kOffDelta = kOffAct + 4 * kTileBytes;  // delta tile
constexpr uint32_t kOffPad = kOffDelta + kTileBytes;      // read by the unused upper MMA rows
constexpr uint32_t kOffBias = kOffPad + kTileBytes;       // 4 x 64 floats
constexpr uint32_t kOffW4 = kOffBias + 1024;              // 64 floats
constexpr uint32_t kOffBar = kOffW4 + 256;                // mbarrier
constexpr uint32_t kOffSlot = kOffBar + 8;                // TMEM address
constexpr uint32_t kSmemTrainTc = kOffSlot + 8 + 1024;    // + alignment slack
constexpr uint32_t kTmemCols = 512;                       // z: 0..255, dW: 256..511
constexpr uint64_t kWaitNs = 2000000000ull;

// MN-major operand descriptor (128-byte swizzle): rows of 64 BF16 values
// contiguous along M or N, eight K rows per 1024-byte atom (stride byte
// offset 1024), the next 64-wide M/N block `lbo` bytes further.
__device__ __forceinline__ uint64_t sw128_mnmajor_desc(uint32_t saddr, uint32_t lbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptors: BF16 x BF16 -> F32, M = 128, N = 64; bit 15 / 16
// mark A / B as MN-major
constexpr uint32_t kIdescFwd = tc::make_idesc(1, 1, 128, 64);
constexpr uint32_t kIdescDx = kIdescFwd | (1u << 16);
constexpr uint32_t kIdescDw = kIdescFwd | (1u << 15) | (1u << 16);

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

// 32 values of a row written as BF16 into chunks 4h .. 4h+3 of the row's
// 128 bytes (swizzled).
__device__ __forceinline__ void store_row_half(uint8_t* tile, int row, int h, const float* v)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(tile + tc::sw128_offset(row, 4 * h + q)) =
            make_uint4(pack2(v[8 * q], v[8 * q + 1]), pack2(v[8 * q + 2], v[8 * q + 3]),
                       pack2(v[8 * q + 4], v[8 * q + 5]), pack2(v[8 * q + 6], v[8 * q + 7]));
}

// Sum over the warp's 32 rows of 32 per-row values: afterwards lane l holds
// the sum of value l (a reduce-scatter in five exchange rounds).
__device__ __forceinline__ float warp_reduce_scatter32(float* v)
{
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool upper = (lane & (unsigned)half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0];
}

struct TrainTcArgs {
    MlpDev m;
    const float* u[3];
    const float* k[3];
    const float* y;
    const float* w;  // nullable: all ones
    int64_t n;
    DeviceStats* stats;
};

__global__ void __launch_bounds__(kTT, 1) k_train_tc(TrainTcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const unsigned lane = tid & 31u;
    const MlpDev& m = a.m;
    uint8_t* Wt = sm + kOffW;
    uint8_t* Act = sm + kOffAct;  // tile t: input of layer t (t = 0: features)
    uint8_t* Dl = sm + kOffDelta;
    float* bias = reinterpret_cast<float*>(sm + kOffBias);
    float* w4 = reinterpret_cast<float*>(sm + kOffW4);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffSlot);

    const uint4* wsrc = reinterpret_cast<const uint4*>(m.wbf16);
    for (int i = tid; i < (int)(4 * kWBytes / 16); i += kTT) reinterpret_cast<uint4*>(Wt)[i] = wsrc[i];
    // activation, delta and padding tiles start at zero (the feature tile's
    // chunks 1..7 stay zero: layer 0's K padding)
    for (int i = tid; i < (int)(6 * kTileBytes / 16); i += kTT)
        reinterpret_cast<uint4*>(Act)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < 256; i += kTT) bias[i] = m.bias[i];
    if (tid < 64) w4[tid] = m.w4[tid];
    const float b4 = m.b4[0];
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lanes
    const uint32_t sW = tc::smem_u32(Wt), sAct = tc::smem_u32(Act), sD = tc::smem_u32(Dl);
    const uint32_t pad_lbo = kOffPad - kOffDelta;  // upper M block of the dW A operand

    uint32_t phase = 0;
    bool failed = false;
    // one MMA group issued by thread 0, committed, and waited for by all
    auto wait_mma = [&]() -> bool {
        const bool ok = tc::mbar_wait(bar, phase, kWaitNs);
        phase ^= 1u;
        tc::fence_after_sync();
        return __all_sync(0xffffffffu, ok);  // warp-uniform: the TMEM loads are warp-wide
    };
    // every thread's shared-memory writes and TMEM reads done before the next MMA
    auto sync_for_mma = [&](bool bad) -> bool {
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        const int any_bad = __syncthreads_or(bad ? 1 : 0);
        tc::fence_after_sync();
        return any_bad != 0;
    };

    // per-lane sums over the CTA's rows: db_l (lane l holds units l and l+32),
    // dw_4 (same), db_4, loss numerator and weight sum
    float db[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    float dw4[2] = {0, 0};
    float db4 = 0.0f, loss_num = 0.0f, wsum = 0.0f;
    bool first = true;  // the CTA's first tile starts the dW accumulators

    const int64_t n_tiles = (a.n + kTT - 1) / kTT;
    for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int64_t row = tile * kTT + tid;
        const bool live = row < a.n;
        float f[6] = {0, 0, 0, 0, 0, 0};
        if (live) features(m, a.u[0][row], a.u[1][row], a.u[2][row], a.k[0][row], a.k[1][row], a.k[2][row], f);
        *reinterpret_cast<uint4*>(Act + tc::sw128_offset(tid, 0)) =
            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), 0u);
        const float yt = live ? a.y[row] : 0.0f;
        const float wt = live ? (a.w ? a.w[row] : 1.0f) : 0.0f;
        if (sync_for_mma(false)) break;

        // ---------------- forward ----------------
        float out = b4;
        for (int l = 0; l < 4; ++l) {
            if (tid == 0) {
                const uint64_t ad = tc::sw128_kmajor_desc(sAct + l * kTileBytes);
                const uint64_t bd = tc::sw128_kmajor_desc(sW + l * kWBytes);
                const int n_ks = l == 0 ? 1 : 4;  // layer 0: the six features fit one K step
                for (int ks = 0; ks < n_ks; ++ks) tc::mma_bf16(tmem + 64 * l, ad + 2 * ks, bd + 2 * ks, kIdescFwd, ks > 0);
                tc::mma_commit(bar);
            }
            const bool ok = wait_mma();
            if (ok) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float v[32];
                    tc::tmem_ld32(tmem + lane_base + 64 * l + 32 * h, v);
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const float zb = v[c] + bias[64 * l + 32 * h + c];
                        v[c] = zb * sigm(zb);
                    }
                    if (l < 3) {
                        store_row_half(Act + (l + 1) * kTileBytes, tid, h, v);
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) out = fmaf(v[c], w4[32 * h + c], out);
                    }
                }
            }
            if (sync_for_mma(!ok)) {
                failed = true;
                break;
            }
        }
        if (failed) break;

        // ---------------- output and loss ----------------
        const float yp = sigm(out);
        const float diff = yp - yt;
        loss_num += wt * fabsf(diff);
        wsum += wt;
        const float g = diff > 0.0f ? wt : (diff < 0.0f ? -wt : 0.0f);
        const float d_out = live ? g * yp * (1.0f - yp) : 0.0f;
        db4 += d_out;

        // ---------------- backward ----------------
        // delta_3 from z_3 (tensor memory), with dw_4 and db_3 on the way
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[32], p[32];
            tc::tmem_ld32(tmem + lane_base + 64 * 3 + 32 * h, v);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const float zb = v[c] + bias[64 * 3 + 32 * h + c];
                const float s = sigm(zb);
                p[c] = zb * s * d_out;                                        // a_3 d_out
                v[c] = d_out * w4[32 * h + c] * s * fmaf(zb, 1.0f - s, 1.0f);  // delta_3
            }
            store_row_half(Dl, tid, h, v);
            dw4[h] += warp_reduce_scatter32(p);
            db[3][h] += warp_reduce_scatter32(v);
        }
        for (int l = 3; l >= 0 && !failed; --l) {
            if (sync_for_mma(false)) {
                failed = true;
                break;
            }
            if (tid == 0) {
                // dW_l += delta_l^T a_{l-1}: K = the tile's 128 samples, 16 per MMA (2048 B)
                const uint32_t d_w = tmem + 256 + 64 * l;
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t ad = sw128_mnmajor_desc(sD + 2048 * ks, pad_lbo);
                    const uint64_t bd = sw128_mnmajor_desc(sAct + l * kTileBytes + 2048 * ks, 0);
                    tc::mma_bf16(d_w, ad, bd, kIdescDw, (first && ks == 0) ? 0u : 1u);
                }
                // g_{l-1} = delta_l W_l into z_l's columns: K = 64 output units,
                // 16 per MMA (32 B of the K-major delta row, 2048 B of W_l)
                if (l > 0) {
                    const uint64_t ad = tc::sw128_kmajor_desc(sD);
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t bd = sw128_mnmajor_desc(sW + l * kWBytes + 2048 * ks, 0);
                        tc::mma_bf16(tmem + 64 * l, ad + 2 * ks, bd, kIdescDx, ks > 0);
                    }
                }
                tc::mma_commit(bar);
            }
            const bool ok = wait_mma();
            if (!ok) {
                failed = true;
            } else if (l > 0) {
                // delta_{l-1} = g_{l-1} * SiLU'(z_{l-1} + b_{l-1})
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float gv[32], zv[32];
                    tc::tmem_ld32(tmem + lane_base + 64 * l + 32 * h, gv);
                    tc::tmem_ld32(tmem + lane_base + 64 * (l - 1) + 32 * h, zv);
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const float zb = zv[c] + bias[64 * (l - 1) + 32 * h + c];
                        const float s = sigm(zb);
                        gv[c] *= s * fmaf(zb, 1.0f - s, 1.0f);
                    }
                    store_row_half(Dl, tid, h, gv);
                    db[l - 1][h] += warp_reduce_scatter32(gv);
                }
            }
            if (__syncthreads_or(failed ? 1 : 0)) failed = true;
        }
        first = false;
    }
    if (failed && tid == 0) atomicOr(&a.stats->error_flags, (unsigned long long)kErrTimeout);

    // ---------------- the CTA's sums into the context's gradient ----------------
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!failed && !first && warp < 2) {
        // rows 0..63 of each dW block (TMEM lanes of warps 0 and 1)
        const int j = tid;  // output unit
        for (int l = 0; l < 4; ++l) {
            float* gw = m.grad + mlp_off_w(l);
            const int n_in = l == 0 ? 6 : 64;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tc::tmem_ld32(tmem + lane_base + 256 + 64 * l + 32 * h, v);
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (32 * h + c < n_in) atomicAdd(&gw[j * n_in + 32 * h + c], v[c]);
            }
        }
    }
    if (!failed) {
        for (int l = 0; l < 4; ++l)
            for (int h = 0; h < 2; ++h) atomicAdd(&m.grad[mlp_off_b(l) + 32 * h + (int)lane], db[l][h]);
        for (int h = 0; h < 2; ++h) atomicAdd(&m.grad[mlp_off_w(4) + 32 * h + (int)lane], dw4[h]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            db4 += __shfl_xor_sync(0xffffffffu, db4, d);
            loss_num += __shfl_xor_sync(0xffffffffu, loss_num, d);
            wsum += __shfl_xor_sync(0xffffffffu, wsum, d);
        }
        if (lane == 0) {
            atomicAdd(&m.grad[mlp_off_b(4)], db4);
            atomicAdd(&m.loss[0], loss_num);
            atomicAdd(&m.loss[1], wsum);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

// The gradient of one minibatch on the tensor cores (the caller zeroes the
// gradient and loss sums before, and runs Adam after).
compton_status launch_mlp_grad_tc(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                  const float* kx, const float* ky, const float* kz, const float* y, const float* w,
                                  int64_t n, cudaStream_t stream)
{
    if (n <= 0) return COMPTON_OK;
    TrainTcArgs a;
    a.m = ctx->mlp;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.y = y;
    a.w = w;
    a.n = n;
    a.stats = ctx->stats;
    COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmemTrainTc));
    int n_sm = 0, dev = 0;
    COMPTON_CUDA_TRY(ctx, cudaGetDevice(&dev));
    COMPTON_CUDA_TRY(ctx, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = (n + kTT - 1) / kTT;
    const int64_t grid = tiles < n_sm ? tiles : n_sm;  // one CTA per SM (all 512 TMEM columns)
    k_train_tc<<<(unsigned)grid, kTT, kSmemTrainTc, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_train_tc");
    return COMPTON_OK;
}

}  // namespace compton
