// mlp_train.cu -- training of the surrogate network on the GPU (arXiv
// 2206.02937, Sec. 3.2: the network is trained against the analytic
// probability with the mean absolute error loss and the Adam optimizer at
// learning rate 1e-3; Sec. 4: the implementation also allows training inside
// the simulation).
//
// One training step over a minibatch of n samples (inputs u, k; targets y;
// per-sample weights w from the data balancing):
//   k_train_fwd_bwd  one sample per thread, FP32: forward through the four
//                    SiLU layers and the sigmoid output, storing each hidden
//                    pre-activation z_l; the weighted MAE subgradient
//                    w sign(y' - y) (0 at equality); backward through the
//                    sigmoid and each layer, storing each layer's delta
//                    (dL/dz_l); loss numerator and weight sum accumulated.
//   k_train_dw       dW_l = sum_s delta_l(s) h_{l-1}(s)^T and db_l = sum_s
//                    delta_l(s) over the batch: each CTA reduces a chunk of
//                    samples for one layer into registers and adds its
//                    partial sums to the gradient.
//   k_train_adam     Adam (Kingma and Ba 2014, Algorithm 1) on the FP32 master
//                    parameters with the gradient divided by sum w, then the
//                    inference images are rebuilt (k_mlp_pack).
// With the tensor-core training precision selected (compton_mlp_set_train_
// precision), the gradient comes from k_train_tc (mlp_train_tc.cu) instead of
// the first two kernels; Adam and the repacking are shared.
// Scratch: z and delta for 4 layers x 64 units x n samples, laid out
// [layer][unit][sample] so that consecutive threads touch consecutive words.
#include "ctx.hpp"
#include "features.cuh"

namespace compton {
namespace {

constexpr int kTrThreads = 128;

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

struct TrainArgs {
    MlpDev m;
    const float* u[3];
    const float* k[3];
    const float* y;
    const float* w;  // nullable: all ones
    int64_t n;
    float* z;        // [4][64][n]
    float* delta;    // [4][64][n]
    float* dout;     // [n] delta of the output unit
    float* feat;     // [6][n]
};

__global__ void __launch_bounds__(kTrThreads) k_train_fwd_bwd(TrainArgs a)
{
    extern __shared__ float sm[];
    float* wt = sm;                          // 4 x 64 x 64: wt[l][i][j] = W_l[j][i]
    float* hs = wt + 4 * 4096;               // 64 x kTrThreads activations / deltas
    float* bias = hs + 64 * kTrThreads;      // 256
    float* w4 = bias + 256;                  // 64
    const int tid = threadIdx.x;
    const MlpDev& m = a.m;
    for (int i = tid; i < 4096; i += kTrThreads) reinterpret_cast<float4*>(wt)[i] = reinterpret_cast<const float4*>(m.wt32)[i];
    for (int i = tid; i < 256; i += kTrThreads) bias[i] = m.bias[i];
    if (tid < 64) w4[tid] = m.w4[tid];
    const float b4 = m.b4[0];
    __syncthreads();
    const int64_t n = a.n;
    float loss_num = 0.0f, wsum = 0.0f;
    for (int64_t s = (int64_t)blockIdx.x * kTrThreads + tid; s < n; s += (int64_t)gridDim.x * kTrThreads) {
        // ---- forward ----
        float f[6];
        features(m, a.u[0][s], a.u[1][s], a.u[2][s], a.k[0][s], a.k[1][s], a.k[2][s], f);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            hs[i * kTrThreads + tid] = f[i];
            a.feat[i * n + s] = f[i];
        }
        float acc[64];
        for (int l = 0; l < 4; ++l) {
#pragma unroll
            for (int j = 0; j < 64; ++j) acc[j] = bias[l * 64 + j];
            const int n_in = l == 0 ? 6 : 64;
            for (int i = 0; i < n_in; ++i) {
                const float hi = hs[i * kTrThreads + tid];
                const float4* wr = reinterpret_cast<const float4*>(wt + l * 4096 + i * 64);
#pragma unroll
                for (int j4 = 0; j4 < 16; ++j4) {
                    const float4 wv = wr[j4];
                    acc[4 * j4 + 0] = fmaf(wv.x, hi, acc[4 * j4 + 0]);
                    acc[4 * j4 + 1] = fmaf(wv.y, hi, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(wv.z, hi, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(wv.w, hi, acc[4 * j4 + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                a.z[((int64_t)l * 64 + j) * n + s] = acc[j];
                hs[j * kTrThreads + tid] = acc[j] * sigm(acc[j]);
            }
        }
        float zo = b4;
#pragma unroll
        for (int j = 0; j < 64; ++j) zo = fmaf(hs[j * kTrThreads + tid], w4[j], zo);
        const float yp = sigm(zo);
        const float wi = a.w ? a.w[s] : 1.0f;
        const float diff = yp - a.y[s];
        loss_num += wi * fabsf(diff);
        wsum += wi;
        // ---- backward ----  (unnormalised: the 1/sum w factor is applied in Adam)
        const float g = diff > 0.0f ? wi : (diff < 0.0f ? -wi : 0.0f);
        const float d_out = g * yp * (1.0f - yp);
        a.dout[s] = d_out;
        // delta of the last hidden layer: W4^T d_out times silu'(z_3); acc holds z_3
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            const float sg = sigm(acc[j]);
            const float ds = sg * (1.0f + acc[j] * (1.0f - sg));
            acc[j] = w4[j] * d_out * ds;
        }
        for (int l = 3; l >= 0; --l) {
#pragma unroll
            for (int j = 0; j < 64; ++j) a.delta[((int64_t)l * 64 + j) * n + s] = acc[j];
            if (l == 0) break;
            // dh_{l-1}[i] = sum_j W_l[j][i] delta_l[j] = sum_j wt[l][i][j] delta_l[j]
            for (int i = 0; i < 64; ++i) {
                const float4* wr = reinterpret_cast<const float4*>(wt + l * 4096 + i * 64);
                float t = 0.0f;
#pragma unroll
                for (int j4 = 0; j4 < 16; ++j4) {
                    const float4 wv = wr[j4];
                    t = fmaf(wv.x, acc[4 * j4 + 0], t);
                    t = fmaf(wv.y, acc[4 * j4 + 1], t);
                    t = fmaf(wv.z, acc[4 * j4 + 2], t);
                    t = fmaf(wv.w, acc[4 * j4 + 3], t);
                }
                hs[i * kTrThreads + tid] = t;
            }
            // delta_{l-1} = dh_{l-1} * silu'(z_{l-1}), silu' = s (1 + z (1 - s))
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                const float zz = a.z[((int64_t)(l - 1) * 64 + i) * n + s];
                const float sg = sigm(zz);
                acc[i] = hs[i * kTrThreads + tid] * sg * (1.0f + zz * (1.0f - sg));
            }
        }
    }
    // loss and weight sums
    for (int d = 16; d > 0; d >>= 1) {
        loss_num += __shfl_xor_sync(0xffffffffu, loss_num, d);
        wsum += __shfl_xor_sync(0xffffffffu, wsum, d);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&m.loss[0], loss_num);
        atomicAdd(&m.loss[1], wsum);
    }
}

// Weight gradient of one layer over a chunk of samples.  256 threads, each
// owning 16 consecutive entries (j, i..i+15) of the 64 x 64 block (layer 0:
// 64 x 6, the output layer: 1 x 64 plus its bias).  Inputs h_{l-1} are the
// features (l = 0) or silu(z_{l-1}); deltas are stored per layer.
constexpr int kDwThreads = 256;
constexpr int kDwChunk = 256;

__global__ void __launch_bounds__(kDwThreads) k_train_dw(TrainArgs a, int64_t chunk)
{
    __shared__ float hsh[64][kDwChunk / 8 + 1];   // 64 inputs x 32 samples (+1: no bank conflicts)
    __shared__ float dsh[64][kDwChunk / 8 + 1];   // 64 deltas x 32 samples
    const int l = blockIdx.y;                  // 0..4 (4 = output layer)
    const int tid = threadIdx.x;
    const int64_t n = a.n;
    const int64_t s0 = (int64_t)blockIdx.x * chunk;
    const int64_t s1 = s0 + chunk < n ? s0 + chunk : n;
    const int n_in = l == 0 ? 6 : 64;
    const int n_out = l == 4 ? 1 : 64;
    const int j = tid / 4;                     // output unit
    const int i0 = (tid % 4) * 16;             // first input of this thread
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    float accb = 0.0f;
    constexpr int S = kDwChunk / 8;
    for (int64_t sb = s0; sb < s1; sb += S) {
        const int ns = (int)(s1 - sb < S ? s1 - sb : S);
        __syncthreads();
        for (int e = tid; e < 64 * S; e += kDwThreads) {
            const int unit = e / S, ss = e % S;
            float h = 0.0f, d = 0.0f;
            if (ss < ns) {
                const int64_t s = sb + ss;
                if (unit < n_in) {
                    if (l == 0) {
                        h = a.feat[unit * n + s];
                    } else {
                        const float zz = a.z[((int64_t)(l - 1) * 64 + unit) * n + s];
                        h = zz / (1.0f + expf(-zz));
                    }
                }
                if (unit < n_out) d = l == 4 ? a.dout[s] : a.delta[((int64_t)l * 64 + unit) * n + s];
            }
            hsh[unit][ss] = h;
            dsh[unit][ss] = d;
        }
        __syncthreads();
        if (j < n_out) {
            for (int ss = 0; ss < ns; ++ss) {
                const float d = dsh[j][ss];
                accb += (i0 == 0) ? d : 0.0f;
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = fmaf(d, hsh[i0 + q][ss], acc[q]);
            }
        }
    }
    if (j < n_out) {
        float* gw = a.m.grad + mlp_off_w(l);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (i0 + q < n_in) atomicAdd(&gw[j * n_in + i0 + q], acc[q]);
        if (i0 == 0) atomicAdd(&a.m.grad[mlp_off_b(l) + j], accb);
    }
}

__global__ void k_train_adam(MlpDev m, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float ws = m.loss[1];
    const float g = ws > 0.0f ? m.grad[i] / ws : 0.0f;
    const float mm = b1 * m.adam_m[i] + (1.0f - b1) * g;
    const float vv = b2 * m.adam_v[i] + (1.0f - b2) * g * g;
    m.adam_m[i] = mm;
    m.adam_v[i] = vv;
    const float mh = mm / bc1;
    const float vh = vv / bc2;
    m.theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Data balancing (Sec. 3.2: events of every probability range should appear
// about equally often).  Sample i belongs to bin b = number of inner edges
// <= r_i; its weight is n / (count_b * number of non-empty bins).
constexpr int kMaxBalanceBins = 256;

__device__ __forceinline__ int balance_bin(const float* inner, int n_inner, float r)
{
    int lo = 0, hi = n_inner;  // first inner edge > r
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (inner[mid] <= r) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_balance_hist(const float* __restrict__ r, int64_t n, const float* __restrict__ edges, int n_bins,
                               int* __restrict__ count)
{
    __shared__ float inner[kMaxBalanceBins];
    __shared__ int h[kMaxBalanceBins];
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x) {
        h[i] = 0;
        if (i < n_bins - 1) inner[i] = edges[i + 1];
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[balance_bin(inner, n_bins - 1, r[i])], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x)
        if (h[i]) atomicAdd(&count[i], h[i]);
}

__global__ void k_balance_weights(const float* __restrict__ r, int64_t n, const float* __restrict__ edges,
                                  int n_bins, const int* __restrict__ count, float* __restrict__ w)
{
    __shared__ float inner[kMaxBalanceBins];
    __shared__ float inv[kMaxBalanceBins];
    __shared__ int nonempty;
    if (threadIdx.x == 0) {
        int ne = 0;
        for (int i = 0; i < n_bins; ++i) ne += count[i] > 0;
        nonempty = ne;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x) {
        if (i < n_bins - 1) inner[i] = edges[i + 1];
        inv[i] = count[i] > 0 ? (float)((double)n / ((double)count[i] * (double)nonempty)) : 0.0f;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = inv[balance_bin(inner, n_bins - 1, r[i])];
}

}  // namespace

compton_status launch_balance_weights(compton_ctx* ctx, const float* r, int64_t n, const float* edges_host,
                                      int n_bins, float* w_out, cudaStream_t stream)
{
    if (n_bins < 1 || n_bins > kMaxBalanceBins) return COMPTON_EINVAL;
    COMPTON_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mlp.edges, edges_host, sizeof(float) * (n_bins + 1),
                                          cudaMemcpyHostToDevice, stream));
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->mlp.hist, 0, sizeof(int) * n_bins, stream));
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)ctx->n_sm * 8) blocks = (int64_t)ctx->n_sm * 8;
    k_balance_hist<<<(unsigned)blocks, 256, 0, stream>>>(r, n, ctx->mlp.edges, n_bins, ctx->mlp.hist);
    COMPTON_LAUNCH_CHECK(ctx, "k_balance_hist");
    k_balance_weights<<<(unsigned)blocks, 256, 0, stream>>>(r, n, ctx->mlp.edges, n_bins, ctx->mlp.hist, w_out);
    COMPTON_LAUNCH_CHECK(ctx, "k_balance_weights");
    return COMPTON_OK;
}

size_t train_scratch_bytes(int64_t max_batch)
{
    return (size_t)max_batch * sizeof(float) * (2 * 4 * 64 + 1 + 6);
}

compton_status adam_and_repack(compton_ctx* ctx, float lr, cudaStream_t stream);

compton_status launch_mlp_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                     const float* kx, const float* ky, const float* kz, const float* y,
                                     const float* w, int64_t n, float lr, cudaStream_t stream)
{
    TrainArgs a;
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
    float* base = reinterpret_cast<float*>(ctx->train_scratch);
    a.z = base;
    a.delta = base + (size_t)4 * 64 * n;
    a.dout = a.delta + (size_t)4 * 64 * n;
    a.feat = a.dout + n;
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->mlp.grad, 0, sizeof(float) * kMlpParams, stream));
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(ctx->mlp.loss, 0, 2 * sizeof(float), stream));
    if (ctx->train_tc) {
        const compton_status st = launch_mlp_grad_tc(ctx, ux, uy, uz, kx, ky, kz, y, w, n, stream);
        if (st != COMPTON_OK) return st;
        return adam_and_repack(ctx, lr, stream);
    }
    const int smem = (4 * 4096 + 64 * kTrThreads + 256 + 64) * 4;
    COMPTON_CUDA_TRY(ctx, cudaFuncSetAttribute(k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int n_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + kTrThreads - 1) / kTrThreads;
    if (blocks > (int64_t)n_sm * 2) blocks = (int64_t)n_sm * 2;
    k_train_fwd_bwd<<<(unsigned)blocks, kTrThreads, smem, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_train_fwd_bwd");
    int64_t chunk = (n + 4 * n_sm - 1) / (4 * n_sm);
    if (chunk < kDwChunk) chunk = kDwChunk;
    const dim3 grid((unsigned)((n + chunk - 1) / chunk), 5);
    k_train_dw<<<grid, kDwThreads, 0, stream>>>(a, chunk);
    COMPTON_LAUNCH_CHECK(ctx, "k_train_dw");
    return adam_and_repack(ctx, lr, stream);
}

// Adam on the gradient sums of the step, then the inference images.
compton_status adam_and_repack(compton_ctx* ctx, float lr, cudaStream_t stream)
{
    ctx->adam_step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-7f;
    const float bc1 = 1.0f - (float)std::pow(0.9, (double)ctx->adam_step);
    const float bc2 = 1.0f - (float)std::pow(0.999, (double)ctx->adam_step);
    k_train_adam<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(ctx->mlp, lr, b1, b2, eps, bc1, bc2);
    COMPTON_LAUNCH_CHECK(ctx, "k_train_adam");
    return mlp_repack(ctx, stream);
}

}  // namespace compton
