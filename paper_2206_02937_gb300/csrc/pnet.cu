// pnet.cu -- the paper's own surrogate network (arXiv 2206.02937, Sec. 3.2:
// three hidden layers of 9, 12 and 9 ReLU units, one sigmoid output, trained
// with the mean absolute error and Adam).
//
// Inputs (Fig. 2a: both momenta, both macro-particle weights and the cell's
// maximum probability): f = [sgnlog(u/s_u)/n_u (3), sgnlog(k/s_k)/n_k (3),
// ln(w_e)/8, ln(w_g)/8, ln(P_max)/8] with P_max = 2 n dt; output
// r = sigma_KN v / (2 sigma_T) (the probability over P_max).  337
// parameters, W0 (9x9) b0 W1 (12x9) b1 W2 (9x12) b2 W3 (1x9) b3, each W
// (out, in) row-major.
//
// The network is tiny (306 multiply-adds per sample), so everything runs on
// the CUDA cores in FP32, one sample per thread, with the parameters staged
// in shared memory:
//   k_pnet_infer   r per explicit pair, or -- in the surrogate step -- per
//                  candidate of the candidate list (weights w/V of the pair's
//                  particles, P_max = 2 n_p dt of the pair) with the decision
//                  made in the same thread (analytic probability outside the
//                  training range) and accepted pairs appended to the list;
//   k_pnet_train   forward and backward per sample; each parameter's
//                  gradient is summed over the warp by shuffles, then over
//                  the block in shared memory, then once per block in global
//                  memory;
//   k_pnet_adam    Adam over the 337 parameters.
#include "ctx.hpp"
#include "device_math.cuh"
#include "features.cuh"

namespace compton {
namespace {

constexpr int kPnetThreads = 256;
constexpr int kP_W0 = 0, kP_B0 = 81, kP_W1 = 90, kP_B1 = 198, kP_W2 = 210, kP_B2 = 318, kP_W3 = 327, kP_B3 = 336;
static_assert(kP_B3 + 1 == kPnetParams, "layout");

struct PnetArgs {
    PnetDev p;
    const float* u[3];
    const float* k[3];
    int64_t n;
    float ln_we, ln_wg, ln_pmax;  // scalar inputs of explicit rows (ln of w_e, w_g, P_max)
    float* r_out;
    // candidate rows (surrogate step): the candidate list and its decision
    const CandPair* cand;
    const uint32_t* n_cand;
    float dt, gamma64, ln_w;
    const float* w_e;  // per-particle weights of the sorted species (nullptr: ln_w)
    const float* w_g;
    float* prob_out;
    uint8_t* flag_out;
    AcceptedPair* accepted;
    uint32_t* n_accepted;
    DeviceStats* stats;
    MlpDev range;  // training range (range_* fields)
    // training
    const float* y;
    const float* wts;
    float* loss;  // [2] weighted |error| sum, weight sum
};

__device__ __forceinline__ void pnet_features(const PnetDev& p, const float* q, float lwe, float lwg, float lpm,
                                              float* f)
{
    const float iu = __fdividef(1.0f, p.fs[0]), nu = __fdividef(1.0f, p.fs[1]);
    const float ik = __fdividef(1.0f, p.fs[2]), nk = __fdividef(1.0f, p.fs[3]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f[i] = sgnlog(q[i] * iu) * nu;
        f[3 + i] = sgnlog(q[3 + i] * ik) * nk;
    }
    f[6] = lwe * 0.125f;
    f[7] = lwg * 0.125f;
    f[8] = lpm * 0.125f;
}

// Forward pass; keeps the hidden activations for the backward pass.
__device__ __forceinline__ float pnet_forward(const float* th, const float* f, float* h1, float* h2, float* h3)
{
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        float z = th[kP_B0 + o];
#pragma unroll
        for (int i = 0; i < 9; ++i) z = fmaf(th[kP_W0 + 9 * o + i], f[i], z);
        h1[o] = fmaxf(z, 0.0f);
    }
#pragma unroll
    for (int o = 0; o < 12; ++o) {
        float z = th[kP_B1 + o];
#pragma unroll
        for (int i = 0; i < 9; ++i) z = fmaf(th[kP_W1 + 9 * o + i], h1[i], z);
        h2[o] = fmaxf(z, 0.0f);
    }
#pragma unroll
    for (int o = 0; o < 9; ++o) {
        float z = th[kP_B2 + o];
#pragma unroll
        for (int i = 0; i < 12; ++i) z = fmaf(th[kP_W2 + 12 * o + i], h2[i], z);
        h3[o] = fmaxf(z, 0.0f);
    }
    float z = th[kP_B3];
#pragma unroll
    for (int i = 0; i < 9; ++i) z = fmaf(th[kP_W3 + i], h3[i], z);
    return __fdividef(1.0f, 1.0f + __expf(-z));
}

__device__ __forceinline__ void stage_params(const PnetDev& p, float* th)
{
    for (int i = threadIdx.x; i < kPnetParams; i += blockDim.x) th[i] = p.theta[i];
    __syncthreads();
}

// kCand: rows are candidates, decided here; else explicit rows, r written.
template <bool kCand>
__global__ void __launch_bounds__(kPnetThreads, 3) k_pnet_infer(PnetArgs a)
{
    __shared__ float th[kPnetParams];
    stage_params(a.p, th);
    const unsigned lane = threadIdx.x & 31u;
    const int64_t n = kCand ? (int64_t)*a.n_cand : a.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count, so the ballots see whole warps
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    unsigned n_hit = 0, n_fb = 0;
    for (int64_t base = first; base < n; base += stride) {
        const int64_t row = base + lane;
        const bool live = row < n;
        float q[6] = {0, 0, 0, 0, 0, 0};
        CandPair c{};
        if (live) {
            if (kCand) {
                c = a.cand[row];
                q[0] = c.u[0];
                q[1] = c.u[1];
                q[2] = c.u[2];
                q[3] = c.k[0];
                q[4] = c.k[1];
                q[5] = c.k[2];
            } else {
                q[0] = a.u[0][row];
                q[1] = a.u[1][row];
                q[2] = a.u[2][row];
                q[3] = a.k[0][row];
                q[4] = a.k[1][row];
                q[5] = a.k[2][row];
            }
        }
        float f[9], h1[9], h2[12], h3[9];
        const float lpm = kCand ? logf(fmaxf(2.0f * c.dens * a.dt, 1e-30f)) : a.ln_pmax;
        float lwe = kCand ? a.ln_w : a.ln_we, lwg = kCand ? a.ln_w : a.ln_wg;
        if (kCand && live) {
            if (a.w_e) lwe = logf(a.w_e[c.ie]);
            if (a.w_g) lwg = logf(a.w_g[c.ig]);
        }
        pnet_features(a.p, q, lwe, lwg, lpm, f);
        const float r = pnet_forward(th, f, h1, h2, h3);
        if (!kCand) {
            if (live) a.r_out[row] = r;
            continue;
        }
        bool hit = false, fb = false;
        float x = -1.0f;
        if (live) {
            const float g2 = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], 1.0f)));
            const float e2 = fmaf(q[3], q[3], fmaf(q[4], q[4], q[5] * q[5]));
            float P;
            if (mlp_in_range(a.range, g2, e2)) {
                P = one_minus_exp_neg(2.0f * c.dens * a.dt * r);
            } else {
                fb = true;
                P = analytic_prob(q[0], q[1], q[2], q[3], q[4], q[5], c.dens, a.dt, a.gamma64, &x);
            }
            hit = c.u0 < P;
            if (a.prob_out) a.prob_out[c.p] = P;
            if (a.flag_out) a.flag_out[c.p] = hit ? 1 : 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (fb) ++n_fb;
        if (m) {
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(a.n_accepted, (uint32_t)__popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (hit) {
                a.accepted[at + __popc(m & ((1u << lane) - 1u))] =
                    AcceptedPair{c.ie, c.ig, x, c.p, {q[0], q[1], q[2]}, {q[3], q[4], q[5]}, {0u, 0u}};
                ++n_hit;
            }
        }
    }
    if (kCand) {
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
}

// Adds v summed over the warp to acc (lane 0 does the add).
__device__ __forceinline__ void warp_add(float* acc, float v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31u) == 0) atomicAdd(acc, v);
}

__global__ void __launch_bounds__(kPnetThreads, 2) k_pnet_train(PnetArgs a)
{
    __shared__ float th[kPnetParams];
    __shared__ float g[kPnetParams];
    for (int i = threadIdx.x; i < kPnetParams; i += blockDim.x) g[i] = 0.0f;
    stage_params(a.p, th);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    const unsigned lane = threadIdx.x & 31u;
    float loss_num = 0.0f, wsum = 0.0f;
    for (int64_t base = first; base < a.n; base += stride) {
        const int64_t s = base + lane;
        const bool live = s < a.n;
        float q[6] = {0, 0, 0, 0, 0, 0};
        float y = 0.0f, wt = 0.0f;
        if (live) {
            q[0] = a.u[0][s];
            q[1] = a.u[1][s];
            q[2] = a.u[2][s];
            q[3] = a.k[0][s];
            q[4] = a.k[1][s];
            q[5] = a.k[2][s];
            y = a.y[s];
            wt = a.wts ? a.wts[s] : 1.0f;
        }
        float f[9], h1[9], h2[12], h3[9];
        pnet_features(a.p, q, a.ln_we, a.ln_wg, a.ln_pmax, f);
        const float yp = pnet_forward(th, f, h1, h2, h3);
        const float err = yp - y;
        loss_num += wt * fabsf(err);
        wsum += wt;
        // d loss / d z of the output times sum w: w sign(err) sigma'(z) (the
        // Adam kernel divides by the weight sum)
        const float sgn = err > 0.0f ? 1.0f : (err < 0.0f ? -1.0f : 0.0f);
        const float dz3 = wt * sgn * yp * (1.0f - yp);
        // output layer
#pragma unroll
        for (int i = 0; i < 9; ++i) warp_add(&g[kP_W3 + i], dz3 * h3[i]);
        warp_add(&g[kP_B3], dz3);
        float dz2[9];
#pragma unroll
        for (int o = 0; o < 9; ++o) dz2[o] = h3[o] > 0.0f ? dz3 * th[kP_W3 + o] : 0.0f;
#pragma unroll
        for (int o = 0; o < 9; ++o) {
#pragma unroll
            for (int i = 0; i < 12; ++i) warp_add(&g[kP_W2 + 12 * o + i], dz2[o] * h2[i]);
            warp_add(&g[kP_B2 + o], dz2[o]);
        }
        float dz1[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            float d = 0.0f;
#pragma unroll
            for (int o = 0; o < 9; ++o) d = fmaf(th[kP_W2 + 12 * o + i], dz2[o], d);
            dz1[i] = h2[i] > 0.0f ? d : 0.0f;
        }
#pragma unroll
        for (int o = 0; o < 12; ++o) {
#pragma unroll
            for (int i = 0; i < 9; ++i) warp_add(&g[kP_W1 + 9 * o + i], dz1[o] * h1[i]);
            warp_add(&g[kP_B1 + o], dz1[o]);
        }
        float dz0[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            float d = 0.0f;
#pragma unroll
            for (int o = 0; o < 12; ++o) d = fmaf(th[kP_W1 + 9 * o + i], dz1[o], d);
            dz0[i] = h1[i] > 0.0f ? d : 0.0f;
        }
#pragma unroll
        for (int o = 0; o < 9; ++o) {
#pragma unroll
            for (int i = 0; i < 9; ++i) warp_add(&g[kP_W0 + 9 * o + i], dz0[o] * f[i]);
            warp_add(&g[kP_B0 + o], dz0[o]);
        }
    }
    warp_add(&a.loss[0], loss_num);
    warp_add(&a.loss[1], wsum);
    __syncthreads();
    for (int i = threadIdx.x; i < kPnetParams; i += blockDim.x) atomicAdd(&a.p.grad[i], g[i]);
}

__global__ void k_pnet_adam(PnetDev p, float lr, float b1t, float b2t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPnetParams) return;
    const float gr = p.grad[i] / p.loss[1];  // mean over the weights
    p.grad[i] = gr;
    const float m = 0.9f * p.adam_m[i] + 0.1f * gr;
    const float v = 0.999f * p.adam_v[i] + 0.001f * gr * gr;
    p.adam_m[i] = m;
    p.adam_v[i] = v;
    const float mh = m / (1.0f - b1t), vh = v / (1.0f - b2t);
    p.theta[i] -= lr * mh / (sqrtf(vh) + 1e-7f);
}

int pnet_grid(int64_t rows)
{
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    const int64_t want = (rows + kPnetThreads - 1) / kPnetThreads;
    const int64_t cap = (int64_t)n_sm * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

compton_status launch_pnet_infer(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                 const float* kx, const float* ky, const float* kz, int64_t n, float w_e, float w_g,
                                 float p_max, float* r_out, cudaStream_t stream)
{
    if (n <= 0) return COMPTON_OK;
    PnetArgs a{};
    a.p = ctx->pnet;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.n = n;
    a.ln_we = logf(w_e);
    a.ln_wg = logf(w_g);
    a.ln_pmax = logf(p_max);
    a.r_out = r_out;
    {
        TimedScope ts_(ctx, COMPTON_K_MLP, stream);
        k_pnet_infer<false><<<pnet_grid(n), kPnetThreads, 0, stream>>>(a);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_pnet_infer");
    return COMPTON_OK;
}

compton_status launch_pnet_decide(compton_ctx* ctx, int64_t rows, const MlpDecide& dec, const float* w_e,
                                  const float* w_g, cudaStream_t stream)
{
    PnetArgs a{};
    a.p = ctx->pnet;
    a.cand = ctx->cand;
    a.n_cand = ctx->n_cand;
    a.dt = dec.dt;
    a.gamma64 = dec.gamma64;
    a.ln_w = logf((float)ctx->cfg.w_over_v);
    a.w_e = w_e;
    a.w_g = w_g;
    a.prob_out = dec.prob_out;
    a.flag_out = dec.flag_out;
    a.accepted = ctx->accepted;
    a.n_accepted = ctx->n_accepted;
    a.stats = ctx->stats;
    a.range = ctx->mlp;
    a.range.range_g2max = ctx->pnet.range[0];
    a.range.range_e2min = ctx->pnet.range[1];
    a.range.range_e2max = ctx->pnet.range[2];
    {
        TimedScope ts_(ctx, COMPTON_K_MLP, stream);
        k_pnet_infer<true><<<pnet_grid(rows), kPnetThreads, 0, stream>>>(a);
    }
    COMPTON_LAUNCH_CHECK(ctx, "k_pnet_infer<cand>");
    return COMPTON_OK;
}

compton_status launch_pnet_train_step(compton_ctx* ctx, const float* ux, const float* uy, const float* uz,
                                      const float* kx, const float* ky, const float* kz, const float* y,
                                      const float* w, int64_t n, float w_e, float w_g, float p_max, float lr,
                                      cudaStream_t stream)
{
    if (n <= 0) return COMPTON_EINVAL;
    PnetDev& P = ctx->pnet;
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(P.grad, 0, sizeof(float) * kPnetParams, stream));
    COMPTON_CUDA_TRY(ctx, cudaMemsetAsync(P.loss, 0, sizeof(float) * 2, stream));
    PnetArgs a{};
    a.p = P;
    a.u[0] = ux;
    a.u[1] = uy;
    a.u[2] = uz;
    a.k[0] = kx;
    a.k[1] = ky;
    a.k[2] = kz;
    a.n = n;
    a.ln_we = logf(w_e);
    a.ln_wg = logf(w_g);
    a.ln_pmax = logf(p_max);
    a.y = y;
    a.wts = w;
    a.loss = P.loss;
    k_pnet_train<<<pnet_grid(n), kPnetThreads, 0, stream>>>(a);
    COMPTON_LAUNCH_CHECK(ctx, "k_pnet_train");
    ++P.step;
    const float b1t = powf(0.9f, (float)P.step), b2t = powf(0.999f, (float)P.step);
    k_pnet_adam<<<(kPnetParams + 127) / 128, 128, 0, stream>>>(P, lr, b1t, b2t);
    COMPTON_LAUNCH_CHECK(ctx, "k_pnet_adam");
    return COMPTON_OK;
}

}  // namespace compton
