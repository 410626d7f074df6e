// features.cuh -- the surrogate network's inputs from a pair's momenta.
//
// Momenta (the paper's choice, Sec. 3.2: the network sees the particles'
// momenta):  f = [sgnlog(u_i / s_u) / n_u, sgnlog(k_i / s_k) / n_k],
// sgnlog(z) = sign(z) log(1 + |z|), with the scales fs = {s_u, n_u, s_k, n_k}
// (kFast: the hardware-log form, for the BF16 / E4M3 tensor-core network).
// Invariants (an ablation of that choice): f = [ln(x) / 8, ln(v) / 8, 0, 0,
// 0, 0] with x the photon energy in the electron rest frame and
// v = 1 - beta cos psi, from the cancellation-free FP32 invariants.
#pragma once
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {

__device__ __forceinline__ float sgnlog(float z) { return copysignf(log1pf(fabsf(z)), z); }

// The same with the hardware log2 (lg2.approx, absolute error about 2^-22):
// ln(1 + a) = log2(1 + a) ln 2 for a >= 2^-6, and below it the series
// a - a^2/2 + a^3/3 (truncation below a^4/4 <= 1.5e-8 relative); absolute
// error below 2e-7, far under the BF16 and E4M3 rounding of the tensor-core
// inputs (the FP32 network keeps sgnlog).
__device__ __forceinline__ float sgnlog_fast(float z)
{
    const float a = fabsf(z);
    const float big = __log2f(1.0f + a) * 0.69314718055994531f;
    const float small = a * fmaf(a, fmaf(a, 1.0f / 3.0f, -0.5f), 1.0f);
    return copysignf(a >= 0.015625f ? big : small, z);
}

template <bool kFast = false>
__device__ __forceinline__ void features(const MlpDev& m, float ux, float uy, float uz, float kx, float ky, float kz,
                                         float* f)
{
    if (m.feat_mode == COMPTON_FEATURES_INVARIANTS) {
        const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
        f[0] = logf(fmaxf(inv.x, 1e-30f)) * 0.125f;
        f[1] = logf(fmaxf(inv.v, 1e-30f)) * 0.125f;
        f[2] = f[3] = f[4] = f[5] = 0.0f;
        return;
    }
    const float iu = __fdividef(1.0f, m.fs[0]), nu = __fdividef(1.0f, m.fs[1]);
    const float ik = __fdividef(1.0f, m.fs[2]), nk = __fdividef(1.0f, m.fs[3]);
    if (kFast) {
        f[0] = sgnlog_fast(ux * iu) * nu;
        f[1] = sgnlog_fast(uy * iu) * nu;
        f[2] = sgnlog_fast(uz * iu) * nu;
        f[3] = sgnlog_fast(kx * ik) * nk;
        f[4] = sgnlog_fast(ky * ik) * nk;
        f[5] = sgnlog_fast(kz * ik) * nk;
        return;
    }
    f[0] = sgnlog(ux * iu) * nu;
    f[1] = sgnlog(uy * iu) * nu;
    f[2] = sgnlog(uz * iu) * nu;
    f[3] = sgnlog(kx * ik) * nk;
    f[4] = sgnlog(ky * ik) * nk;
    f[5] = sgnlog(kz * ik) * nk;
}

}  // namespace compton
