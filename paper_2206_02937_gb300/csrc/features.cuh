// features.cuh -- the surrogate network's inputs from a pair's momenta.
//
// Momenta (the paper's choice, Sec. 3.2: the network sees the particles'
// momenta):  f = [sgnlog(u_i / s_u) / n_u, sgnlog(k_i / s_k) / n_k],
// sgnlog(z) = sign(z) log(1 + |z|), with the scales fs = {s_u, n_u, s_k, n_k}.
// Invariants (an ablation of that choice): f = [ln(x) / 8, ln(v) / 8, 0, 0,
// 0, 0] with x the photon energy in the electron rest frame and
// v = 1 - beta cos psi, from the cancellation-free FP32 invariants.
#pragma once
#include "ctx.hpp"
#include "device_math.cuh"

namespace compton {

__device__ __forceinline__ float sgnlog(float z) { return copysignf(log1pf(fabsf(z)), z); }

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
    f[0] = sgnlog(ux * iu) * nu;
    f[1] = sgnlog(uy * iu) * nu;
    f[2] = sgnlog(uz * iu) * nu;
    f[3] = sgnlog(kx * ik) * nk;
    f[4] = sgnlog(ky * ik) * nk;
    f[5] = sgnlog(kz * ik) * nk;
}

}  // namespace compton
