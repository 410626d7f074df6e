// device_math.cuh -- per-pair arithmetic of the Compton step on the GPU.
//
// Everything here is device code used by the binning and scattering kernels:
//   * Philox4x32-10 (Salmon et al., SC'11), the counter-based generator that
//     draws the pairing keys and the collision randoms (Sec. 3.1);
//   * the pair invariants x (photon energy in the electron rest frame) and
//     v = 1 - beta cos(psi) (flux factor back to the simulation frame), formed
//     without cancellation in FP32 (Sec. 3.2: boost to the lepton frame and
//     back);
//   * the Klein-Nishina total cross section and its cumulative angular
//     distribution in FP32 (Sec. 3.2);
//   * the inverse-CDF sampler of the scattering angle and the FP64 momentum
//     update of a collided pair (Sec. 3.1, "the kinetic collision is
//     resolved").
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace compton {

// ---------------------------------------------------------------------------
// Philox4x32-10 from its published definition: ten rounds; each round takes
// the two 32x32->64 products of words 0 and 2 with the round multipliers,
// xors the high halves with words 1 and 3 and the key, and permutes; the key
// advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct Philox4 {
    uint32_t r0, r1, r2, r3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Counter layout: (id, step low word, stream, step high word), key = seed.
__device__ __forceinline__ Philox4 draw(uint64_t seed, uint64_t step, uint32_t stream, uint32_t id)
{
    return philox4x32_10(id, (uint32_t)step, stream, (uint32_t)(step >> 32), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

enum : uint32_t { kStreamPairE = 1u, kStreamPairG = 2u, kStreamScatter = 3u };

__device__ __forceinline__ float u24_closed0(uint32_t r) { return (float)(r >> 8) * 0x1.0p-24f; }
__device__ __forceinline__ float u24_open(uint32_t r) { return ((float)(r >> 8) + 0.5f) * 0x1.0p-24f; }

// ---------------------------------------------------------------------------
// a*b - c*d with one rounding error at most 1.5 ulp: Kahan's algorithm with a
// fused multiply-add recovering the rounding error of c*d (analysed by
// Jeannerod, Louvet and Muller, Math. Comp. 82, 2013).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d)
{
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

// ---------------------------------------------------------------------------
// Pair invariants.  gamma = sqrt(1+|u|^2), eps = |k|,
//   1 - beta     = 1 / (gamma (gamma + |u|))
//   1 - cos psi  = sin^2 psi / (1 + cos psi) for cos psi > 0, with sin psi from
//                  the cross product u x k, else 1 - cos psi directly,
//   v = (1 - beta) + beta (1 - cos psi),  x = gamma eps v.
// No step subtracts nearly equal quantities, so FP32 keeps ~1e-6 relative
// accuracy for any gamma.
// ---------------------------------------------------------------------------
struct Invariants {
    float x, v, gamma, eps;
};

__device__ __forceinline__ Invariants invariants_f32(float ux, float uy, float uz, float kx, float ky, float kz)
{
    Invariants r;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float un = sqrtf(uu);
    r.gamma = sqrtf(1.0f + uu);
    r.eps = sqrtf(fmaf(kx, kx, fmaf(ky, ky, kz * kz)));
    float v = 1.0f;
    if (un > 0.0f && r.eps > 0.0f) {
        const float beta = un / r.gamma;
        const float omb = 1.0f / (r.gamma * (r.gamma + un));
        const float uk = fmaf(ux, kx, fmaf(uy, ky, uz * kz));
        const float ue = un * r.eps;
        const float cosp = uk / ue;
        float omc;
        if (cosp > 0.0f) {
            const float cx = diff_of_products(uy, kz, uz, ky);
            const float cy = diff_of_products(uz, kx, ux, kz);
            const float cz = diff_of_products(ux, ky, uy, kx);
            const float sn = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz))) / ue;
            omc = sn * sn / (1.0f + cosp);
        } else {
            omc = 1.0f - cosp;
        }
        v = fmaf(beta, omc, omb);
    }
    r.v = v;
    r.x = r.gamma * r.eps * v;
    return r;
}

// The same invariants in FP64 (used for electrons above the configured gamma).
__device__ __forceinline__ void invariants_f64(float ux, float uy, float uz, float kx, float ky, float kz,
                                               float* x_out, float* v_out)
{
    const double Ux = ux, Uy = uy, Uz = uz, Kx = kx, Ky = ky, Kz = kz;
    const double uu = Ux * Ux + Uy * Uy + Uz * Uz;
    const double un = sqrt(uu);
    const double gamma = sqrt(1.0 + uu);
    const double eps = sqrt(Kx * Kx + Ky * Ky + Kz * Kz);
    double v = 1.0;
    if (un > 0.0 && eps > 0.0) {
        const double beta = un / gamma;
        const double omb = 1.0 / (gamma * (gamma + un));
        const double cosp = (Ux * Kx + Uy * Ky + Uz * Kz) / (un * eps);
        double omc;
        if (cosp > 0.0) {
            // products of two FP32 values are exact in FP64
            const double cx = Uy * Kz - Uz * Ky, cy = Uz * Kx - Ux * Kz, cz = Ux * Ky - Uy * Kx;
            const double sn = sqrt(cx * cx + cy * cy + cz * cz) / (un * eps);
            omc = sn * sn / (1.0 + cosp);
        } else {
            omc = 1.0 - cosp;
        }
        v = omb + beta * omc;
    }
    *x_out = (float)(gamma * eps * v);
    *v_out = (float)v;
}

// ---------------------------------------------------------------------------
// Klein-Nishina cumulative cross section in FP32.
// With xi = 1/(1 + x t), t = 1 - cos(theta') in [0, 2], the angular density
// per unit t (azimuth integrated, in units of 3/8 sigma_T) is
//   f(x, t) = xi^3 + xi - xi^2 t (2 - t),
// and its integral from 0 to t is F = A + B - C with w = x t:
//   A = t (2 + w) / (2 (1 + w)^2)
//   B = ln(1 + w) / x
//   C = 2 g1(w) / x^2 - g2(w) / x^3,
//   g1 = ln(1+w) - w/(1+w),  g2 = w - 2 ln(1+w) + w/(1+w).
// g1 and g2 cancel for small w.  With z = w/(2+w) (so ln(1+w) = 2 atanh z and
// w/(1+w) = 2z/(1+z)) both become sums of positive terms:
//   g1 = 2 z^2 [ z S1 + 1/(1+z) ],   g2 = 4 z^3 S2,
//   S1 = sum_{j>=1} z^(2j-2)/(2j+1),  S2 = sum_{j>=1} 2j/(2j+1) z^(2j-2),
// and with q = z/x = t/(2+w):  B = 2q (1 + z^2 S1),
//   C = 4 q^2 [ z S1 + 1/(1+z) ] - 4 q^3 S2.
// For w < 1 (z^2 < 1/9) ten terms of S1, S2 reach FP32 precision; above it the
// direct forms lose at most a few bits.  The total cross section is
// sigma/sigma_T = 3/8 F(x, 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kn_F(float x, float t)
{
    const float w = x * t;
    const float opw = 1.0f + w;
    const float A = t * (2.0f + w) / (2.0f * opw * opw);
    float B, C;
    if (w < 1.0f) {
        const float q = t / (2.0f + w);
        const float z = x * q;
        const float z2 = z * z;
        float S1 = 0.0f, S2 = 0.0f;
#pragma unroll
        for (int j = 10; j >= 1; --j) {
            S1 = fmaf(S1, z2, 1.0f / (float)(2 * j + 1));
            S2 = fmaf(S2, z2, (float)(2 * j) / (float)(2 * j + 1));
        }
        B = 2.0f * q * fmaf(z2, S1, 1.0f);
        const float q2 = q * q;
        C = 4.0f * q2 * (fmaf(z, S1, 1.0f / (1.0f + z)) - q * S2);
    } else {
        const float L = log1pf(w);
        const float r = w / opw;
        B = L / x;
        C = (2.0f * x * (L - r) - (w - 2.0f * L + r)) / (x * x * x);
    }
    return A + B - C;
}

__device__ __forceinline__ float kn_f(float x, float t)
{
    const float xi = 1.0f / fmaf(x, t, 1.0f);
    const float xi2 = xi * xi;
    return fmaf(xi2, xi, xi) - xi2 * t * (2.0f - t);
}

// sigma_KN(x) / sigma_T
__device__ __forceinline__ float kn_sigma(float x) { return 0.375f * kn_F(x, 2.0f); }

// ---------------------------------------------------------------------------
// Scattering angle: the t in [0, 2] with F(x, t) = u1 F(x, 2).  Start from the
// exact root of the Thomson-limit cubic (x -> 0: F = 2t - t^2 + t^3/3, i.e.
// y^3 + 3y = 8 u1 - 4 with y = t - 1, solved by Cardano's formula) for x < 1,
// or from the large-x form F ~ ln(1 + x t)/x otherwise, then at most eight
// Newton steps kept inside a shrinking bracket (bisection when a step leaves
// it).  F is strictly increasing, so the bracket always holds the root.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kn_sample_t(float x, float u1, float F2)
{
    const float target = u1 * F2;
    float t;
    if (x < 1.0f) {
        const float q = fmaf(8.0f, u1, -4.0f);
        const float D = sqrtf(fmaf(0.25f * q, q, 1.0f));
        t = cbrtf(0.5f * q + D) + cbrtf(0.5f * q - D) + 1.0f;
    } else {
        t = expm1f(target * x) / x;
    }
    float lo = 0.0f, hi = 2.0f;
    t = fminf(fmaxf(t, 0.0f), 2.0f);
    for (int it = 0; it < 8; ++it) {
        const float R = kn_F(x, t) - target;
        if (R == 0.0f) break;
        if (R < 0.0f) lo = t; else hi = t;
        float tn = t - R / kn_f(x, t);
        if (!(tn >= lo && tn <= hi)) tn = 0.5f * (lo + hi);
        if (tn == t) break;
        t = tn;
    }
    return t;
}

// ---------------------------------------------------------------------------
// Collision of one accepted pair, in FP64 (rest-frame boost and momentum
// update, where cancellation at large gamma breaks FP32):
//   photon in the electron rest frame: k' = k + u [ (u.k)/(gamma+1) - eps ],
//   direction n = k'/|k'|, scattered rest-frame photon of energy
//   x/(1 + x t) at polar angle acos(1 - t) from n and azimuth phi in the
//   orthonormal basis of Duff et al. (JCGT 6(1), 2017), boosted back with
//   k1 = k1' + u [ (u.k1')/(gamma+1) + eps1' ], and u <- u + k - k1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void collide_f64(float& ux, float& uy, float& uz, float& kx, float& ky, float& kz,
                                            float x, float t, float u2)
{
    const double U0 = ux, U1 = uy, U2 = uz, K0 = kx, K1 = ky, K2 = kz;
    const double gamma = sqrt(1.0 + (U0 * U0 + U1 * U1 + U2 * U2));
    const double eps = sqrt(K0 * K0 + K1 * K1 + K2 * K2);
    const double uk = U0 * K0 + U1 * K1 + U2 * K2;
    const double f = uk / (gamma + 1.0) - eps;
    const double r0 = K0 + U0 * f, r1 = K1 + U1 * f, r2 = K2 + U2 * f;
    const double inv = 1.0 / sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    const double n0 = r0 * inv, n1 = r1 * inv, n2 = r2 * inv;
    // Duff et al. basis completing n
    const double sg = copysign(1.0, n2);
    const double a = -1.0 / (sg + n2);
    const double b = n0 * n1 * a;
    const double b10 = 1.0 + sg * n0 * n0 * a, b11 = sg * b, b12 = -sg * n0;
    const double b20 = b, b21 = sg + n1 * n1 * a, b22 = -n1;
    float sphf, cphf;
    sincospif(2.0f * u2, &sphf, &cphf);
    const double cth = 1.0 - (double)t;
    const double sth = sqrt((double)t * (2.0 - (double)t));
    const double xd = x;
    const double e1r = xd / (1.0 + xd * (double)t);
    const double cph = cphf, sph = sphf;
    const double d0 = cth * n0 + sth * (cph * b10 + sph * b20);
    const double d1 = cth * n1 + sth * (cph * b11 + sph * b21);
    const double d2 = cth * n2 + sth * (cph * b12 + sph * b22);
    const double q0 = e1r * d0, q1 = e1r * d1, q2 = e1r * d2;
    const double uq = U0 * q0 + U1 * q1 + U2 * q2;
    const double g = uq / (gamma + 1.0) + e1r;
    const double k10 = q0 + U0 * g, k11 = q1 + U1 * g, k12 = q2 + U2 * g;
    ux = (float)(U0 + K0 - k10);
    uy = (float)(U1 + K1 - k11);
    uz = (float)(U2 + K2 - k12);
    kx = (float)k10;
    ky = (float)k11;
    kz = (float)k12;
}

}  // namespace compton
