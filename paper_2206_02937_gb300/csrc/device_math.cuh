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
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;  // one wide multiply: high and low halves
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
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

// Streams: pairing keys of electrons (1) and photons (2) at the particle id;
// the Bernoulli uniforms of pairs 4j..4j+3 as the four words of the stream-3
// block at counter j; the two angle words of pair p from stream 4 at p.
enum : uint32_t { kStreamPairE = 1u, kStreamPairG = 2u, kStreamScatter = 3u, kStreamAngle = 4u };

// Uniform on [0, 1) from the top 24 bits of a word (exact in FP32).
__device__ __forceinline__ float u24_closed0(uint32_t r) { return (float)(r >> 8) * 0x1.0p-24f; }

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

// sqrt(x) from the hardware reciprocal square root (a few ulp), 0 at 0.
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Straight-line form (no branch, so the pairs of a thread interleave): the
// reciprocal square roots give 1/gamma, 1/|u| and 1/|k| directly, so
// beta = |u|/gamma, 1 - beta = (1/gamma)/(gamma + |u|), cos psi = u.k/(|u||k|)
// and sin^2 psi = |u x k|^2/(|u|^2 |k|^2) need two divisions in all.  An
// electron at rest or a photon of zero energy gives v = 1 (x = gamma eps).
__device__ __forceinline__ Invariants invariants_f32(float ux, float uy, float uz, float kx, float ky, float kz)
{
    Invariants r;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float kk = fmaf(kx, kx, fmaf(ky, ky, kz * kz));
    const float ru = rsqrtf(uu), rk = rsqrtf(kk);
    const float g2 = 1.0f + uu;
    const float rg = rsqrtf(g2);  // 1/gamma
    const bool moving = uu > 0.0f, lit = kk > 0.0f;
    const float un = moving ? uu * ru : 0.0f;
    r.gamma = g2 * rg;
    r.eps = lit ? kk * rk : 0.0f;
    const float rur = ru * rk;
    const float cosp = fmaf(ux, kx, fmaf(uy, ky, uz * kz)) * rur;
    const float cx = diff_of_products(uy, kz, uz, ky);
    const float cy = diff_of_products(uz, kx, ux, kz);
    const float cz = diff_of_products(ux, ky, uy, kx);
    const float s2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz)) * rur * rur;  // sin^2 psi
    const float omc = cosp > 0.0f ? __fdividef(s2, 1.0f + cosp) : 1.0f - cosp;
    const float v = fmaf(un * rg, omc, __fdividef(rg, r.gamma + un));
    r.v = moving && lit ? v : 1.0f;
    r.x = r.gamma * r.eps * r.v;
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
//   C = int_0^t s(2-s)/(1+xs)^2 ds = [(2x+2) ln(1+w) - w - (2x+1) w/(1+w)] / x^3.
// C cancels for small |w|.  With z = w/(2+w) (ln(1+w) = 2 atanh z,
// w/(1+w) = 2z/(1+z)) and q = z/x = t/(2+w) it becomes
//   C = 4 q^2 [ z S1 + 1/(1+z) - q S2 ],   B = 2 q (1 + z^2 S1),
//   S1 = sum_{j>=1} z^(2j-2)/(2j+1),  S2 = sum_{j>=1} 2j/(2j+1) z^(2j-2),
// series of positive terms; since sum_{j>=1} z^(2j-2) = 1/(1 - z^2),
// S2 = 1/(1 - z^2) - S1 (about 2/3: no cancellation), so only S1 is summed.
// For -0.6 < w < 1 (z^2 < 0.19) twelve terms reach FP32 precision.  Outside
// that range the closed forms lose only a few bits.  sigma/sigma_T = 3/8 F(x, 2).
// ---------------------------------------------------------------------------
template <int kTerms>
__device__ __forceinline__ void kn_series(float z2, float& S1, float& S2)
{
    S1 = 0.0f;
#pragma unroll
    for (int j = kTerms; j >= 1; --j) S1 = fmaf(S1, z2, 1.0f / (float)(2 * j + 1));
    S2 = __fdividef(1.0f, 1.0f - z2) - S1;
}

// C(x, t) in the series range -0.6 < x t < 1 (x may be negative).
__device__ __forceinline__ float kn_C_series(float x, float t)
{
    const float w = x * t;
    const float q = __fdividef(t, 2.0f + w);
    const float z = x * q;
    float S1, S2;
    kn_series<12>(z * z, S1, S2);
    return 4.0f * q * q * (fmaf(z, S1, __fdividef(1.0f, 1.0f + z)) - q * S2);
}

__device__ __forceinline__ float kn_F(float x, float t)
{
    const float w = x * t;
    const float opw = 1.0f + w;
    const float A = __fdividef(t * (2.0f + w), 2.0f * opw * opw);
    if (w < 1.0f) {
        const float q = __fdividef(t, 2.0f + w);
        const float z = x * q;
        const float z2 = z * z;
        float S1, S2;
        kn_series<12>(z2, S1, S2);
        const float B = 2.0f * q * fmaf(z2, S1, 1.0f);
        const float C = 4.0f * q * q * (fmaf(z, S1, __fdividef(1.0f, 1.0f + z)) - q * S2);
        return A + B - C;
    }
    const float L = log1pf(w);
    const float B = __fdividef(L, x);
    const float C = __fdividef(fmaf(2.0f * x + 2.0f, L, -w) - (2.0f * x + 1.0f) * __fdividef(w, opw), x * x * x);
    return A + B - C;
}

// Complementary cumulative G(x, tau) = int_{2-tau}^{2} f(x, t) dt, computed
// without forming F(2) - F(2 - tau).  With a = 1 + 2x and d = 1 + x(2 - tau)
// (so a - d = x tau exactly):
//   int xi^3 = tau (a + d) / (2 a^2 d^2),   int xi = ln(a/d)/x = log1p(x tau/d)/x,
//   int xi^2 t(2-t) = C(-x/a, tau)/a^2, which for x tau/a >= 0.6 equals
//   [2 (1 + x) log1p(x tau/d) - x tau (d + 1)/d] / x^3.
__device__ __forceinline__ float kn_G(float x, float tau)
{
    const float a = fmaf(2.0f, x, 1.0f);
    const float d = fmaf(x, 2.0f - tau, 1.0f);
    const float Ac = __fdividef(tau * (a + d), 2.0f * a * a * d * d);
    const float Lc = log1pf(__fdividef(x * tau, d));
    const float Bc = x > 0.0f ? __fdividef(Lc, x) : tau;
    float Cc;
    if (x * tau < 0.6f * a) {
        Cc = __fdividef(kn_C_series(-__fdividef(x, a), tau), a * a);
    } else {
        Cc = __fdividef(fmaf(2.0f * (1.0f + x), Lc, -__fdividef(x * tau * (d + 1.0f), d)), x * x * x);
    }
    return Ac + Bc - Cc;
}

// Angular density at t (lower branch) and at t = 2 - s (upper branch).
__device__ __forceinline__ float kn_f_lower(float x, float t)
{
    const float xi = __fdividef(1.0f, fmaf(x, t, 1.0f));
    const float xi2 = xi * xi;
    return fmaf(xi2, xi, xi) - xi2 * t * (2.0f - t);
}
__device__ __forceinline__ float kn_f_upper(float x, float s)
{
    const float xi = __fdividef(1.0f, fmaf(x, 2.0f - s, 1.0f));
    const float xi2 = xi * xi;
    return fmaf(xi2, xi, xi) - xi2 * s * (2.0f - s);
}

// sigma_KN(x) / sigma_T
// F(x, 2) = (8/3) sigma_KN(x)/sigma_T, the total of the angular cumulative.  At
// t = 2: w = 2x, q = 1/(1+x), z = x/(1+x), and with r = 1/(1+2x) also
// 1/(1+z) = (1+x) r, 1/(1-z^2) = (1+x)^2 r, A = 2(1+x) r^2: two reciprocals.
// For x < 1 (z^2 < 1/4) twelve terms of S1 reach FP32 precision.
__device__ __forceinline__ float kn_F2_series(float x)
{
    const float opx = 1.0f + x;
    const float q = __fdividef(1.0f, opx);
    const float r = __fdividef(1.0f, fmaf(2.0f, x, 1.0f));
    const float z = x * q;
    const float z2 = z * z;
    float S1 = 0.0f;
#pragma unroll
    for (int j = 12; j >= 1; --j) S1 = fmaf(S1, z2, 1.0f / (float)(2 * j + 1));
    const float S2 = opx * opx * r - S1;
    const float A = 2.0f * opx * r * r;
    const float B = 2.0f * q * fmaf(z2, S1, 1.0f);
    const float C = 4.0f * q * q * (fmaf(z, S1, opx * r) - q * S2);
    return A + B - C;
}

__device__ __forceinline__ float kn_F2(float x) { return x < 1.0f ? kn_F2_series(x) : kn_F(x, 2.0f); }

__device__ __forceinline__ float kn_sigma(float x) { return 0.375f * kn_F2(x); }

// ---------------------------------------------------------------------------
// Scattering angle from the 24-bit draw r24 (u1 = (r24 + 1/2) 2^-24).
// Lower half (r24 < 2^23): solve F(x, t) = u1 F(x, 2) for t.  Upper half:
// solve G(x, tau) = (1 - u1) F(x, 2) for tau = 2 - t, with
// 1 - u1 = (2^24 - 1 - r24 + 1/2) 2^-24 formed exactly, so that directions
// near backscatter (t -> 2) keep full relative precision in tau.
// Start: the exact root of the Thomson-limit cubic (x -> 0, where both halves
// follow 2s - s^2 + s^3/3 = 8 uu/3, i.e. y^3 + 3y = 8uu - 4 with y = s - 1,
// Cardano's formula) for x < 1; for x >= 1 the large-x forms
// s = expm1(x target)/x (lower) or target/f(x, 2) (upper).  Then at most eight
// Newton steps inside a shrinking bracket (bisection when a step leaves it).
// Returns cos(theta'), sin(theta') and 1/(1 + x t) (the Compton energy ratio).
// ---------------------------------------------------------------------------
struct Angle {
    float cth, sth, ratio;
};

__device__ __forceinline__ Angle kn_sample_angle(float x, uint32_t r24, float F2)
{
    const bool upper = r24 >= (1u << 23);
    const float uu = ((float)(upper ? 16777215u - r24 : r24) + 0.5f) * 0x1.0p-24f;
    const float target = uu * F2;
    float s;
    if (x < 1.0f) {
        const float q = fmaf(8.0f, uu, -4.0f);
        const float D = sqrtf(fmaf(0.25f * q, q, 1.0f));
        s = cbrtf(0.5f * q + D) + cbrtf(0.5f * q - D) + 1.0f;
    } else {
        s = upper ? __fdividef(target, kn_f_upper(x, 0.0f)) : __fdividef(expm1f(target * x), x);
    }
    float lo = 0.0f, hi = 2.0f;
    s = fminf(fmaxf(s, 0.0f), 2.0f);
    for (int it = 0; it < 8; ++it) {
        const float R = (upper ? kn_G(x, s) : kn_F(x, s)) - target;
        if (R == 0.0f) break;
        if (R < 0.0f) lo = s; else hi = s;
        float sn = s - __fdividef(R, upper ? kn_f_upper(x, s) : kn_f_lower(x, s));
        const bool newton = sn >= lo && sn <= hi;
        if (!newton) sn = 0.5f * (lo + hi);
        // a Newton step this small is at the FP32 resolution of s: the next
        // one would only move s between neighbouring floats
        const bool done = newton && fabsf(sn - s) <= 2.5e-7f * s;
        s = sn;
        if (done) break;
    }
    Angle a;
    a.cth = upper ? s - 1.0f : 1.0f - s;
    a.sth = sqrtf(s * (2.0f - s));
    a.ratio = __fdividef(1.0f, upper ? fmaf(x, 2.0f - s, 1.0f) : fmaf(x, s, 1.0f));
    return a;
}

// ---------------------------------------------------------------------------
// FP64 reciprocal, reciprocal square root and square root from an FP32 seed
// and one Newton-Raphson step (the seed's error squares: within 5e-14
// relative, checked against CUDA's correctly rounded operators).  Arguments
// far outside the FP32 range take the full-precision operator instead.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_nr(double d)
{
    const double ad = fabs(d);
    if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
    const double y = (double)__frcp_rn((float)d);
    return fma(y, fma(-d, y, 1.0), y);
}

__device__ __forceinline__ double rsqrt_nr(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    const double y = (double)rsqrtf((float)d);
    return fma(0.5 * y, fma(-d * y, y, 1.0), y);
}

__device__ __forceinline__ double sqrt_nr(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return sqrt(d);
    const float s0 = sqrtf((float)d);
    const double s = (double)s0;
    return fma(fma(-s, s, d), (double)(0.5f / s0), s);
}

// ---------------------------------------------------------------------------
// The same collision in FP32, in a form without cancellation.  With u = |u| u^
// and beta = |u|/gamma, split every vector into its parts along u^ and across
// it; the part across is taken from cross products (no subtraction), and the
// part along from the identities
//   boost to the rest frame:  k'_par = gamma eps (c_psi - beta),
//   boost back:               k1_par = gamma eps1' (c + beta),
// with c_psi = u^.k^ and c = u^.d (d the scattered rest-frame direction);
// when the two terms of (c_psi - beta) or (c + beta) nearly cancel they are
// formed as (1/gamma^2 - s_psi^2)/(c_psi + beta) and
// (s^2 - 1/gamma^2)/(beta - c), s^2 = 1 - c^2 from the cross product, whose
// denominators do not cancel.  So no step loses digits: the photon emitted
// backward in the electron frame, whose lab energy is a small fraction of
// gamma eps1', keeps FP32 relative accuracy, and both momenta match the FP64
// formulas to a few times 1e-7 of their own magnitude (only u <- u + k - k1
// can lose digits, when the electron ends far slower than it was).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross3(float a0, float a1, float a2, float b0, float b1, float b2, float& c0, float& c1,
                                       float& c2)
{
    c0 = diff_of_products(a1, b2, a2, b1);
    c1 = diff_of_products(a2, b0, a0, b2);
    c2 = diff_of_products(a0, b1, a1, b0);
}

__device__ __forceinline__ void collide_f32(float& ux, float& uy, float& uz, float& kx, float& ky, float& kz,
                                            float x, Angle ang, float u2)
{
    const float U0 = ux, U1 = uy, U2 = uz, K0 = kx, K1 = ky, K2 = kz;
    const float uu = fmaf(U0, U0, fmaf(U1, U1, U2 * U2));
    const float kk = fmaf(K0, K0, fmaf(K1, K1, K2 * K2));
    const float rg = rsqrtf(1.0f + uu);  // 1/gamma
    const float gamma = (1.0f + uu) * rg;
    const float ig2 = rg * rg;           // 1/gamma^2 = 1 - beta^2
    const float rk = rsqrtf(kk);
    // the photon energy eps = kk rk enters only through x and the unit vector e
    const bool moving = uu > 0.0f;
    const float ru = moving ? rsqrtf(uu) : 0.0f;
    const float un = uu * ru;
    const float beta = un * rg;
    // unit vectors along u (any unit vector at rest) and along k
    const float h0 = moving ? U0 * ru : 0.0f, h1 = moving ? U1 * ru : 0.0f, h2 = moving ? U2 * ru : 1.0f;
    const float e0 = K0 * rk, e1 = K1 * rk, e2 = K2 * rk;
    // incoming photon in the rest frame: across part eps (h x e) x h, along part gamma eps (c_psi - beta)
    float c0, c1, c2;
    cross3(h0, h1, h2, e0, e1, e2, c0, c1, c2);
    const float sp2 = fmaf(c0, c0, fmaf(c1, c1, c2 * c2));
    const float cp = fmaf(h0, e0, fmaf(h1, e1, h2 * e2));
    const float cmb = cp > 0.0f ? __fdividef(ig2 - sp2, cp + beta) : cp - beta;
    float p0, p1, p2;
    cross3(c0, c1, c2, h0, h1, h2, p0, p1, p2);
    const float along = gamma * cmb;
    const float r0 = fmaf(along, h0, p0), r1 = fmaf(along, h1, p1), r2 = fmaf(along, h2, p2);
    const float inv = rsqrtf(fmaf(r0, r0, fmaf(r1, r1, r2 * r2)));
    const float n0 = r0 * inv, n1 = r1 * inv, n2 = r2 * inv;
    // scattered direction: polar angle theta' from n, azimuth in the
    // orthonormal basis of Duff et al. completing n
    const float sg = n2 >= 0.0f ? 1.0f : -1.0f;
    const float a = -__fdividef(1.0f, sg + n2);
    const float b = n0 * n1 * a;
    const float b10 = fmaf(sg * n0 * n0, a, 1.0f), b11 = sg * b, b12 = -sg * n0;
    const float b20 = b, b21 = fmaf(n1 * n1, a, sg), b22 = -n1;
    float sph, cph;
    sincospif(2.0f * u2, &sph, &cph);
    const float e1r = x * ang.ratio;
    const float d0 = fmaf(ang.cth, n0, ang.sth * fmaf(cph, b10, sph * b20));
    const float d1 = fmaf(ang.cth, n1, ang.sth * fmaf(cph, b11, sph * b21));
    const float d2 = fmaf(ang.cth, n2, ang.sth * fmaf(cph, b12, sph * b22));
    // back to the lab: across part eps1' (h x d) x h, along part gamma eps1' (c + beta)
    float x0, x1, x2;
    cross3(h0, h1, h2, d0, d1, d2, x0, x1, x2);
    const float s2 = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
    const float c = fmaf(h0, d0, fmaf(h1, d1, h2 * d2));
    const float cpb = c < 0.0f ? __fdividef(s2 - ig2, beta - c) : c + beta;
    float q0, q1, q2;
    cross3(x0, x1, x2, h0, h1, h2, q0, q1, q2);
    const float al = gamma * cpb;
    const float k10 = e1r * fmaf(al, h0, q0), k11 = e1r * fmaf(al, h1, q1), k12 = e1r * fmaf(al, h2, q2);
    ux = (U0 + K0) - k10;
    uy = (U1 + K1) - k11;
    uz = (U2 + K2) - k12;
    kx = k10;
    ky = k11;
    kz = k12;
}

// 1 - exp(-a) for a >= 0 without cancellation: the Taylor series of
// -expm1(-a) in nested form below a = 1/4 (truncation < 4e-10 relative),
// 1 - exp(-a) above it (where the result is >= 0.22).
__device__ __forceinline__ float one_minus_exp_neg(float a)
{
    float s = 1.0f - a * (1.0f / 8.0f);
    s = 1.0f - a * (1.0f / 7.0f) * s;
    s = 1.0f - a * (1.0f / 6.0f) * s;
    s = 1.0f - a * (1.0f / 5.0f) * s;
    s = 1.0f - a * (1.0f / 4.0f) * s;
    s = 1.0f - a * (1.0f / 3.0f) * s;
    s = 1.0f - a * 0.5f * s;
    const float e = 1.0f - __expf(-a);
    return a < 0.25f ? a * s : e;  // both evaluated: no divergence
}

// ---------------------------------------------------------------------------
// Collision of one accepted pair, in FP64 (rest-frame boost and momentum
// update, where cancellation at large gamma breaks FP32):
//   photon in the electron rest frame: k' = k + u [ (u.k)/(gamma+1) - eps ],
//   direction n = k'/|k'|, scattered rest-frame photon of energy
//   x/(1 + x t) at polar angle theta' from n and azimuth phi in the
//   orthonormal basis of Duff et al. (JCGT 6(1), 2017), boosted back with
//   k1 = k1' + u [ (u.k1')/(gamma+1) + eps1' ], and u <- u + k - k1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void collide_f64(float& ux, float& uy, float& uz, float& kx, float& ky, float& kz,
                                            float x, Angle ang, float u2)
{
    const double U0 = ux, U1 = uy, U2 = uz, K0 = kx, K1 = ky, K2 = kz;
    const double gamma = sqrt_nr(1.0 + (U0 * U0 + U1 * U1 + U2 * U2));
    const double eps = sqrt_nr(K0 * K0 + K1 * K1 + K2 * K2);
    const double uk = U0 * K0 + U1 * K1 + U2 * K2;
    const double igp1 = rcp_nr(gamma + 1.0);
    const double f = fma(uk, igp1, -eps);
    const double r0 = fma(U0, f, K0), r1 = fma(U1, f, K1), r2 = fma(U2, f, K2);
    const double inv = rsqrt_nr(r0 * r0 + r1 * r1 + r2 * r2);
    const double n0 = r0 * inv, n1 = r1 * inv, n2 = r2 * inv;
    // Duff et al. basis completing n
    const double sg = n2 >= 0.0 ? 1.0 : -1.0;
    const double a = -rcp_nr(sg + n2);
    const double b = n0 * n1 * a;
    const double b10 = fma(sg * n0 * n0, a, 1.0), b11 = sg * b, b12 = -sg * n0;
    const double b20 = b, b21 = fma(n1 * n1, a, sg), b22 = -n1;
    float sphf, cphf;
    sincospif(2.0f * u2, &sphf, &cphf);
    const double cth = ang.cth, sth = ang.sth, cph = cphf, sph = sphf;
    const double e1r = (double)x * (double)ang.ratio;
    const double d0 = fma(cth, n0, sth * fma(cph, b10, sph * b20));
    const double d1 = fma(cth, n1, sth * fma(cph, b11, sph * b21));
    const double d2 = fma(cth, n2, sth * fma(cph, b12, sph * b22));
    const double q0 = e1r * d0, q1 = e1r * d1, q2 = e1r * d2;
    const double g = fma(U0 * q0 + U1 * q1 + U2 * q2, igp1, e1r);
    const double k10 = fma(U0, g, q0), k11 = fma(U1, g, q1), k12 = fma(U2, g, q2);
    ux = (float)((U0 + K0) - k10);
    uy = (float)((U1 + K1) - k11);
    uz = (float)((U2 + K2) - k12);
    kx = (float)k10;
    ky = (float)k11;
    kz = (float)k12;
}

// ---------------------------------------------------------------------------
// The collision of one accepted pair: FP64 when gamma eps exceeds the
// configured threshold (c64sq = its square), FP32 below it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void collide_pair(float& ux, float& uy, float& uz, float& kx, float& ky, float& kz,
                                             float x, Angle ang, float u2, float c64sq)
{
    const float ge2 = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, 1.0f))) * fmaf(kx, kx, fmaf(ky, ky, kz * kz));
    if (ge2 > c64sq) collide_f64(ux, uy, uz, kx, ky, kz, x, ang, u2);
    else collide_f32(ux, uy, uz, kx, ky, kz, x, ang, u2);
}

// ---------------------------------------------------------------------------
// The analytic probability of one pair, P = 1 - exp(-n dt sigma_KN(x)/sigma_T
// v), and its rest-frame photon energy x; FP64 invariants for electrons above
// gamma64, the series or closed-form sigma_KN as x requires.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float analytic_prob(float ux, float uy, float uz, float kx, float ky, float kz, float dens,
                                              float dt, float gamma64, float* x_out)
{
    const Invariants inv = invariants_f32(ux, uy, uz, kx, ky, kz);
    float x = inv.x, v = inv.v;
    if (inv.gamma > gamma64) invariants_f64(ux, uy, uz, kx, ky, kz, &x, &v);
    *x_out = x;
    return inv.eps > 0.0f ? one_minus_exp_neg(dens * dt * 0.375f * kn_F2(x) * v) : 0.0f;
}

}  // namespace compton
