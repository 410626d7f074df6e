// act_math.cuh -- the SiLU activation of the surrogate network's tensor-core
// epilogue, two samples' values at a time.
//
// Blackwell's paired FP32 instructions (add / mul / fma .rn.f32x2: one
// instruction, two independent results, each rounded as the scalar operation
// would be) halve the instructions of the element-wise work.  A pair lives in
// one 64-bit register: the low half is the first value.
//
// SiLU(z) = z sigma(z) = h (1 + tanh h) with h = z / 2.  Two forms:
//   silu2_mufu  tanh.approx.f32 on the multi-function unit, then one paired
//               FMA: y = h + h tanh(h).
//   silu2_fma   the same value computed on the FMA pipe only, so that a share
//               of a row's activations does not queue on the multi-function
//               unit:  sigma(z) = 1 / (1 + E),  E = 2^y,  y = -z log2(e),
//               * y clamped to [-126, 126] (E then stays a normal float; below
//                 -126 the sum 1 + E is 1 in FP32 anyway, above 126 sigma is
//                 below 1e-38) with a saturating FMA,
//               * 2^y by range reduction y = j + f, j = rint(y), |f| <= 1/2
//                 (j taken with the round-to-nearest shifter 1.5 * 2^23, f
//                 exact by Sterbenz), 2^f from a degree-3 polynomial that is
//                 minimax for relative error on [-1/2, 1/2] (Remez exchange;
//                 7.5e-5), and 2^j put into the exponent field by an integer
//                 multiply-add,
//               * 1/d for d = (1 + E) / 2 (so that the reciprocal is 2 sigma
//                 and SiLU = h / d) by Newton-Raphson iteration
//                 r <- r + r (1 - d r) from the seed whose bits are
//                 K - bits(d); K = 0x7EF311C2 minimises the seed's relative
//                 error (5.1e-2) over the binades, and two steps take it to
//                 (5.1e-2)^4 = 6.5e-6.
//               Relative error of sigma below 1e-4 for every finite z: well
//               under the 2^-9 of the BF16 value the epilogue stores.
#pragma once
#include <cstdint>

namespace compton {
namespace act {

__device__ __forceinline__ uint64_t pk2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float fma_sat(float a, float b, float c)
{
    float d;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU of the pair z = 2 h, given h (tanh on the multi-function unit).
__device__ __forceinline__ uint64_t silu2_mufu(uint64_t h)
{
    float h0, h1;
    upk2(h, h0, h1);
    return fma2(h, pk2(tanh_hw(h0), tanh_hw(h1)), h);
}

// Degree-3 minimax (relative error) polynomial of 2^f on [-1/2, 1/2].
constexpr float kExp2C0 = 0.99992805719375610f;
constexpr float kExp2C1 = 0.69326096773147583f;
constexpr float kExp2C2 = 0.24261112511157990f;
constexpr float kExp2C3 = 0.05517166852951050f;
constexpr uint32_t kRcpSeed = 0x7EF311C2u;

// SiLU of the pair z = 2 h, given h, on the FMA pipe (no multi-function-unit
// instruction).
__device__ __forceinline__ uint64_t silu2_fma(uint64_t h)
{
    // t = sat(1/2 - h 2 log2(e) / 252) in [0, 1], y = 252 t - 126 = -z log2(e) clamped
    constexpr float kL = 2.0f * 1.4426950408889634f / 252.0f;
    float h0, h1;
    upk2(h, h0, h1);
    const uint64_t t = pk2(fma_sat(h0, -kL, 0.5f), fma_sat(h1, -kL, 0.5f));
    const uint64_t y = fma2(t, pk2(252.0f, 252.0f), pk2(-126.0f, -126.0f));
    const uint64_t sh = pk2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: adding it rounds to an integer
    const uint64_t jm = add2(y, sh);                     // low mantissa bits hold rint(y)
    const uint64_t j = add2(jm, pk2(-12582912.0f, -12582912.0f));
    const uint64_t f = fma2(j, pk2(-1.0f, -1.0f), y);  // y - j, exact
    uint64_t p = fma2(pk2(kExp2C3, kExp2C3), f, pk2(kExp2C2, kExp2C2));
    p = fma2(p, f, pk2(kExp2C1, kExp2C1));
    p = fma2(p, f, pk2(kExp2C0, kExp2C0));
    // E = p 2^j: j added to the exponent field of p (bits 0..8 of jm's
    // pattern hold j mod 2^9, so jm's pattern times 2^23 is j << 23 mod 2^32)
    const uint32_t e0 = (uint32_t)jm * 8388608u + (uint32_t)p;
    const uint32_t e1 = (uint32_t)(jm >> 32) * 8388608u + (uint32_t)(p >> 32);
    const uint64_t E = ((uint64_t)e1 << 32) | e0;
    // -d = -(1 + E) / 2 in [-2^125, -1/2]; the seed K - bits(d) is
    // (K + 2^31) - bits(-d) mod 2^32
    const uint64_t nd = fma2(E, pk2(-0.5f, -0.5f), pk2(-0.5f, -0.5f));
    const uint32_t r0 = (kRcpSeed ^ 0x80000000u) - (uint32_t)nd;
    const uint32_t r1 = (kRcpSeed ^ 0x80000000u) - (uint32_t)(nd >> 32);
    uint64_t r = ((uint64_t)r1 << 32) | r0;
    const uint64_t one = pk2(1.0f, 1.0f);
    uint64_t e = fma2(nd, r, one);  // 1 - d r
    r = fma2(r, e, r);
    e = fma2(nd, r, one);
    r = fma2(r, e, r);
    return mul2(h, r);  // h / d = z sigma(z)
}

}  // namespace act
}  // namespace compton
