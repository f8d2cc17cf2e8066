// polar_common.cuh -- shared device-side definitions of the GB300 polar decoder.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "polar_gb300.h"

namespace polar {

constexpr int kMaxN = POLAR_MAX_N;
constexpr int kMaxWords = kMaxN / 32;

// Per-code tables derived on the host from (N, K, frozen, CRC) and kept in a static device
// array, one slot per distinct code.
struct DevCode {
    int32_t N, n, K, P, c;
    uint32_t poly;
    uint32_t frozen_bits[kMaxWords];  // bit i of word i/32 set = node i frozen
    uint32_t decided_bits[kMaxWords]; // information positions CA-SCL decides without branching
    // Syndrome column of node i: x^(K-1-k) mod g(x) for the node's information index k, 0 for a
    // frozen node.  The XOR of the columns of the information nodes decided 1 is the remainder of
    // the decided K-bit word divided by g(x): zero iff the CRC holds.
    uint32_t colsyn[kMaxN];
    int16_t paypos[kMaxN];    // payload position of node i, -1 for frozen and CRC nodes
    int16_t info_idx[kMaxN];  // node of information index k (k < K)
};

// ---------------------------------------------------------------------------- FP32 primitives
// min-sum PE function g(a, b) = sign(a) sign(b) min(|a|, |b|) as one instruction: the magnitude
// is min(|a|, |b|), the sign bit the XOR of the operands' sign bits.
__device__ __forceinline__ float xmin(float a, float b)
{
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Clip to [-m, m] for m > 0, also as one instruction: sign(x) xor sign(m) = sign(x).
__device__ __forceinline__ float clipm(float x, float m) { return xmin(x, m); }

// Staging clip of a channel LLR: NaN reads as 0 (an erasure), then [-m, m].
__device__ __forceinline__ float stage_clip(float v, float m)
{
    v = (v == v) ? v : 0.0f;
    return fminf(fmaxf(v, -m), m);
}

// Channel LLR as CA-SCL reads it: NaN is an erasure (0); magnitudes beyond 2^100, +-inf included,
// saturate at 2^100, above any LLR a channel gives and small enough that no sum of the SC
// recursion (at most N channel values) or of a path metric (at most N such sums) overflows.
__device__ __forceinline__ float scl_stage(float v) { return stage_clip(v, 0x1p100f); }

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

// Base-2 exponential and logarithm of the special-function unit (approximate, subnormals flushed).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact PE function g(a, b) = ln((1 + e^(a+b)) / (e^a + e^b)) (Sec. II-B), in the form
//   sign(a) sign(b) min(|a|, |b|) + ln(p / q),  p = 1 + 2^-|s|,  q = 1 + 2^-|d|,
//   s = (a + b) log2 e, d = (a - b) log2 e
// (the same function: the LLR of the XOR of two independent bits), whose exponentials never
// overflow.  Working in base 2 lets the special-function unit's ex2 / lg2 take the arguments as
// they are (s, d from one multiply and two fused multiply-adds, the ln 2 folded into the final
// fused add).  The quotient costs one logarithm instead of the two of ln p - ln q: 1/q (q in
// [1, 2]) comes from Newton-Raphson on the FMA pipe, started from the minimax quadratic
// 70/33 - 16/11 q + 32/99 q^2 (relative error at most 1/99 on [1, 2]) and refined twice by
// r <- r + r (1 - q r), which squares the relative error each time (1e-4, then ~1e-8).  So the
// special-function unit does three operations per g: two ex2 (full rate) and one lg2 (half
// rate).  The approximate ex2 / lg2 leave an absolute error of a few 1e-7 on the clipped
// magnitudes, so results agree with the exact value to a tolerance, not to the bit.
__device__ __forceinline__ float g_exact(float a, float b)
{
    const float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float ta = __fmul_rn(a, kLog2e);
    const float s = __fmaf_rn(b, kLog2e, ta), d = __fmaf_rn(b, -kLog2e, ta);
    const float p = fadd(1.0f, ex2_approx(-fabsf(s)));
    const float nq = __fmaf_rn(ex2_approx(-fabsf(d)), -1.0f, -1.0f);  // -q
    float r = __fmaf_rn(__fmaf_rn(32.0f / 99.0f, nq, 16.0f / 11.0f), nq, 70.0f / 33.0f);
    r = __fmaf_rn(r, __fmaf_rn(nq, r, 1.0f), r);
    r = __fmaf_rn(r, __fmaf_rn(nq, r, 1.0f), r);
    return __fmaf_rn(kLn2, lg2_approx(__fmul_rn(p, r)), xmin(a, b));
}

// Two exact PE functions at once, bit for bit the arithmetic of g_exact on each lane: everything
// but the special-function operations and the final min runs as packed FP32 (fma / add / mul
// .f32x2, one instruction for both lanes).  Both forms work on nq = -q so that no packed operand
// needs a negation: the seed becomes 70/33 + 16/11 nq + 32/99 nq^2 and 1 - q r = nq r + 1.
__device__ __forceinline__ float2 g_exact2(float2 a, float2 b)
{
    const float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float2 one = make_float2(1.0f, 1.0f), mone = make_float2(-1.0f, -1.0f);
    const float2 ta = __fmul2_rn(a, make_float2(kLog2e, kLog2e));
    const float2 s = __ffma2_rn(b, make_float2(kLog2e, kLog2e), ta);
    const float2 d = __ffma2_rn(b, make_float2(-kLog2e, -kLog2e), ta);
    const float2 xs = make_float2(ex2_approx(-fabsf(s.x)), ex2_approx(-fabsf(s.y)));
    const float2 xd = make_float2(ex2_approx(-fabsf(d.x)), ex2_approx(-fabsf(d.y)));
    const float2 p = __fadd2_rn(one, xs);
    const float2 nq = __ffma2_rn(xd, mone, mone);
    float2 r = __ffma2_rn(__ffma2_rn(make_float2(32.0f / 99.0f, 32.0f / 99.0f), nq,
                                     make_float2(16.0f / 11.0f, 16.0f / 11.0f)),
                          nq, make_float2(70.0f / 33.0f, 70.0f / 33.0f));
    r = __ffma2_rn(r, __ffma2_rn(nq, r, one), r);
    r = __ffma2_rn(r, __ffma2_rn(nq, r, one), r);
    const float2 pr = __fmul2_rn(p, r);
    return __ffma2_rn(make_float2(kLn2, kLn2), make_float2(lg2_approx(pr.x), lg2_approx(pr.y)),
                      make_float2(xmin(a.x, b.x), xmin(a.y, b.y)));
}

// ---------------------------------------------------------------------------- half2 primitives
__device__ __forceinline__ __half2 xmin(__half2 a, __half2 b)
{
    uint32_t d;
    asm("min.xorsign.abs.f16x2 %0, %1, %2;"
        : "=r"(d)
        : "r"(*reinterpret_cast<uint32_t*>(&a)), "r"(*reinterpret_cast<uint32_t*>(&b)));
    return *reinterpret_cast<__half2*>(&d);
}
__device__ __forceinline__ __half2 clipm(__half2 x, __half2 m) { return xmin(x, m); }
__device__ __forceinline__ __half2 fadd(__half2 a, __half2 b) { return __hadd2(a, b); }
__device__ __forceinline__ __half2 fmul(__half2 a, __half2 b) { return __hmul2(a, b); }

// ---------------------------------------------------------------------------- barriers
// Synchronise the T threads that decode one frame: the warp itself for T <= 32, otherwise the
// whole CTA (plans with T > 32 put one frame group in a CTA).
template <int T>
__device__ __forceinline__ void frame_sync(int slot)
{
    (void)slot;
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        __syncthreads();
    }
}

// compile-time loops: fn(integral_constant<int, i>) for i = I..E-1 (static_for) or I..E
// descending (static_for_down); the index is a constant expression inside fn
template <int I, int E, class Fn>
__device__ __forceinline__ void static_for(Fn&& fn)
{
    if constexpr (I < E) {
        fn(std::integral_constant<int, I>{});
        static_for<I + 1, E>(fn);
    }
}

template <int I, int E, class Fn>
__device__ __forceinline__ void static_for_down(Fn&& fn)
{
    if constexpr (I >= E) {
        fn(std::integral_constant<int, I>{});
        static_for_down<I - 1, E>(fn);
    }
}

__device__ __forceinline__ int frozen_at(const uint32_t* fb, int i) { return (fb[i >> 5] >> (i & 31)) & 1; }

}  // namespace polar
