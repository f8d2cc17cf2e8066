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
//   sign(a) sign(b) min(|a|, |b|) + ln 2 [log2(1 + 2^-|s|) - log2(1 + 2^-|d|)],
//   s = (a + b) log2 e, d = (a - b) log2 e
// (the same function: the LLR of the XOR of two independent bits), whose exponentials never
// overflow.  Working in base 2 lets the special-function unit's ex2 / lg2 take the arguments as
// they are (s, d from one multiply and two fused multiply-adds, the ln 2 folded into the final
// fused add).  The approximate ex2 / lg2 leave an absolute error of a few 1e-7 on the clipped
// magnitudes, so results agree with the exact value to a tolerance, not to the bit.
__device__ __forceinline__ float g_exact(float a, float b)
{
    const float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float tb = __fmul_rn(b, kLog2e);
    const float s = __fmaf_rn(a, kLog2e, tb), d = __fmaf_rn(a, kLog2e, -tb);
    const float ls = lg2_approx(fadd(1.0f, ex2_approx(-fabsf(s))));
    const float ld = lg2_approx(fadd(1.0f, ex2_approx(-fabsf(d))));
    return __fmaf_rn(kLn2, __fsub_rn(ls, ld), xmin(a, b));
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
