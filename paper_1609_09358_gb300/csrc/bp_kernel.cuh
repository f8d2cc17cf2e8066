// bp_kernel.cuh -- min-sum belief propagation with CRC early stop (Sec. II-B of the paper),
// register-blocked for sm_103a.
//
// Graph (Fig. 1, PE of Fig. 2): columns s = 1..n+1 (u side .. channel side); the PE of stage s
// joins nodes j and j + 2^(s-1) (bit s-1 of j clear).  One iteration runs the R sweep over
// stages 1..n and then the L sweep over stages n..1:
//   R sweep:  R[s+1][j]   = g(R[s][j], L[s+1][j+d] + R[s][j+d])
//             R[s+1][j+d] = g(R[s][j], L[s+1][j])   + R[s][j+d]
//   L sweep:  L[s][j]     = g(L[s+1][j], L[s+1][j+d] + R[s][j+d])
//             L[s][j+d]   = g(R[s][j], L[s+1][j])   + L[s+1][j+d]
// every result clipped to [-M, M]; g is min-sum.  After the L sweep the hard decision of
// L[1][i] + R[1][i] is CRC-checked and the frame stops when the syndrome is zero.
//
// Execution plan (own design, not the paper's one-thread-per-PE layout): a frame is decoded by
// T = N / 2^b threads, each owning 2^b nodes of every column.  The n index bits are cut into
// groups of b consecutive bits; while the sweep is inside group g, a thread's 2^b nodes differ
// exactly in the bits of g's window, so b consecutive PE stages run entirely in registers.  At
// a group boundary the boundary column is exchanged once through a swizzled shared-memory
// buffer (bank-conflict free for every access of every plan, checked at compile time).  All
// messages stay in registers for the frame's whole life (most kernels from N = 1024 on keep the
// channel column, read at two stages per iteration, in shared memory instead: CHS below); HBM is
// touched once to read the channel LLRs and once to write the decided payload bits.
//
// Storage of column c: R[c] lives in the mapping of stage c (the group that reads it), L[c] in
// the mapping of stage c-1.  The clip of g(R[s][j], .) and g(L[s+1][j], .) is skipped when no
// learned weight scales it: |g(a, b)| <= |a| <= M already.
#pragma once

#include <cstring>
#include <type_traits>
#include <utility>

#include "polar_common.cuh"

namespace polar {

template <int LOGN_, int LOGR_>
struct BPPlan {
    static constexpr int LOGN = LOGN_, LOGR = LOGR_;
    static constexpr int N = 1 << LOGN, R = 1 << LOGR, T = N >> LOGR;
    static constexpr int NG = (LOGN + LOGR - 1) / LOGR;
    static constexpr int NW = (T + 31) / 32;
    static constexpr int TB = LOGN - LOGR;  // thread-index bits
    // group of the PE stage with index bit q (stage s = q + 1)
    __host__ __device__ static constexpr int grp(int q) { return q / LOGR; }
    // first index bit of group g's register window (the last window is pulled down to fit)
    __host__ __device__ static constexpr int win(int g) { return (g + 1) * LOGR <= LOGN ? g * LOGR : LOGN - LOGR; }

    // Exchange-buffer addressing.  PAD plans use addr(j) = j + (j >> 5) + (j >> 10): it is
    // additive over disjoint bit sets, so the R accesses of a thread are one per-thread base plus
    // compile-time offsets (no address arithmetic per access), and it is bank-conflict free when
    // in every group the 5 lane bits of the thread index land on node bits whose addresses are
    // 1, 2, 4, 8, 16 modulo 32 in some order -- for group 1 that takes node bits 0, 1, 2, 8, 9
    // with b = 3, and 0, 1, 2, 3, 9 with b = 4 (a search over the plans finds such bits for
    // N >= 1024 with b = 3 and b = 4 only).  The other plans
    // keep an XOR swizzle of index bits 5..7 into the bank bits (one XOR per access).
    static constexpr bool PAD = (LOGR == 3 && LOGN >= 10) || (LOGR == 4 && LOGN >= 10);
    // node bit receiving thread-index bit q in group g: the non-window bits in ascending order,
    // except that group 1 of a PAD plan puts lane bits 3, 4 on node bits 8, 9 (b = 3) or lane
    // bit 4 on node bit 9 (b = 4)
    __host__ __device__ static constexpr int tbit(int g, int q)
    {
        if (PAD && LOGR == 3 && g == 1)  // window 3..5: thread bits -> node bits 0 1 2 8 9 6 7 10 ...
            return q < 3 ? q : q < 5 ? q + 5 : q < 7 ? q + 1 : q + 3;
        if (PAD && LOGR == 4 && g == 1)  // window 4..7: thread bits -> node bits 0 1 2 3 9 8 10 11
            return q < 4 ? q : q == 4 ? 9 : q == 5 ? 8 : q + 4;
        return q < win(g) ? q : q + LOGR;
    }
    // node bits from the thread index t (group g) and from the register index k
    __host__ __device__ static constexpr int tpart(int g, int t)
    {
        int v = 0;
        for (int q = 0; q < TB; ++q) v |= ((t >> q) & 1) << tbit(g, q);
        return v;
    }
    __host__ __device__ static constexpr int kpart(int g, int k) { return k << win(g); }
    // node held in register k by thread t while in group g
    __host__ __device__ static constexpr int node(int g, int t, int k) { return tpart(g, t) | kpart(g, k); }
    // column exchanges: the R sweep leaving stage s crosses into another group, or the L sweep
    // leaving stage s does; xidx numbers the exchanges of one iteration in execution order
    __host__ __device__ static constexpr bool rcross(int s) { return s < LOGN && grp(s) != grp(s - 1); }
    __host__ __device__ static constexpr bool lcross(int s) { return s > 1 && grp(s - 2) != grp(s - 1); }
    __host__ __device__ static constexpr int xidx_r(int s)
    {
        int c = 0;
        for (int i = 1; i < s; ++i) c += rcross(i);
        return c;
    }
    __host__ __device__ static constexpr int xidx_l(int s)
    {
        int c = xidx_r(LOGN + 1);
        for (int i = LOGN; i > s; --i) c += lcross(i);
        return c;
    }
    // XOR swizzle of the non-PAD plans: index bits 5..7 into the bank bits
    __host__ __device__ static constexpr int swz(int j)
    {
        if constexpr (LOGR == 3)
            return j ^ (((j >> 5) & 1) * 1) ^ (((j >> 6) & 1) * 10) ^ (((j >> 7) & 1) * 20);
        else
            return j ^ (((j >> 5) & 1) * 5) ^ (((j >> 6) & 1) * 26);
    }
    __host__ __device__ static constexpr int addr(int j) { return PAD ? j + (j >> 5) + (j >> 10) : swz(j); }
    // words of one exchange buffer
    static constexpr int XW = PAD ? ((N + (N >> 5) + (N >> 10)) + 3) & ~3 : N;
};

// Compile-time checks of a plan, one group at a time (each its own constant expression, so the
// checks of long codes stay within the compiler's evaluation budget).
template <class P, int G>
constexpr bool plan_group_bijective()
{
    // group G maps (thread, register) onto the N nodes one to one
    uint32_t seen[P::N / 32] = {};
    for (int t = 0; t < P::T; ++t)
        for (int k = 0; k < P::R; ++k) {
            const int j = P::node(G, t, k);
            if (j < 0 || j >= P::N || ((seen[j >> 5] >> (j & 31)) & 1u)) return false;
            seen[j >> 5] |= 1u << (j & 31);
        }
    return true;
}
template <class P, int G, int K>
constexpr bool plan_group_banks()
{
    // register K of the 32 threads of every warp: distinct banks; PAD plans: the address splits
    // into the thread's base and the register's offset
    for (int w = 0; w < P::NW; ++w) {
        uint32_t banks = 0;
        for (int l = 0; l < 32 && w * 32 + l < P::T; ++l) {
            const int t = w * 32 + l;
            const int a = P::addr(P::node(G, t, K));
            if (a < 0 || a >= P::XW) return false;
            if (P::PAD && a != P::addr(P::tpart(G, t)) + P::addr(P::kpart(G, K))) return false;
            const uint32_t bit = 1u << (a & 31);
            if (banks & bit) return false;
            banks |= bit;
        }
    }
    return true;
}
template <class P, int G, int K>
struct PlanBankCheck {
    static_assert(plan_group_banks<P, G, K>(), "exchange layout has bank conflicts");
    static constexpr bool ok = true;
};
template <class P, int G, class KS>
struct PlanGroupCheck;
template <class P, int G, int... K>
struct PlanGroupCheck<P, G, std::integer_sequence<int, K...>> {
    static_assert(plan_group_bijective<P, G>(), "exchange layout: a group does not cover the nodes once");
    static constexpr bool ok = (PlanBankCheck<P, G, K>::ok && ...);
};
template <class P, class GS>
struct PlanCheck;
template <class P, int... G>
struct PlanCheck<P, std::integer_sequence<int, G...>> {
    static constexpr bool ok = (PlanGroupCheck<P, G, std::make_integer_sequence<int, P::R>>::ok && ...);
};
template <class P>
constexpr bool plan_is_conflict_free()
{
    return PlanCheck<P, std::make_integer_sequence<int, P::NG>>::ok;
}

// Exchange-buffer access of register k of thread t in group G: the thread's base of group G
// (xbase[G] = addr(tpart(G, t)), computed once) plus a compile-time offset for PAD plans, the
// XOR-swizzled node index otherwise.
template <class P, int G, class MSG>
__device__ __forceinline__ void xput(MSG* xb, const int* xbase, int t, int k, MSG v)
{
    if constexpr (P::PAD)
        xb[xbase[G] + P::addr(P::kpart(G, k))] = v;
    else
        xb[P::swz(P::node(G, t, k))] = v;
}
template <class P, int G, class MSG>
__device__ __forceinline__ MSG xget(const MSG* xb, const int* xbase, int t, int k)
{
    if constexpr (P::PAD)
        return xb[xbase[G] + P::addr(P::kpart(G, k))];
    else
        return xb[P::swz(P::node(G, t, k))];
}

struct BPArgs {
    const float* llr;
    int B;
    int max_iters;
    float llr_max;
    const void* w;   // learned weights in the prepared layout (wms_prep_index) or null
    int w_iters;
    uint8_t* bits;
    uint8_t* status;
    uint16_t* iters;
    float* llr_u;
    float* llr_x;
    const DevCode* code;
    int* fail_count;  // hybrid: compaction of the CRC-failed frames (null for bp_decode)
    int* fail_list;
    int* fail_total;  // optional running total of CRC-failed frames
    int* next;        // work counter (zero before the launch): groups refill from it; null = one frame group per CTA slot
    const long long* llr_off;  // element offset of each frame's LLR row (null: frame * N)
    int row_bytes;
    int fixed_iters;           // run max_iters iterations regardless of the CRC
    int frame0;                // index of the launch's first frame (frames frame0 .. frame0 + B - 1)
};

// Message traits: FP32 (one frame per thread) or half2 (two frames per thread).
template <class MSG>
struct MsgTraits;
template <>
struct MsgTraits<float> {
    static constexpr int FPT = 1;
    __device__ static float splat(float v) { return v; }
    __device__ static float load2(const float* a, const float* b, int j, float m)
    {
        return stage_clip(__ldg(a + j), m);
    }
    __device__ static bool neg(float v, int h) { return v < 0.0f; }
    __device__ static float to_f(float v, int h) { return v; }
    __device__ static float set_half(float, float x, int) { return x; }
    __device__ static float zero_half(float, int) { return 0.0f; }
    __device__ static float pair(float a, float) { return a; }
};
template <>
struct MsgTraits<__half2> {
    static constexpr int FPT = 2;
    __device__ static __half2 splat(float v) { return __float2half2_rn(v); }
    __device__ static __half2 load2(const float* a, const float* b, int j, float m)
    {
        const float x = stage_clip(__ldg(a + j), m);
        const float y = b ? stage_clip(__ldg(b + j), m) : 0.0f;
        return __floats2half2_rn(x, y);
    }
    __device__ static bool neg(__half2 v, int h)
    {
        return __hlt(h ? __high2half(v) : __low2half(v), __float2half(0.0f));
    }
    __device__ static float to_f(__half2 v, int h) { return __half2float(h ? __high2half(v) : __low2half(v)); }
    __device__ static __half2 set_half(__half2 v, float x, int h)
    {
        const __half hx = __float2half_rn(x);
        return h ? __halves2half2(__low2half(v), hx) : __halves2half2(hx, __high2half(v));
    }
    __device__ static __half2 zero_half(__half2 v, int h)
    {
        const __half z = __float2half_rn(0.0f);
        return h ? __halves2half2(__low2half(v), z) : __halves2half2(z, __high2half(v));
    }
    __device__ static __half2 pair(float a, float b) { return __floats2half2_rn(a, b); }
};

// Barrier of one frame group: the warp (T <= 32), the whole CTA (the group owns its CTA), or a
// named barrier (several groups wider than a warp share the CTA; ids 1.. by slot).
template <int T, bool SHARED_CTA>
__device__ __forceinline__ void group_sync(int slot)
{
    if constexpr (T <= 32) {
        __syncwarp();
    } else if constexpr (!SHARED_CTA) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(slot + 1), "r"(T) : "memory");
    }
}

// Frame source of the per-length kernel: the group's own frames (no counter) or a work counter.
struct CounterSource {
    int* next;
    int B;
    int first;  // first static frame of the group
    int FPT;
    int frame0;  // offset of the launch's frames
    int nfetch = 0;
    template <int T, bool SHARED_CTA>
    __device__ int fetch(int slot, int t, int* cell)
    {
        int f;
        if (next) {
            if (t == 0) cell[0] = atomicAdd(next, 1);
            group_sync<T, SHARED_CTA>(slot);
            f = cell[0];
            group_sync<T, SHARED_CTA>(slot);
        } else {
            f = nfetch < FPT ? first + nfetch : B;
        }
        ++nfetch;
        return f < B ? frame0 + f : -1;
    }
};

// Frame source of the mixed-length kernel: a queue of frame indices of one code.
struct QueueSource {
    const int* list;
    int count;
    int* next;
    template <int T, bool SHARED_CTA>
    __device__ int fetch(int slot, int t, int* cell)
    {
        if (t == 0) {
            const int k = atomicAdd(next, 1);
            cell[0] = k < count ? list[k] : -1;
        }
        group_sync<T, SHARED_CTA>(slot);
        const int f = cell[0];
        group_sync<T, SHARED_CTA>(slot);
        return f;
    }
};

// Learned scales in the kernel's register layout ("prepared" weights).  Element (it, dir, s, t, k)
// is the scale of the g term written to node P::node(P::grp(s-1), t, k) at stage s of sweep dir
// (0: R, 1: L) in iteration it, stored [it][dir][s-1][t][k]: a thread reads the R scales of one
// stage as one or two 16-byte vectors, and a warp reads contiguous memory.  Element type: float
// for FP32 messages, binary16 (rounded to nearest even once) for half2 messages.
template <class P>
__host__ __device__ constexpr size_t wms_prep_index(int it, int dir, int s, int t, int k)
{
    return ((((size_t)it * 2 + dir) * P::LOGN + (s - 1)) * P::T + t) * P::R + k;
}

template <class E>
__device__ __forceinline__ E wms_elem(float v);
template <>
__device__ __forceinline__ float wms_elem<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half wms_elem<__half>(float v) { return __float2half_rn(v); }

// Natural layout w[it][dir][s-1][node] -> prepared layout; one thread per element.
template <class P, class E>
__global__ void wms_prepare_kernel(const float* __restrict__ w, int iters, E* __restrict__ out)
{
    const size_t total = (size_t)iters * 2 * P::LOGN * P::N;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int k = (int)(e % P::R);
    const int t = (int)((e / P::R) % P::T);
    const size_t row = e / P::N;                  // (it * 2 + dir) * n + (s - 1)
    const int s1 = (int)(row % P::LOGN);
    out[e] = wms_elem<E>(__ldg(w + row * P::N + P::node(P::grp(s1), t, k)));
}

// One thread's R prepared scales of one stage.
template <class E, int R>
struct WRow {
    E v[R];
};

template <class E, int R>
__device__ __forceinline__ WRow<E, R> wms_row(const E* p)
{
    constexpr int BYTES = R * (int)sizeof(E);
    static_assert(BYTES == 8 || BYTES % 16 == 0, "prepared row size");
    WRow<E, R> r;
    if constexpr (BYTES == 8) {
        const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
        memcpy(r.v, &x, 8);
    } else {
#pragma unroll
        for (int q = 0; q < BYTES / 16; ++q) {
            const uint4 x = __ldg(reinterpret_cast<const uint4*>(p) + q);
            memcpy(reinterpret_cast<char*>(r.v) + 16 * q, &x, 16);
        }
    }
    return r;
}

template <class E, int R>
__device__ __forceinline__ WRow<E, R> wms_ones()
{
    WRow<E, R> r;
#pragma unroll
    for (int k = 0; k < R; ++k) r.v[k] = wms_elem<E>(1.0f);
    return r;
}

template <int LOGN>
struct BPConfig;  // thread plan and frames (or frame pairs) per CTA for each block length
// MIN_CTAS / MIN_CTAS_W / MIN_CTAS_U: resident CTAs per SM the register allocation of the plain /
// weighted / unit-scale weighted kernel must allow (launch bounds).  The unit-scale kernel at
// N = 2048 takes 2 CTAs (128 registers, 68 bytes of spill): 15% faster than 1 CTA at 171
// registers; at N = 1024 4 CTAs measured no faster than 3.
template <> struct BPConfig<7>  { using Plan = BPPlan<7, 2>;  static constexpr int F = 4, MIN_CTAS = 4, MIN_CTAS_W = 4, MIN_CTAS_U = 4; };
template <> struct BPConfig<8>  { using Plan = BPPlan<8, 3>;  static constexpr int F = 4, MIN_CTAS = 4, MIN_CTAS_W = 3, MIN_CTAS_U = 3; };
template <> struct BPConfig<9>  { using Plan = BPPlan<9, 3>;  static constexpr int F = 1, MIN_CTAS = 8, MIN_CTAS_W = 5, MIN_CTAS_U = 5; };
template <> struct BPConfig<10> { using Plan = BPPlan<10, 3>; static constexpr int F = 1, MIN_CTAS = 4, MIN_CTAS_W = 3, MIN_CTAS_U = 3; };
template <> struct BPConfig<11> { using Plan = BPPlan<11, 3>; static constexpr int F = 1, MIN_CTAS = 2, MIN_CTAS_W = 1, MIN_CTAS_U = 2; };
// N = 4096: one frame group of 512 threads per SM; the live messages of a thread (about n + 1
// columns of 8 nodes: the R columns the coming L sweep reads and the L columns the coming R sweep
// reads) fit its 128 registers, so the frame stays on one SM without a cluster
template <> struct BPConfig<12> { using Plan = BPPlan<12, 3>; static constexpr int F = 1, MIN_CTAS = 1, MIN_CTAS_W = 1, MIN_CTAS_U = 1; };

// first R-sweep stage whose outputs cross into another group (0: none)
template <class P>
__host__ __device__ constexpr int first_rcross()
{
    for (int s = 1; s <= P::LOGN; ++s)
        if (P::rcross(s)) return s;
    return 0;
}

// Plan and frame groups per CTA of a kernel (FPT: frames per thread, 2 for half2): the plain
// min-sum kernels at N = 1024 and the plain FP32 one at N = 4096 take 16 nodes per thread (64 / 256
// threads per frame, 4 column exchanges per iteration instead of 6), the others the length's plan
// (at N = 4096 the exact-g kernel measured 11% slower with 16, the half2 one 3-9% slower).
template <int LOGN, int WEIGHTED, int VAR, int FPT>
struct BPKernelPlan {
    using Plan = typename BPConfig<LOGN>::Plan;
    static constexpr int F = BPConfig<LOGN>::F;
};
template <int FPT>
struct BPKernelPlan<10, 0, 0, FPT> {
    using Plan = BPPlan<10, 4>;
    static constexpr int F = 1;
};
template <>
struct BPKernelPlan<12, 0, 0, 1> {
    using Plan = BPPlan<12, 4>;
    static constexpr int F = 1;
};

template <class P>
__host__ __device__ constexpr int bp_slot_words()
{
    // exchange buffers [2][XW] | syndrome columns, thread-major [R][T] | partial syndromes
    // [2][2][NW] | packed payload bits [2][N/32] | fetched frame index [4] | from N = 1024 on the
    // channel column [XW], in the last group's exchange layout
    return 2 * P::XW + P::N + 4 * P::NW + 2 * (P::N / 32) + 4 + (P::LOGN >= 10 ? P::XW : 0);
}

// One frame group of T threads decoding frames from `src` until it runs dry.  Group `slot` of
// the CTA uses the shared-memory slice `slot_smem` (bp_slot_words<P>() words).
// SYNP (CRCs of at most 16 bits): half2 keeps both frames' CRC syndromes in one word; FP32 with
// the PE pairs keeps the syndrome columns of two adjacent nodes in one word.
// VAR (FP32, unweighted): bit 0 the exact PE function instead of min-sum, bit 1 the re-encoding
// stop -- the frame stops at the first iteration where HD(LLR(x)) equals the re-encoded HD(LLR(u))
// (x = u G, Sec. II-B) and counts as decoded iff its CRC then holds.
template <int R>
__host__ __device__ constexpr uint32_t pe_low_mask(int dd)
{
    uint32_t m = 0;
    for (int k = 0; k < R; ++k)
        if (!(k & dd)) m |= 1u << k;
    return m;
}

// register index of the i-th PE of a stage whose partner registers are dd apart: i with a zero
// bit inserted at dd's position
__host__ __device__ constexpr int pe_k(int dd, int i) { return ((i & ~(dd - 1)) << 1) | (i & (dd - 1)); }

// WEIGHTED: 0 plain min-sum; 1 learned scales; 2 learned scales within [-1, 1] (|w g| <= |g| <= M,
// so the scaled term needs no clip) and, for half2, both frames of a register kept on the same
// iteration (a frame that stops waits for its partner; the pair refills together), so that one
// binary16 scale, duplicated in the register, scales both -- used when every iteration is a
// learned one.  (Scales stored as ready (w, w) pairs instead measured slower: twice the bytes
// read from L2 per frame pair and iteration, which is what bounds the weighted kernel.)
template <class P, class MSG, int WEIGHTED, bool SHARED_CTA, class Src, bool SYNP = false, int VAR = 0>
__device__ __forceinline__ void bp_run_group(const BPArgs& a, const DevCode& C, int slot, int t, uint32_t* slot_smem,
                                             Src& src)
{
    using MT = MsgTraits<MSG>;
    constexpr int N = P::N, R = P::R, T = P::T, NG = P::NG, NW = P::NW, n = P::LOGN;
    constexpr int FPT = MT::FPT;
    static_assert(plan_is_conflict_free<P>(), "exchange layout has bank conflicts");
    // exchanges alternate between the two buffers; an even count per iteration keeps the
    // alternation across iterations, so a buffer is rewritten only after a barrier that follows
    // every read of its previous contents
    static_assert(P::xidx_l(0) % 2 == 0, "odd number of exchanges per iteration");
    constexpr bool EXACT = (VAR & 1) != 0, REENC = (VAR & 2) != 0;
    constexpr bool UNIT = WEIGHTED == 2, ALIGNED = UNIT && FPT == 2;
    static_assert(VAR == 0 || (FPT == 1 && !WEIGHTED), "exact g and the re-encoding stop: FP32, unweighted");
    static_assert(!REENC || (T % 32 == 0 && (!SHARED_CTA || T == 32)), "re-encoding vote: whole warps, own barrier");
    // PE function: min-sum (one instruction) or exact; the exact value is clipped like every
    // message, since its fast logarithms may overshoot min(|a|, |b|) by an ulp
    auto gf = [&](MSG x, MSG y) -> MSG {
        if constexpr (EXACT)
            return clipm(g_exact(x, y), MT::splat(a.llr_max));
        else
            return xmin(x, y);
    };
    // both PE functions of a node pair; the exact form evaluates the two as one packed pair
    auto gf2 = [&](MSG x1, MSG y1, MSG x2, MSG y2, MSG& o1, MSG& o2) {
        if constexpr (EXACT) {
            const float2 g = g_exact2(make_float2(x1, x2), make_float2(y1, y2));
            o1 = clipm(g.x, a.llr_max);
            o2 = clipm(g.y, a.llr_max);
        } else {
            o1 = gf(x1, y1);
            o2 = gf(x2, y2);
        }
    };

    // FP32 without learned weights: the PEs of a stage are processed two at a time, so that each
    // of the two additions of a PE pair runs as one packed instruction (add.rn.f32x2, rounded
    // like the scalar add: the results are the same bits); the comparisons stay scalar.  Not for
    // the re-encoding stop, whose kernels spill more with the pairs and measured slower.
    constexpr bool PAIRS = FPT == 1 && !WEIGHTED && !REENC;
    // g of two PEs: o = (g(x.x, y.x), g(x.y, y.y))
    auto gpair = [&](float2 x, float2 y) -> float2 {
        if constexpr (EXACT) {
            const float2 g = g_exact2(x, y);
            return make_float2(clipm(g.x, a.llr_max), clipm(g.y, a.llr_max));
        } else {
            return make_float2(xmin(x.x, y.x), xmin(x.y, y.y));
        }
    };

    MSG* xbuf = reinterpret_cast<MSG*>(slot_smem);         // [2][XW]
    uint32_t* csyn = slot_smem + 2 * P::XW;                // [R][T]
    int xbase[NG];                                         // exchange base of each group (PAD plans)
    static_for<0, NG>([&](auto G) { xbase[G.value] = P::addr(P::tpart(G.value, t)); });
    uint32_t* synp = csyn + N;                             // [2 parity][2 frame][NW]
    uint32_t* pbits = synp + 4 * NW;                       // [2 frame][N/32]
    int* fetched = reinterpret_cast<int*>(pbits + 2 * (N / 32));
    // CHS (N >= 1024): the channel column lives in shared memory and is read into registers at the
    // two stages that use it (stage n of each sweep) and by the outputs, so that its R registers
    // are free for the rest of the iteration (the long kernels run at the register file's limit;
    // measured: N = 4096 exact g 7% faster, half2 9%, N = 2048 learned 5%, N = 1024 FP32 1.6%).
    // Each thread reads back only the nodes it wrote: no barrier.  Not for the plain and the
    // aligned-pair half2 kernels at N = 1024 (3.4% and 0.2% slower with it).
    constexpr bool CHS = n >= 11 || (n == 10 && (FPT == 1 || WEIGHTED == 1));
    MSG* chs = reinterpret_cast<MSG*>(fetched + 4);

    // Frames of this group: half h (h < FPT) decodes frame fr[h]; when it stops it fetches the
    // next frame from the source.
    auto fetch = [&]() -> int { return src.template fetch<T, SHARED_CTA>(slot, t, fetched); };
    auto row = [&](int f) -> const float* { return a.llr + (a.llr_off ? a.llr_off[f] : (long long)f * N); };
    int fr[2] = {-1, -1}, itc[2] = {0, 0};
    fr[0] = fetch();
    if constexpr (FPT == 2) fr[1] = fetch();
    if (fr[0] < 0 && fr[1] < 0) return;  // uniform over the group
    const float M = a.llr_max;
    const MSG Mv = MT::splat(M);

    MSG Lc[n + 2][R];
    MSG Rc[n + 2][R];
    auto chan_reload = [&]() {
        if constexpr (CHS) {
#pragma unroll
            for (int k = 0; k < R; ++k) Lc[n + 1][k] = xget<P, NG - 1>(chs, xbase, t, k);
        }
    };
    // SYNP, half2: both frames' syndromes share one word (frame 0 in the low half, frame 1 in the
    // high half), the columns are stored doubled.  SYNP, FP32 pairs: registers k and k + 1 share
    // one column word (k's column low, k + 1's high), two such words per thread and uint2,
    // [R/4][T]; the accumulated word's halves XOR to the syndrome.
    static_assert(!SYNP || FPT == 2 || (PAIRS && R % 4 == 0), "packed syndromes: half2, or FP32 pairs");
    constexpr bool syn_packed = SYNP;
    constexpr bool syn_nodes = SYNP && FPT == 1;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int j = P::node(0, t, k);
        const uint32_t col = C.colsyn[j];
        if constexpr (syn_nodes) {
            if (!(k & 1))
                csyn[(k >> 2) * 2 * T + 2 * t + ((k >> 1) & 1)] = col | (C.colsyn[P::node(0, t, k + 1)] << 16);
        } else {
            csyn[k * T + t] = syn_packed ? (col | (col << 16)) : col;
        }
        Rc[1][k] = frozen_at(C.frozen_bits, j) ? Mv : MT::splat(0.0f);
    }
    {
        const float* y0 = fr[0] >= 0 ? row(fr[0]) : nullptr;
        const float* y1 = fr[1] >= 0 ? row(fr[1]) : nullptr;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int j = P::node(NG - 1, t, k);
            const MSG v = MT::pair(y0 ? stage_clip(__ldg(y0 + j), M) : 0.0f, y1 ? stage_clip(__ldg(y1 + j), M) : 0.0f);
            if constexpr (CHS)
                xput<P, NG - 1>(chs, xbase, t, k, v);
            else
                Lc[n + 1][k] = v;
        }
    }
    // messages start at 0; only the L columns 2..n need it, since every R sweep writes R[2..n]
    // before anything reads them.  The half2 kernels zero the R columns too: with it the compiler
    // places their spills so that N = 4096 runs 8% faster (measured), at no cost at N = 1024.
    constexpr bool ZERO_R = FPT == 2;
#pragma unroll
    for (int c = 2; c <= n; ++c)
#pragma unroll
        for (int k = 0; k < R; ++k) {
            Lc[c][k] = MT::splat(0.0f);
            if constexpr (ZERO_R) Rc[c][k] = MT::splat(0.0f);
        }

    // Learned scales: iteration `it` of half h reads its prepared rows; past the learned
    // iterations (and for an idle half) the scale is 1, the same value as the plain update since
    // 1 * g = g and |g| <= M needs no clip.
    using WE = std::conditional_t<FPT == 2, __half, float>;
    using Row = WRow<WE, R>;
    const WE* wp = static_cast<const WE*>(a.w);
    struct WPair {
        Row h[FPT];
    };
    // ALIGNED: one row of scales for both halves, at the pair's iteration itp
    int itp = 0;
    using WSet = std::conditional_t<ALIGNED, Row, WPair>;
    auto wload = [&](int dir, int s) -> WSet {
        WSet r;
        if constexpr (ALIGNED) {
            r = itp < a.w_iters ? wms_row<WE, R>(wp + wms_prep_index<P>(itp, dir, s, t, 0)) : wms_ones<WE, R>();
        } else {
#pragma unroll
            for (int h = 0; h < FPT; ++h)
                r.h[h] = (fr[h] >= 0 && itc[h] < a.w_iters) ? wms_row<WE, R>(wp + wms_prep_index<P>(itc[h], dir, s, t, 0))
                                                            : wms_ones<WE, R>();
        }
        return r;
    };
    auto wk = [&](const WSet& r, int k) -> MSG {
        if constexpr (ALIGNED)
            return __half2half2(r.v[k]);
        else if constexpr (FPT == 2)
            return __halves2half2(r.h[0].v[k], r.h[1].v[k]);
        else
            return r.h[0].v[k];
    };
    // scalar scale (LLR(x) output of one half): iteration it, stage s, register k
    auto wscalar = [&](int it, int dir, int s, int k) -> float {
        if (it >= a.w_iters) return 1.0f;
        if constexpr (FPT == 2)
            return __half2float(wp[wms_prep_index<P>(it, dir, s, t, k)]);
        else
            return wp[wms_prep_index<P>(it, dir, s, t, k)];
    };

    // write the decided payload bits, status and optional LLRs of frame half h after `it_done`
    // iterations; called uniformly by the T threads of the frame group
    auto finalize = [&](int h, int it_done, bool ok) {
        const int frame = fr[h];
        uint32_t* pb = pbits + h * (N / 32);
        for (int i = t; i < N / 32; i += T) pb[i] = 0u;
        group_sync<T, SHARED_CTA>(slot);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int j = P::node(0, t, k);
            const int pos = C.paypos[j];
            if (pos >= 0 && MT::neg(fadd(Lc[1][k], Rc[1][k]), h)) atomicOr(&pb[pos >> 5], 1u << (pos & 31));
        }
        group_sync<T, SHARED_CTA>(slot);
        // the packed payload has ceil(P/8) <= N/8 bytes; a wider output row (a mixed batch uses
        // the widest code's row) is zero-filled beyond it
        const uint8_t* pbb = reinterpret_cast<const uint8_t*>(pb);
        uint8_t* out = a.bits + (size_t)frame * a.row_bytes;
        const int prow = (C.P + 7) >> 3;
        for (int i = t; i < a.row_bytes; i += T) out[i] = i < prow ? pbb[i] : (uint8_t)0;
        if (t == 0) {
            a.iters[frame] = (uint16_t)it_done;
            a.status[frame] = ok ? POLAR_FRAME_BP_OK : POLAR_FRAME_BP_FAIL;
            if (!ok && a.fail_list) {
                a.fail_list[atomicAdd(a.fail_count, 1)] = frame;
                if (a.fail_total) atomicAdd(a.fail_total, 1);
            }
        }
        if (a.llr_u) {
#pragma unroll
            for (int k = 0; k < R; ++k)
                a.llr_u[(size_t)frame * N + P::node(0, t, k)] = MT::to_f(fadd(Lc[1][k], Rc[1][k]), h);
        }
        if (a.llr_x) {
            // R[n+1] of the last R sweep, recomputed from R[n] and the channel column
            chan_reload();
            constexpr int q = n - 1, g = P::grp(q), dd = 1 << (q - P::win(g));
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (k & dd) continue;
                const int k2 = k | dd;
                MSG o1, gg;
                gf2(Rc[n][k], fadd(Lc[n + 1][k2], Rc[n][k2]), Rc[n][k], Lc[n + 1][k], o1, gg);
                if constexpr (WEIGHTED) {
                    // itc of this half was already advanced past the last iteration
                    const MSG w1 = MT::splat(wscalar(it_done - 1, 0, n, k));
                    const MSG w2 = MT::splat(wscalar(it_done - 1, 0, n, k2));
                    o1 = clipm(fmul(w1, o1), Mv);
                    gg = fmul(w2, gg);
                }
                const MSG o2 = clipm(fadd(gg, Rc[n][k2]), Mv);
                a.llr_x[(size_t)frame * N + P::node(g, t, k)] = MT::to_f(fadd(Lc[n + 1][k], o1), h);
                a.llr_x[(size_t)frame * N + P::node(g, t, k2)] = MT::to_f(fadd(Lc[n + 1][k2], o2), h);
            }
        }
    };

    // replace the frame of half h by the next one: channel column and zeroed L messages (R too
    // where ZERO_R; the next R sweep rewrites them before it reads them)
    auto refill = [&](int h) {
        fr[h] = fetch();
        itc[h] = 0;
        const float* y = fr[h] >= 0 ? row(fr[h]) : nullptr;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float v = y ? stage_clip(__ldg(y + P::node(NG - 1, t, k)), M) : 0.0f;
            if constexpr (CHS)
                xput<P, NG - 1>(chs, xbase, t, k, MT::set_half(xget<P, NG - 1>(chs, xbase, t, k), v, h));
            else
                Lc[n + 1][k] = MT::set_half(Lc[n + 1][k], v, h);
        }
#pragma unroll
        for (int c = 2; c <= n; ++c)
#pragma unroll
            for (int k = 0; k < R; ++k) {
                Lc[c][k] = MT::zero_half(Lc[c][k], h);
                if constexpr (ZERO_R) Rc[c][k] = MT::zero_half(Rc[c][k], h);
            }
    };

    // DEFER (one FP32 frame over several warps): the warps' partial syndromes of an iteration are
    // read after the first exchange barrier of the next one, which orders them, instead of after
    // a barrier of their own.  The next iteration's stages before that barrier are computed
    // before the stop decision; if the frame stops they are dropped.  They write only R[2..SC]
    // and the exchange buffer, and the outputs read L[1], R[1], R[n] and L[n+1] (SC < n).
    constexpr int SC = first_rcross<P>();
    // (Not in the mixed kernel, whose many plans would spill more with it, and not in the exact-g
    // kernel at N = 4096, measured 4% slower with it.)
    constexpr bool DEFER = FPT == 1 && !WEIGHTED && !REENC && NW > 1 && SC > 0 && SC < n &&
                           !(EXACT && n == 12) && std::is_same<Src, CounterSource>::value;
    bool pending = false;  // DEFER: an iteration's partial syndromes are written, not yet read
    int it = 0;  // iterations run by this group (selects the partial-syndrome slot parity)
    for (;;) {
        // scales of the stage being computed and of the next one (loaded a stage ahead)
        WSet wc{}, wn{};
        if constexpr (WEIGHTED) wc = wload(0, 1);
        uint32_t xh = 0;  // re-encoding stop: HD(LLR(x)) of this thread's channel-column nodes
        // ------------------------------------------------------------------ R sweep
        auto rstage = [&](auto S) {
            constexpr int s = S.value, q = s - 1, g = P::grp(q), dd = 1 << (q - P::win(g));
            constexpr bool last = s == n;
            constexpr bool cross = P::rcross(s);
            MSG* xb = xbuf + (P::xidx_r(s) & 1) * P::XW;
            if constexpr (WEIGHTED) wn = last ? wload(1, n) : wload(0, s + 1);
            if constexpr (last) chan_reload();
            // outputs of the PE (k, k2): R[s+1] registers, the exchange buffer, or (last stage) only
            // the re-encoding stop's hard decisions of LLR(x)
            auto emit = [&](int k, int k2, MSG o1, MSG o2) {
                if constexpr (REENC && last) {
                    // LLR(x) = L[n+1] + R[n+1]: the channel column plus this stage's output
                    xh |= (MT::neg(fadd(Lc[s + 1][k], o1), 0) ? 1u : 0u) << k;
                    xh |= (MT::neg(fadd(Lc[s + 1][k2], o2), 0) ? 1u : 0u) << k2;
                }
                if constexpr (!last) {
                    if constexpr (cross) {
                        xput<P, g>(xb, xbase, t, k, o1);
                        xput<P, g>(xb, xbase, t, k2, o2);
                    } else {
                        Rc[s + 1][k] = o1;
                        Rc[s + 1][k2] = o2;
                    }
                }
            };
            if constexpr (PAIRS) {
#pragma unroll
                for (int i = 0; i < R / 2; i += 2) {
                    const int kA = pe_k(dd, i), kB = pe_k(dd, i + 1), kA2 = kA | dd, kB2 = kB | dd;
                    const float2 a1 = make_float2(Rc[s][kA], Rc[s][kB]);
                    const float2 a2 = make_float2(Rc[s][kA2], Rc[s][kB2]);
                    const float2 o1 = gpair(a1, __fadd2_rn(make_float2(Lc[s + 1][kA2], Lc[s + 1][kB2]), a2));
                    const float2 o2 = __fadd2_rn(gpair(a1, make_float2(Lc[s + 1][kA], Lc[s + 1][kB])), a2);
                    emit(kA, kA2, o1.x, clipm(o2.x, M));
                    emit(kB, kB2, o1.y, clipm(o2.y, M));
                }
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if (k & dd) continue;
                    const int k2 = k | dd;
                    const MSG a1 = Rc[s][k], a2 = Rc[s][k2], l1 = Lc[s + 1][k], l2 = Lc[s + 1][k2];
                    MSG o1, gg;
                    gf2(a1, fadd(l2, a2), a1, l1, o1, gg);
                    if constexpr (WEIGHTED) {
                        o1 = fmul(wk(wc, k), o1);
                        if constexpr (!UNIT) o1 = clipm(o1, Mv);
                        gg = fmul(wk(wc, k2), gg);
                    }
                    emit(k, k2, o1, clipm(fadd(gg, a2), Mv));
                }
            }
            if constexpr (cross) {
                group_sync<T, SHARED_CTA>(slot);
                if constexpr (!(DEFER && s == SC)) {
#pragma unroll
                    for (int k = 0; k < R; ++k) Rc[s + 1][k] = xget<P, P::grp(s)>(xb, xbase, t, k);
                }
            }
            if constexpr (WEIGHTED) wc = wn;
        };
        if constexpr (DEFER) {
            static_for<1, SC + 1>(rstage);
            if (pending) {
                // the previous iteration's stop decision, from its partial syndromes
                pending = false;
                const uint32_t* sp = synp + ((it - 1) & 1) * 2 * NW;
                uint32_t sy = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) sy ^= sp[w];
                if constexpr (syn_nodes) sy = (sy ^ (sy >> 16)) & 0xFFFFu;
                const bool ok = sy == 0u;
                if ((ok && !a.fixed_iters) || itc[0] >= a.max_iters) {
                    finalize(0, itc[0], ok);
                    refill(0);
                    if (fr[0] < 0) break;
                    continue;  // the new frame starts its first R sweep
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k) Rc[SC + 1][k] = xget<P, P::grp(SC)>(xbuf + (P::xidx_r(SC) & 1) * P::XW, xbase, t, k);
            static_for<SC + 1, n + 1>(rstage);
        } else {
            static_for<1, n + 1>(rstage);
        }
        // ------------------------------------------------------------------ L sweep
        uint32_t syn0 = 0, syn1 = 0;
        static_for_down<n, 1>([&](auto S) {
            constexpr int s = S.value, q = s - 1, g = P::grp(q), dd = 1 << (q - P::win(g));
            constexpr bool first = s == 1;
            constexpr bool cross = P::lcross(s);
            MSG* xb = xbuf + (P::xidx_l(s) & 1) * P::XW;
            if constexpr (WEIGHTED && !first) wn = wload(1, s - 1);
            if constexpr (s == n) chan_reload();
            auto emit = [&](int k, int k2, MSG o1, MSG o2) {
                if constexpr (cross) {
                    xput<P, g>(xb, xbase, t, k, o1);
                    xput<P, g>(xb, xbase, t, k2, o2);
                } else {
                    Lc[s][k] = o1;
                    Lc[s][k2] = o2;
                }
            };
            if constexpr (PAIRS) {
#pragma unroll
                for (int i = 0; i < R / 2; i += 2) {
                    const int kA = pe_k(dd, i), kB = pe_k(dd, i + 1), kA2 = kA | dd, kB2 = kB | dd;
                    const float2 l1 = make_float2(Lc[s + 1][kA], Lc[s + 1][kB]);
                    const float2 l2 = make_float2(Lc[s + 1][kA2], Lc[s + 1][kB2]);
                    const float2 o1 = gpair(l1, __fadd2_rn(l2, make_float2(Rc[s][kA2], Rc[s][kB2])));
                    const float2 o2 = __fadd2_rn(gpair(make_float2(Rc[s][kA], Rc[s][kB]), l1), l2);
                    emit(kA, kA2, o1.x, clipm(o2.x, M));
                    emit(kB, kB2, o1.y, clipm(o2.y, M));
                }
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    if (k & dd) continue;
                    const int k2 = k | dd;
                    const MSG a1 = Rc[s][k], a2 = Rc[s][k2], l1 = Lc[s + 1][k], l2 = Lc[s + 1][k2];
                    MSG o1, gg;
                    gf2(l1, fadd(l2, a2), a1, l1, o1, gg);
                    if constexpr (WEIGHTED) {
                        o1 = fmul(wk(wc, k), o1);
                        if constexpr (!UNIT) o1 = clipm(o1, Mv);
                        gg = fmul(wk(wc, k2), gg);
                    }
                    emit(k, k2, o1, clipm(fadd(gg, l2), Mv));
                }
            }
            if constexpr (cross) {
                group_sync<T, SHARED_CTA>(slot);
#pragma unroll
                for (int k = 0; k < R; ++k) Lc[s][k] = xget<P, P::grp(s - 2)>(xb, xbase, t, k);
            }
            if constexpr (WEIGHTED && !first) wc = wn;
            if constexpr (first) {
                // hard decision of LLR(u) = L[1] + R[1]; XOR of the syndrome columns of the
                // information nodes decided 1 (frozen nodes have column 0).  On an information
                // node R[1] = +0, so u is never -0 and its sign bit is exactly (u < 0): the
                // decision is an arithmetic shift and the update one and-xor.
                if constexpr (syn_nodes) {
                    // one byte permute replicates the sign bits of u[k] and u[k + 1] into a 16|16
                    // mask over the pair's column word; one 64-bit load brings two such words
                    const uint2* cs2 = reinterpret_cast<const uint2*>(csyn);
#pragma unroll
                    for (int k = 0; k < R; k += 4) {
                        const uint2 cw = cs2[(k >> 2) * T + t];
                        const float2 u0 = __fadd2_rn(make_float2(Lc[1][k], Lc[1][k + 1]),
                                                     make_float2(Rc[1][k], Rc[1][k + 1]));
                        const float2 u1 = __fadd2_rn(make_float2(Lc[1][k + 2], Lc[1][k + 3]),
                                                     make_float2(Rc[1][k + 2], Rc[1][k + 3]));
                        uint32_t m0, m1;
                        asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(m0) : "r"(__float_as_uint(u0.x)), "r"(__float_as_uint(u0.y)));
                        asm("prmt.b32 %0, %1, %2, 0xFFBB;" : "=r"(m1) : "r"(__float_as_uint(u1.x)), "r"(__float_as_uint(u1.y)));
                        syn0 ^= cw.x & m0;
                        syn0 ^= cw.y & m1;
                    }
                } else if constexpr (syn_packed) {
                    // one byte permute replicates the sign bits of both halves into a 16|16 mask
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const MSG u = fadd(Lc[1][k], Rc[1][k]);
                        uint32_t ub, m;
                        memcpy(&ub, &u, 4);
                        asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(ub));
                        syn0 ^= csyn[k * T + t] & m;
                    }
                } else if constexpr (PAIRS) {
#pragma unroll
                    for (int k = 0; k < R; k += 2) {
                        const float2 u = __fadd2_rn(make_float2(Lc[1][k], Lc[1][k + 1]),
                                                    make_float2(Rc[1][k], Rc[1][k + 1]));
                        syn0 ^= csyn[k * T + t] & (uint32_t)(__float_as_int(u.x) >> 31);
                        syn0 ^= csyn[(k + 1) * T + t] & (uint32_t)(__float_as_int(u.y) >> 31);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const MSG u = fadd(Lc[1][k], Rc[1][k]);
                        const uint32_t col = csyn[k * T + t];
                        uint32_t ub;
                        memcpy(&ub, &u, 4);
                        if constexpr (FPT == 2) {
                            syn0 ^= col & (uint32_t)((int32_t)(ub << 16) >> 31);
                            syn1 ^= col & (uint32_t)((int32_t)ub >> 31);
                        } else {
                            syn0 ^= col & (uint32_t)((int32_t)ub >> 31);
                        }
                    }
                }
            }
        });
        // ------------------------------------------------------------------ CRC early stop
        syn0 = __reduce_xor_sync(0xffffffffu, syn0);
        if constexpr (DEFER) {
            if ((t & 31) == 0) synp[(it & 1) * 2 * NW + (t >> 5)] = syn0;
            ++it;
            ++itc[0];
            pending = true;
            continue;  // read and decided after the next iteration's first exchange barrier
        }
        if constexpr (FPT == 2 && !syn_packed) syn1 = __reduce_xor_sync(0xffffffffu, syn1);
        if constexpr (NW > 1) {
            uint32_t* sp = synp + (it & 1) * 2 * NW;
            if ((t & 31) == 0) {
                sp[t >> 5] = syn0;
                if constexpr (FPT == 2 && !syn_packed) sp[NW + (t >> 5)] = syn1;
            }
            group_sync<T, SHARED_CTA>(slot);
            syn0 = 0;
            syn1 = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                syn0 ^= sp[w];
                if constexpr (FPT == 2 && !syn_packed) syn1 ^= sp[NW + w];
            }
        }
        if constexpr (syn_nodes) {
            syn0 = (syn0 ^ (syn0 >> 16)) & 0xFFFFu;
        } else if constexpr (syn_packed) {
            syn1 = syn0 >> 16;
            syn0 &= 0xFFFFu;
        }
        bool conv = false;
        if constexpr (REENC) {
            // x = u G by the butterflies of Fig. 1 on the decided bits (stage q XORs node j + 2^q
            // into node j): in registers within a group's window, through the exchange buffers
            // between groups (the R sweep's buffers and alternation; the vote below is the barrier
            // that orders the last exchange's reads before the next iteration's first writes)
            uint32_t v = 0;
#pragma unroll
            for (int k = 0; k < R; ++k) v |= (MT::neg(fadd(Lc[1][k], Rc[1][k]), 0) ? 1u : 0u) << k;
            static_for<1, n + 1>([&](auto S) {
                constexpr int s = S.value, q = s - 1, g = P::grp(q), dd = 1 << (q - P::win(g));
                v ^= (v >> dd) & pe_low_mask<R>(dd);
                if constexpr (P::rcross(s)) {
                    uint32_t* xb = reinterpret_cast<uint32_t*>(xbuf + (P::xidx_r(s) & 1) * P::XW);
#pragma unroll
                    for (int k = 0; k < R; ++k) xput<P, g>(xb, xbase, t, k, (v >> k) & 1u);
                    group_sync<T, SHARED_CTA>(slot);
                    v = 0;
#pragma unroll
                    for (int k = 0; k < R; ++k) v |= xget<P, P::grp(s)>(xb, xbase, t, k) << k;
                }
            });
            // v now holds the re-encoded bits of this thread's channel-column nodes, as xh does
            if constexpr (T == 32)
                conv = !__any_sync(0xffffffffu, v != xh);
            else
                conv = !__syncthreads_or(v != xh);
        }
        ++it;
        const uint32_t syn[2] = {syn0, syn1};
        bool any = false;
        if constexpr (ALIGNED) {
            // a frame that stops is written out and its half idles (its lanes compute values
            // nobody reads) until the partner stops too; then both refill and restart at 0
            ++itp;
            bool pair_done = true;
#pragma unroll
            for (int h = 0; h < FPT; ++h) {
                if (fr[h] >= 0 && itc[h] >= 0) {
                    ++itc[h];
                    const bool ok = syn[h] == 0u;
                    if ((ok && !a.fixed_iters) || itc[h] >= a.max_iters) {
                        finalize(h, itc[h], ok);
                        itc[h] = -1;
                    }
                }
                pair_done &= fr[h] < 0 || itc[h] < 0;
            }
            if (pair_done) {
#pragma unroll
                for (int h = 0; h < FPT; ++h) refill(h);
                itp = 0;
            }
            any = fr[0] >= 0 || fr[1] >= 0;
        } else {
#pragma unroll
            for (int h = 0; h < FPT; ++h) {
                if (fr[h] < 0) continue;
                ++itc[h];
                const bool ok = syn[h] == 0u;
                const bool stop = REENC ? conv : ok;
                if ((stop && !a.fixed_iters) || itc[h] >= a.max_iters) {
                    finalize(h, itc[h], ok);
                    refill(h);
                }
                any |= fr[h] >= 0;
            }
        }
        if (!any) break;
    }
}

// Resident CTAs per SM that a kernel's register allocation targets: the exact PE function (VAR
// bit 0) keeps more temporaries live than min-sum and takes the weighted kernels' budget up to
// N = 1024 (from N = 2048 on, fewer CTAs would leave too few warps per SM).
template <int LOGN, int WEIGHTED, int VAR>
constexpr int bp_min_ctas()
{
    if (WEIGHTED == 2) return BPConfig<LOGN>::MIN_CTAS_U;
    return WEIGHTED != 0 || ((VAR & 1) && LOGN <= 10) ? BPConfig<LOGN>::MIN_CTAS_W : BPConfig<LOGN>::MIN_CTAS;
}

// Per-length kernel: F frame groups per CTA; THREADS = F * T (passed explicitly: launch bounds
// take no dependent member expression).
template <int LOGN, class MSG, int WEIGHTED, int THREADS, bool SYNP = false, int VAR = 0>
__global__ void __launch_bounds__(THREADS, bp_min_ctas<LOGN, WEIGHTED, VAR>()) bp_kernel(const BPArgs a)
{
    using P = typename BPKernelPlan<LOGN, WEIGHTED, VAR, MsgTraits<MSG>::FPT>::Plan;
    constexpr int F = BPKernelPlan<LOGN, WEIGHTED, VAR, MsgTraits<MSG>::FPT>::F;
    static_assert(THREADS == F * P::T, "launch shape");
    static_assert(P::T <= 32 || F == 1, "frame groups wider than a warp own their CTA");
    extern __shared__ uint32_t smem[];
    const int slot = threadIdx.x / P::T;
    const int t = threadIdx.x % P::T;
    constexpr int FPT = MsgTraits<MSG>::FPT;
    CounterSource src{a.next, a.B, (int)((blockIdx.x * F + slot) * FPT), FPT, a.frame0};
    bp_run_group<P, MSG, WEIGHTED, false, CounterSource, SYNP, VAR>(a, *a.code, slot, t,
                                                                    smem + slot * bp_slot_words<P>(), src);
}

}  // namespace polar
