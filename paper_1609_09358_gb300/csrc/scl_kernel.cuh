// scl_kernel.cuh -- CRC-aided successive cancellation list decoding (Sec. II-A of the paper).
//
// One warp decodes one frame; a persistent grid takes frames from a device work counter (the
// CRC-failed frames compacted by the BP kernel, or all frames).  SC tree: level k holds 2^k LLRs
// per path (level n is the channel, level 0 the bit LLR).  For bit i > 0 with t = ctz(i) the
// path recomputes level t by g from level t+1 and the partial sums C_t of the left sibling, then
// levels t-1..0 by f; bit 0 runs f from the channel down.  f(a, b) = sign(a) sign(b) min(|a|,|b|),
// g(a, b, v) = b + (1 - 2v) a.
//
// List step at an information bit (lane = candidate): candidate c = 2p + b of path p gets metric
// m + |lambda| [b != HD(lambda)]; its rank is the number of candidates before it in
// (metric, index) order -- the paper's pruned pseudo sort d = sum H(m_c - m_j) made a total order
// by the index tie-break -- and the rank < L candidates survive, renumbered in ascending index.
//
// Leaf blocks in registers: the tree below level 6 is a 32-bit leaf block.  Lane p holds path p's
// LLR arrays of levels 5..1 (62 values) and its partial sums of levels 0..4 (one word each) in
// registers; the 32 bits of a block are unrolled, so every level index is a compile-time constant.
// When a list step duplicates paths, a survivor copies from its parent's lane (shuffles) only the
// leaf levels that a later bit of the block reads before rewriting -- a set known at compile time.
//
// Upper levels (LLR 6..n-1, partial sums 5..n) are touched once per block.  They use lazy copies:
// every upper level keeps L physical arrays and a path holds one 5-bit pointer per level, packed in
// two registers per table.  A survivor copies only its parent's pointer words; a path about to
// rewrite a level it shares takes a free array of that level (the lowest-numbered sharer keeps the
// old one), so no upper-level data is ever copied.  The small upper levels live in the warp's
// shared memory, the large ones in its slot of the global workspace (L2-resident).
//
// Partial sums: after deciding bit i, the completed subtree re-encodes bottom-up,
// v_{k+1} = (C_k xor v_k) || v_k, until the first level k where the completed node is a left
// child (k = number of trailing ones of i); v_k is stored there.  After the last bit the level-n
// array holds the path's codeword x, and u = x G (G is an involution) gives the decided bits for
// the CRC check and the output.
#pragma once

#include <algorithm>

#include "polar_common.cuh"

namespace polar {

struct SCLArgs {
    const float* llr;
    int B;
    int L;
    uint8_t* bits;
    uint8_t* status;
    const DevCode* code;
    const int* list;   // frame indices to decode (null: 0..B-1)
    const int* count;  // device count of `list` (null: B)
    int* next;         // work counter, zero before the launch
    float* scratch;    // per-warp slots of the global levels (null: all levels in shared memory)
    int row_bytes;
    int KS, KC;        // last LLR / partial-sum level kept in shared memory (single code)
    int warp_words;    // shared-memory words per warp
    long long slot_words;  // global words per warp
    // several codes in one batch: code_of[frame] selects codes[], llr_off[frame] the LLR row
    const int* code_of;
    const long long* llr_off;
    const DevCode* codes[32];
};

__host__ __device__ inline int scl_cw(int k) { return k < 5 ? 1 : 1 << (k - 5); }  // words of a level-k C array
// Per-path stride of the level-k C arrays: one pad word beyond a single word makes the stride
// odd, so the same word of different paths falls in different banks.
__host__ __device__ inline int scl_cs(int k) { return scl_cw(k) > 1 ? scl_cw(k) + 1 : 1; }
__host__ __device__ inline int scl_cssum(int k) { return k <= 5 ? k : (1 << (k - 5)) + k - 2; }  // sum of cs(q), q < k

__host__ __device__ inline int log2_host(int v)
{
    int n = 0;
    while ((1 << n) < v) ++n;
    return n;
}

// Host plan of the shared/global split of the upper levels for (N, L): LLR levels 6..KS and
// partial-sum levels 5..KC in shared memory, the rest in the warp's global slot.
struct SCLPlan {
    int KS, KC;
    int warp_words;
    long long slot_words;
};
// Level 5 of every path is computed element-parallel into a staging row per path (33 words: the
// pad makes both the warp's row-wise writes and the lanes' per-path reads bank-conflict free) and
// then read into the path's registers.
constexpr int kSclStage = 33;
__host__ __device__ inline long long scl_smem_llr_words(int KS, int L) { return KS >= 6 ? (long long)L * ((2 << KS) - 64) : 0; }
__host__ __device__ inline long long scl_smem_c_words(int KC, int L) { return KC >= 5 ? (long long)L * (scl_cssum(KC + 1) - 5) : 0; }
__host__ __device__ inline SCLPlan scl_plan(int N, int L, bool all_smem)
{
    const int n = log2_host(N);
    SCLPlan p{};
    if (all_smem) {
        p.KS = n - 1;
        p.KC = n;
    } else {
        p.KS = 5;
        while (p.KS + 1 <= n - 1 && 4 * scl_smem_llr_words(p.KS + 1, L) <= 6144) ++p.KS;
        p.KC = 4;
        while (p.KC + 1 <= n && 4 * scl_smem_c_words(p.KC + 1, L) <= 2048) ++p.KC;
    }
    // [C levels 5..KC][LLR levels 6..KS][level-5 staging, L rows of 33 words][list scratch, 16 words]
    p.warp_words = (int)(scl_smem_llr_words(p.KS, L) + scl_smem_c_words(p.KC, L)) + L * kSclStage + 16;
    p.warp_words = (p.warp_words + 3) & ~3;
    p.slot_words = (long long)L * (N - (2 << p.KS)) + (long long)L * (scl_cssum(n + 1) - scl_cssum(p.KC + 1));
    return p;
}
inline bool scl_fits_smem(int N, int L) { return 4LL * scl_plan(N, L, true).warp_words <= 80 * 1024; }
constexpr int kSclWarpsPerSM = 32;
constexpr int kSclWarpsPerCTA = 4;
inline int scl_sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}
// global workspace of the SCL list arrays (one slot per resident warp)
inline size_t scl_scratch_bytes(int N, int L)
{
    const SCLPlan p = scl_plan(N, L, false);
    return (size_t)scl_sm_count() * kSclWarpsPerSM * (size_t)p.slot_words * 4;
}

__device__ __forceinline__ uint32_t fld(const uint32_t (&w)[2], int k) { return ((k < 6 ? w[0] : w[1]) >> (5 * (k % 6))) & 31u; }
__device__ __forceinline__ void set_fld(uint32_t (&w)[2], int k, uint32_t v)
{
    const int s = 5 * (k % 6);
    if (k < 6)
        w[0] = (w[0] & ~(31u << s)) | (v << s);
    else
        w[1] = (w[1] & ~(31u << s)) | (v << s);
}

// A path about to rewrite level k that it shares takes a free array of that level (lane = path;
// `act` active paths; the lowest lane of each group of sharers keeps its array).
__device__ __forceinline__ void scl_own(uint32_t (&w)[2], int k, int act, int L)
{
    const int lane = threadIdx.x & 31;
    const bool on = lane < act;
    const uint32_t mine = on ? fld(w, k) : 64u + lane;
    const uint32_t same = __match_any_sync(0xffffffffu, mine);
    const uint32_t below = (1u << lane) - 1u;
    const bool need = on && (same & below) != 0u;
    const uint32_t used = __reduce_or_sync(0xffffffffu, on ? (1u << mine) : 0u);
    uint32_t freem = ~used & (L >= 32 ? 0xffffffffu : ((1u << L) - 1u));
    const int r = __popc(__ballot_sync(0xffffffffu, need) & below);
    if (need) {
        for (int q = 0; q < r; ++q) freem &= freem - 1u;  // drop the r lowest free arrays
        set_fld(w, k, (uint32_t)(__ffs(freem) - 1));
    }
}

__device__ __forceinline__ float scl_g(float a, float b, uint32_t v) { return v ? __fsub_rn(b, a) : __fadd_rn(b, a); }

struct SCLWarp {
    float* stage;  // shared level-5 staging rows [L][kSclStage]
    float* sA;     // shared LLR levels 6..KS
    uint32_t* sC;  // shared partial-sum levels 5..KC
    float* gA;     // global LLR levels KS+1..n-1
    uint32_t* gC;  // global partial-sum levels KC+1..n
    int L, KS, KC;
    __device__ __forceinline__ float* A(int k) const  // k >= 6
    {
        return k <= KS ? sA + L * ((1 << k) - 64) : gA + L * ((1 << k) - (2 << KS));
    }
    __device__ __forceinline__ uint32_t* Cl(int k) const  // k >= 5
    {
        return k <= KC ? sC + L * (scl_cssum(k) - 5) : gC + L * (scl_cssum(k) - scl_cssum(KC + 1));
    }
};

// ------------------------------------------------------------------ leaf block (compile time)
__host__ __device__ constexpr int ctz_c(int v)
{
    int c = 0;
    while (!(v & 1)) {
        v >>= 1;
        ++c;
    }
    return c;
}
__host__ __device__ constexpr int tones_c(int v)  // trailing ones
{
    int c = 0;
    while (v & 1) {
        v >>= 1;
        ++c;
    }
    return c;
}
// Is leaf level k (1..5) read, before being rewritten, by a later bit of the block than r?
__host__ __device__ constexpr bool leaf_live(int r, int k)
{
    for (int q = r + 1; q < 32; ++q) {
        const int t = ctz_c(q);
        if (t + 1 == k) return true;
        if (t >= k) return false;
    }
    return false;
}

template <int LEN>
__device__ __forceinline__ void leaf_f(const float (&src)[2 * LEN], float (&dst)[LEN])
{
#pragma unroll
    for (int j = 0; j < LEN; ++j) dst[j] = xmin(src[j], src[j + LEN]);
}
template <int LEN>
__device__ __forceinline__ void leaf_g(const float (&src)[2 * LEN], float (&dst)[LEN], uint32_t c)
{
#pragma unroll
    for (int j = 0; j < LEN; ++j) dst[j] = scl_g(src[j], src[j + LEN], (c >> j) & 1u);
}
template <int LEN>
__device__ __forceinline__ void leaf_copy(float (&a)[LEN], int parent)
{
#pragma unroll
    for (int j = 0; j < LEN; ++j) a[j] = __shfl_sync(0xffffffffu, a[j], parent);
}

struct Leaf {
    float l5[32], l4[16], l3[8], l2[4], l1[2];
    uint32_t c[5];  // partial sums of the left siblings at levels 0..4
};

// LLR of bit r of the block (levels written: ctz(r)..1, read: ctz(r)+1 and c[ctz(r)])
template <int R>
__device__ __forceinline__ float leaf_llr(Leaf& f)
{
    if constexpr (R == 0) {
        leaf_f<16>(f.l5, f.l4);
        leaf_f<8>(f.l4, f.l3);
        leaf_f<4>(f.l3, f.l2);
        leaf_f<2>(f.l2, f.l1);
        return xmin(f.l1[0], f.l1[1]);
    } else {
        constexpr int t = ctz_c(R);
        if constexpr (t == 4) leaf_g<16>(f.l5, f.l4, f.c[4]);
        if constexpr (t == 3) leaf_g<8>(f.l4, f.l3, f.c[3]);
        if constexpr (t == 2) leaf_g<4>(f.l3, f.l2, f.c[2]);
        if constexpr (t == 1) leaf_g<2>(f.l2, f.l1, f.c[1]);
        if constexpr (t == 0) return scl_g(f.l1[0], f.l1[1], f.c[0] & 1u);
        if constexpr (t >= 4) leaf_f<8>(f.l4, f.l3);
        if constexpr (t >= 3) leaf_f<4>(f.l3, f.l2);
        if constexpr (t >= 2) leaf_f<2>(f.l2, f.l1);
        return xmin(f.l1[0], f.l1[1]);
    }
}

// after a duplicating list step at bit r: survivors take the live leaf state of their parents
template <int R>
__device__ __forceinline__ void leaf_inherit(Leaf& f, int parent)
{
    if constexpr (leaf_live(R, 5)) leaf_copy<32>(f.l5, parent);
    if constexpr (leaf_live(R, 4)) leaf_copy<16>(f.l4, parent);
    if constexpr (leaf_live(R, 3)) leaf_copy<8>(f.l3, parent);
    if constexpr (leaf_live(R, 2)) leaf_copy<4>(f.l2, parent);
    if constexpr (leaf_live(R, 1)) leaf_copy<2>(f.l1, parent);
#pragma unroll
    for (int k = 0; k < 5; ++k) f.c[k] = __shfl_sync(0xffffffffu, f.c[k], parent);
}

// The same inheritance with the bit index at run time: `live` = bit k-1 set when leaf level k is
// live after bit r (leaf_live_mask); one copy of the code serves every bit of the block.
// Closed form of the same table: level k is next touched at q, the first multiple of 2^(k-1) after
// r; bit q reads it (by g) iff ctz(q) = k-1, rewrites it iff ctz(q) >= k.
__host__ __device__ constexpr uint32_t leaf_live_mask(int r)
{
    uint32_t m = 0;
    for (int k = 1; k <= 5; ++k) {
        const int q = (r | ((1 << (k - 1)) - 1)) + 1;
        if (q < 32 && ((q >> (k - 1)) & 1)) m |= 1u << (k - 1);
    }
    return m;
}
constexpr bool leaf_live_mask_matches()
{
    for (int r = 0; r < 32; ++r)
        for (int k = 1; k <= 5; ++k)
            if (((leaf_live_mask(r) >> (k - 1)) & 1u) != (leaf_live(r, k) ? 1u : 0u)) return false;
    return true;
}
static_assert(leaf_live_mask_matches(), "closed form of the leaf liveness table");
__device__ __forceinline__ void leaf_inherit_rt(Leaf& f, int parent, uint32_t live)
{
    if (live & 16u) leaf_copy<32>(f.l5, parent);
    if (live & 8u) leaf_copy<16>(f.l4, parent);
    if (live & 4u) leaf_copy<8>(f.l3, parent);
    if (live & 2u) leaf_copy<4>(f.l2, parent);
    if (live & 1u) leaf_copy<2>(f.l1, parent);
#pragma unroll
    for (int k = 0; k < 5; ++k) f.c[k] = __shfl_sync(0xffffffffu, f.c[k], parent);
}

// partial sums after bit r (value `bitv`): returns the level-5 value when the block completes
template <int R>
__device__ __forceinline__ uint32_t leaf_psum(Leaf& f, uint32_t bitv)
{
    constexpr int kc = tones_c(R);
    uint32_t v = bitv;
#pragma unroll
    for (int k = 0; k < (kc < 5 ? kc : 5); ++k) {
        const uint32_t m = (k == 4) ? 0xFFFFu : ((1u << (1 << k)) - 1u);
        v = ((v ^ f.c[k]) & m) | ((v & m) << (1 << k));
    }
    if constexpr (kc < 5) f.c[kc] = v;
    return v;
}

// Launches the persistent CA-SCL grid (defined in scl_launch.cu).  `a.scratch` null selects the
// all-shared-memory layout; warp_words_max / slot_words_max widen the per-warp storage for mixed
// batches.
cudaError_t scl_launch(SCLArgs a, int N, int L, cudaStream_t st, int warp_words_max = 0,
                       long long slot_words_max = 0);

#ifdef POLAR_SCL_KERNELS
#define SCL_FOR_8(M, B) M(B + 0) M(B + 1) M(B + 2) M(B + 3) M(B + 4) M(B + 5) M(B + 6) M(B + 7)
#define SCL_FOR_32(M) SCL_FOR_8(M, 0) SCL_FOR_8(M, 8) SCL_FOR_8(M, 16) SCL_FOR_8(M, 24)

// One list step at an information bit: candidates, ranks, survivors.  Lane = path in and out;
// returns the survivor's parent lane and decided bit, updates pm/act, reports duplication and
// whether any survivor sits in another lane than its parent (`moved`, warp-uniform).
template <bool TWO>
__device__ __forceinline__ int scl_list_step(float lam, float& pm, int& act, int L, uint8_t* selc, uint32_t& bitv,
                                             bool& dup, bool& moved)
{
    const int lane = threadIdx.x & 31;
    if (act == L) {
        // Full list: when every path's hard-decision child (metric pm) comes before every
        // penalised child (pm + |lambda|), the L survivors are exactly the hard-decision children,
        // in path order -- the same result as the ranking below, without it.  Metrics are >= +0,
        // so their bit patterns order like their values.
        const bool on = lane < act;
        const uint32_t hd_max = __reduce_max_sync(0xffffffffu, on ? __float_as_uint(pm) : 0u);
        const uint32_t pen_min =
            __reduce_min_sync(0xffffffffu, on ? __float_as_uint(__fadd_rn(pm, fabsf(lam))) : 0xffffffffu);
        if (hd_max < pen_min) {
            bitv = lam < 0.0f ? 1u : 0u;
            dup = false;
            moved = false;
            return lane;
        }
    }
    const int nc = 2 * act;
    float cm0, cm1 = 0.0f;
    {
        const float lp = __shfl_sync(0xffffffffu, lam, (lane >> 1) & 31);
        const float pp = __shfl_sync(0xffffffffu, pm, (lane >> 1) & 31);
        cm0 = ((uint32_t)(lane & 1) != (uint32_t)(lp < 0.0f)) ? __fadd_rn(pp, fabsf(lp)) : pp;
    }
    if constexpr (TWO) {
        const float lp = __shfl_sync(0xffffffffu, lam, 16 + (lane >> 1));
        const float pp = __shfl_sync(0xffffffffu, pm, 16 + (lane >> 1));
        cm1 = ((uint32_t)(lane & 1) != (uint32_t)(lp < 0.0f)) ? __fadd_rn(pp, fabsf(lp)) : pp;
    }
    const uint32_t below = (1u << lane) - 1u;
    uint32_t km0, km1 = 0u;
    if (nc <= L) {
        // every candidate survives
        km0 = __ballot_sync(0xffffffffu, lane < nc);
        if constexpr (TWO) km1 = __ballot_sync(0xffffffffu, lane + 32 < nc);
    } else if (TWO || nc > 16) {
        // Threshold selection.  tau = the L-th smallest metric: with two candidates per lane, a
        // bitonic sort of the first 32 ascending and of the second 32 descending, whose
        // element-wise minimum holds the 32 smallest (the half-cleaner of a bitonic merge); with
        // one per lane, the sorted value of lane L - 1.  The survivors are every candidate below
        // tau and the lowest-index candidates equal to tau -- the L smallest in (metric, index)
        // order, the same set as ranking every candidate.
        const float inf = __int_as_float(0x7f800000);
        float x0 = lane < nc ? cm0 : inf;
        float x1 = (TWO && lane + 32 < nc) ? cm1 : inf;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const float o0 = __shfl_xor_sync(0xffffffffu, x0, j);
                const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
                if constexpr (TWO) {
                    const float o1 = __shfl_xor_sync(0xffffffffu, x1, j);
                    x0 = take_min ? fminf(x0, o0) : fmaxf(x0, o0);
                    x1 = take_min ? fmaxf(x1, o1) : fminf(x1, o1);  // descending
                } else {
                    x0 = take_min ? fminf(x0, o0) : fmaxf(x0, o0);
                }
            }
        }
        float tau;
        if constexpr (TWO)
            tau = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fminf(x0, x1))));  // L = 32
        else
            tau = __shfl_sync(0xffffffffu, x0, L - 1);
        const bool v0 = lane < nc, v1 = TWO && lane + 32 < nc;
        const uint32_t lt0 = __ballot_sync(0xffffffffu, v0 && cm0 < tau);
        const uint32_t lt1 = TWO ? __ballot_sync(0xffffffffu, v1 && cm1 < tau) : 0u;
        const uint32_t eq0 = __ballot_sync(0xffffffffu, v0 && cm0 == tau);
        const uint32_t eq1 = TWO ? __ballot_sync(0xffffffffu, v1 && cm1 == tau) : 0u;
        const int need = L - __popc(lt0) - __popc(lt1);
        km0 = lt0 | __ballot_sync(0xffffffffu, ((eq0 >> lane) & 1u) && __popc(eq0 & below) < need);
        if constexpr (TWO)
            km1 = lt1 | __ballot_sync(0xffffffffu, ((eq1 >> lane) & 1u) && __popc(eq0) + __popc(eq1 & below) < need);
    } else {
        // few candidates (at most 16, one per lane): rank by counting
        int rank0 = 0;
#pragma unroll 8
        for (int c2 = 0; c2 < nc; ++c2) {
            const float o = __shfl_sync(0xffffffffu, cm0, c2);
            rank0 += (o < cm0) || (o == cm0 && c2 < lane);
        }
        km0 = __ballot_sync(0xffffffffu, lane < nc && rank0 < L);
    }
    if (km0 & (1u << lane)) selc[__popc(km0 & below)] = (uint8_t)lane;
    if (TWO && (km1 & (1u << lane))) selc[__popc(km0) + __popc(km1 & below)] = (uint8_t)(lane + 32);
    dup = ((km0 & (km0 >> 1) & 0x55555555u) | (km1 & (km1 >> 1) & 0x55555555u)) != 0u;
    const int nact = __popc(km0) + __popc(km1);
    __syncwarp();
    const int cq = lane < nact ? selc[lane] : 0;
    __syncwarp();
    const float m0 = __shfl_sync(0xffffffffu, cm0, cq & 31);
    const float m1 = TWO ? __shfl_sync(0xffffffffu, cm1, cq & 31) : 0.0f;
    bitv = (uint32_t)(cq & 1);
    pm = lane < nact ? (cq < 32 ? m0 : m1) : 0.0f;
    act = nact;
    moved = __any_sync(0xffffffffu, lane < nact && (cq >> 1) != lane);
    return cq >> 1;
}

template <bool TWO>  // TWO: L = 32, two candidates per lane
__device__ void scl_decode_frame(const SCLArgs& a, const DevCode& C, int frame, const SCLWarp& S, uint8_t* selc)
{
    const int lane = threadIdx.x & 31;
    const int N = C.N, n = C.n, L = a.L;
    const float* y = a.llr + (a.llr_off ? a.llr_off[frame] : (long long)frame * N);
    uint32_t pA[2] = {0u, 0u}, pC[2] = {0u, 0u};  // upper-level pointer rows of path `lane`
    float pm = 0.0f;
    int act = 1;
    uint32_t shA = 0u, shC = 0u;  // upper levels that may be shared since the last duplication
    Leaf lf;
#pragma unroll
    for (int k = 0; k < 5; ++k) lf.c[k] = 0u;
    const int nblocks = N >> 5;
    for (int blk = 0; blk < nblocks; ++blk) {
        // ------------------------------------------------ upper levels on entering the block
        const int t = blk == 0 ? n : 5 + __ffs(blk) - 1;
        const int top = blk == 0 ? n - 1 : t;
        for (int k = top; k >= 5; --k) {
            // level 5 goes to the staging rows (indexed by path), levels >= 6 to their arrays
            const bool stage = k == 5;
            if (!stage && ((shA >> k) & 1u)) {
                scl_own(pA, k, act, L);
                shA &= ~(1u << k);
            }
            const bool use_g = blk != 0 && k == t;
            const bool from_ch = k + 1 == n;
            const int len = 1 << k;
            float* dst = stage ? S.stage : S.A(k);
            const int dstride = stage ? kSclStage : len;
            const float* srcb = from_ch ? y : S.A(k + 1);
            const uint32_t* cbk = S.Cl(k);
            const uint32_t my_d = stage ? (uint32_t)lane : fld(pA, k), my_s = from_ch ? 0u : fld(pA, k + 1),
                           my_c = fld(pC, k);
            const int cwk = scl_cs(k), total = act << k;
            // four elements per lane per round: all loads of a round are issued before any store,
            // so the L2 latency of the upper levels overlaps
            for (int e0 = 0; e0 < total; e0 += 128) {
                float va[4], vb[4];
                uint32_t vw[4], pdv[4];
                int jv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = e0 + 32 * q + lane;
                    const int p = (e >> k) & 31;
                    pdv[q] = __shfl_sync(0xffffffffu, my_d, p);
                    const uint32_t ps = __shfl_sync(0xffffffffu, my_s, p);
                    const uint32_t pc = __shfl_sync(0xffffffffu, my_c, p);
                    jv[q] = e & (len - 1);
                    va[q] = vb[q] = 0.0f;
                    vw[q] = 0u;
                    if (e < total) {
                        const float* src = srcb + ps * (2 * len);
                        va[q] = src[jv[q]];
                        vb[q] = src[jv[q] + len];
                        if (use_g) vw[q] = cbk[pc * cwk + (jv[q] >> 5)];
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = e0 + 32 * q + lane;
                    if (e < total) {
                        const float r = use_g ? scl_g(va[q], vb[q], (vw[q] >> (jv[q] & 31)) & 1u) : xmin(va[q], vb[q]);
                        dst[pdv[q] * dstride + jv[q]] = r;
                    }
                }
            }
            __syncwarp();
        }
        // level 5 of every path into its lane's registers (lanes past the list read row 0: the
        // staging area has L rows)
        {
            const float* row = S.stage + (lane < L ? lane : 0) * kSclStage;
#pragma unroll
            for (int j = 0; j < 32; ++j) lf.l5[j] = row[j];
        }
        // ------------------------------------------------ the 32 bits of the block
        // A runtime loop: one copy of the list step serves all 32 bits, and only the per-bit leaf
        // code (whose register indices are compile-time constants) is dispatched by the bit index.
        // Unrolling the block with a list step inlined per bit overflowed the instruction cache.
        const uint32_t fw = C.frozen_bits[blk];
        uint32_t v5 = 0u;
#pragma unroll 1
        for (int r = 0; r < 32; ++r) {
            float lam = 0.0f;
            switch (r) {
#define SCL_LEAF_LLR(R) \
    case R: lam = leaf_llr<R>(lf); break;
                SCL_FOR_32(SCL_LEAF_LLR)
#undef SCL_LEAF_LLR
            }
            uint32_t bitv = 0u;
            bool moved = false;
            int parent = lane;
            if ((fw >> r) & 1u) {
                if (lane < act && lam < 0.0f) pm = __fadd_rn(pm, fabsf(lam));
            } else {
                bool dup = false;
                parent = scl_list_step<TWO>(lam, pm, act, L, selc, bitv, dup, moved);
                if (moved) {
                    leaf_inherit_rt(lf, parent, leaf_live_mask(r));
                    pA[0] = __shfl_sync(0xffffffffu, pA[0], parent);
                    pA[1] = __shfl_sync(0xffffffffu, pA[1], parent);
                    pC[0] = __shfl_sync(0xffffffffu, pC[0], parent);
                    pC[1] = __shfl_sync(0xffffffffu, pC[1], parent);
                }
                if (dup) shA = shC = 0xffffffffu;
            }
            switch (r) {
#define SCL_LEAF_POST(R) \
    case R: v5 = leaf_psum<R>(lf, bitv); break;
                SCL_FOR_32(SCL_LEAF_POST)
#undef SCL_LEAF_POST
            }
        }
        // ------------------------------------------------ block complete: partial sums upward
        {
            const int i_last = blk * 32 + 31;
            const int kc = __ffs(~i_last) - 1;  // >= 5; n after the last block
            if ((shC >> kc) & 1u) {
                scl_own(pC, kc, act, L);
                shC &= ~(1u << kc);
            }
            uint32_t* dstl = S.Cl(kc);
            const int cwk = scl_cs(kc);
            if (lane < act) dstl[fld(pC, kc) * cwk] = v5;
            __syncwarp();
            const uint32_t my_dst = fld(pC, kc);
            for (int k = 5; k < kc; ++k) {
                const int W = 1 << (k - 5), total = act * W;
                const uint32_t* ckb = S.Cl(k);
                const uint32_t my_k = fld(pC, k);
                for (int e0 = 0; e0 < total; e0 += 32) {
                    const int e = e0 + lane;
                    const int p = (e / W) & 31;
                    const uint32_t pd = __shfl_sync(0xffffffffu, my_dst, p);
                    const uint32_t pk = __shfl_sync(0xffffffffu, my_k, p);
                    if (e < total) {
                        const int w = e % W;
                        uint32_t* dst = dstl + pd * cwk;
                        const uint32_t x = dst[w];
                        dst[W + w] = x;
                        dst[w] = x ^ ckb[pk * scl_cs(k) + w];
                    }
                }
                __syncwarp();
            }
        }
    }
    // ------------------------------------------------------------------ CRC selection
    // u = x G on each path's N-bit codeword (level-n array), in place; syndrome of its
    // information bits
    const int words = N >> 5;
    uint32_t* xl = S.Cl(n);
    const uint32_t my_x = fld(pC, n);
    uint32_t synd = 0xffffffffu;  // lane p: syndrome of path p
    for (int p = 0; p < act; ++p) {
        uint32_t* xw = xl + __shfl_sync(0xffffffffu, my_x, p) * scl_cs(n);
        uint32_t w[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (lane + 32 * h < words) w[h] = xw[lane + 32 * h];
        const uint32_t m[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 5; ++e) w[h] ^= (w[h] >> (1 << e)) & m[e];
        for (int D = 1; D < 32 && D < words; D <<= 1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, w[h], D);
                if (!(lane & D)) w[h] ^= o;
            }
        }
        if (words > 32) w[0] ^= w[1];
        uint32_t s = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int wi = lane + 32 * h;
            if (wi < words) {
                xw[wi] = w[h];
                uint32_t bitsw = w[h];
                while (bitsw) {
                    const int b = __ffs(bitsw) - 1;
                    bitsw &= bitsw - 1u;
                    s ^= C.colsyn[wi * 32 + b];
                }
            }
        }
        s = __reduce_xor_sync(0xffffffffu, s);
        if (lane == p) synd = s;
    }
    __syncwarp();
    // first CRC-passing path in (metric, index) order, else the best metric
    const bool ok_lane = lane < act && synd == 0u;
    const bool any_ok = __ballot_sync(0xffffffffu, ok_lane) != 0u;
    const bool cand = any_ok ? ok_lane : lane < act;
    float key = cand ? pm : __int_as_float(0x7f800000);
    int who = cand ? lane : 64;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const float ok2 = __shfl_xor_sync(0xffffffffu, key, off);
        const int ow = __shfl_xor_sync(0xffffffffu, who, off);
        if (ok2 < key || (ok2 == key && ow < who)) {
            key = ok2;
            who = ow;
        }
    }
    const uint32_t* uw = xl + __shfl_sync(0xffffffffu, my_x, who & 31) * scl_cs(n);
    uint8_t* out = a.bits + (size_t)frame * a.row_bytes;
    for (int by = lane; by < a.row_bytes; by += 32) {
        uint32_t v = 0u;
        for (int r = 0; r < 8; ++r) {
            const int p = by * 8 + r;
            if (p >= C.P) break;
            const int j = C.info_idx[p];
            v |= ((uw[j >> 5] >> (j & 31)) & 1u) << r;
        }
        out[by] = (uint8_t)v;
    }
    if (lane == 0) a.status[frame] = any_ok ? POLAR_FRAME_SCL_OK : POLAR_FRAME_SCL_CRC_FAIL;
    __syncwarp();
}

template <bool TWO>
__global__ void __launch_bounds__(kSclWarpsPerCTA * 32) scl_kernel(const SCLArgs a)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int L = a.L;
    uint32_t* ws = smem + (size_t)wid * a.warp_words;
    uint8_t* selc = reinterpret_cast<uint8_t*>(ws + a.warp_words - 16);
    float* slot = a.scratch ? a.scratch + ((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * (size_t)a.slot_words : nullptr;
    const int count = a.count ? *a.count : a.B;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.next, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;
        const int frame = a.list ? a.list[idx] : idx;
        const DevCode& C = a.code_of ? *a.codes[a.code_of[frame]] : *a.code;
        SCLWarp S;
        S.L = L;
        if (a.code_of) {
            const SCLPlan p = scl_plan(C.N, L, slot == nullptr);
            S.KS = p.KS;
            S.KC = p.KC;
        } else {
            S.KS = a.KS;
            S.KC = a.KC;
        }
        S.sC = ws;
        S.sA = reinterpret_cast<float*>(ws + scl_smem_c_words(S.KC, L));
        S.stage = S.sA + scl_smem_llr_words(S.KS, L);
        S.gA = slot;
        S.gC = slot ? reinterpret_cast<uint32_t*>(slot + (size_t)L * (C.N - (2 << S.KS))) : nullptr;
        scl_decode_frame<TWO>(a, C, frame, S, selc);
    }
}

// Persistent launch: as many CTAs as fit on the device (bounded by the global slots and, when it
// is known on the host, by the work); returns cudaSuccess or the launch error.
cudaError_t scl_launch(SCLArgs a, int N, int L, cudaStream_t st, int warp_words_max, long long slot_words_max)
{
    const bool all_smem = a.scratch == nullptr;
    const SCLPlan p = scl_plan(N, L, all_smem);
    a.KS = p.KS;
    a.KC = p.KC;
    a.warp_words = std::max(p.warp_words, warp_words_max);
    a.slot_words = std::max(p.slot_words, slot_words_max);
    const SCLPlan pw = {p.KS, p.KC, a.warp_words, a.slot_words};
    int W = kSclWarpsPerCTA;
    const size_t wb = (size_t)pw.warp_words * 4;
    while (W > 1 && (size_t)W * wb > 200 * 1024) W >>= 1;
    const size_t smem = (size_t)W * wb;
    const bool two = L > 16;
    const void* fn = two ? (const void*)scl_kernel<true> : (const void*)scl_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, W * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int sms = scl_sm_count();
    long long grid = (long long)sms * per_sm;
    if (!all_smem) grid = std::min<long long>(grid, (long long)sms * kSclWarpsPerSM / W);
    if (!a.list) grid = std::min<long long>(grid, (a.B + W - 1) / W);
    if (grid < 1) grid = 1;
    if (two)
        scl_kernel<true><<<(unsigned)grid, W * 32, smem, st>>>(a);
    else
        scl_kernel<false><<<(unsigned)grid, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

#endif  // POLAR_SCL_KERNELS

}  // namespace polar
