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
#include <type_traits>

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
    int list_words;    // shared-memory words per list (two lists per warp when L <= 8)
    long long slot_words;  // global words per list
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
    int warp_words, list_words;
    long long slot_words;
};
// Level 5 of every path is computed element-parallel into a staging row per path (33 words: the
// pad makes both the warp's row-wise writes and the lanes' per-path reads bank-conflict free) and
// then read into the path's registers.
constexpr int kSclStage = 33;
// elements per lane and round of the element-parallel upper-level updates (measured: 8 beats 4,
// which waits on L2 once per 4 loads, and 16, whose registers cost more than the overlap gains
// once 16 warps share the SM)
constexpr int kSclUpRound = 8;
__host__ __device__ inline long long scl_smem_llr_words(int KS, int L) { return KS >= 6 ? (long long)L * ((2 << KS) - 64) : 0; }
__host__ __device__ inline long long scl_smem_c_words(int KC, int L) { return KC >= 5 ? (long long)L * (scl_cssum(KC + 1) - 5) : 0; }
// `lists` = frames per warp (1, or 2 with half-warp lists): the shared-memory budget of a frame
// is divided by it.
__host__ __device__ inline SCLPlan scl_plan(int N, int L, bool all_smem, int lists = 1)
{
    const int n = log2_host(N);
    SCLPlan p{};
    if (all_smem) {
        p.KS = n - 1;
        p.KC = n;
    } else {
        p.KS = 5;
        // up to 6 KB of LLR levels per frame (8 KB, which puts level 6 of a 32-path list in shared
        // memory, measured 3% slower for a single frame and 3% faster for 2^16 frames: not kept)
        while (p.KS + 1 <= n - 1 && 4 * scl_smem_llr_words(p.KS + 1, L) * lists <= 6144) ++p.KS;
        p.KC = 4;
        while (p.KC + 1 <= n && 4 * scl_smem_c_words(p.KC + 1, L) * lists <= 2048) ++p.KC;
    }
    // per list: [C levels 5..KC][LLR levels 6..KS][level-5 staging, L rows of 33 words]; per warp:
    // the lists, then 16 words of list-step scratch
    p.list_words = (int)(scl_smem_llr_words(p.KS, L) + scl_smem_c_words(p.KC, L)) + L * kSclStage;
    p.list_words = (p.list_words + 3) & ~3;
    p.warp_words = lists * p.list_words + 16;
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
// List width of a CA-SCL launch: two frames per warp (half-warp lists) for L <= 8 in the global
// layout with a single code.
inline bool scl_two_lists(int L, bool all_smem) { return L <= 8 && !all_smem; }
// global workspace of the SCL list arrays (one slot per resident list: up to kSclWarpsPerSM lists
// per SM)
inline size_t scl_scratch_bytes(int N, int L)
{
    const long long w = std::max(scl_plan(N, L, false).slot_words, scl_plan(N, L, false, 2).slot_words);
    return (size_t)scl_sm_count() * kSclWarpsPerSM * (size_t)w * 4;
}

// 5-bit pointer of upper level k (5 <= k <= 12) in a path's two pointer words: levels 1..6 in word
// 0, levels 7..12 in word 1
__device__ __forceinline__ uint32_t fld(const uint32_t (&w)[2], int k)
{
    return (k <= 6 ? w[0] >> (5 * (k - 1)) : w[1] >> (5 * (k - 7))) & 31u;
}
__device__ __forceinline__ void set_fld(uint32_t (&w)[2], int k, uint32_t v)
{
    const int s = 5 * (k <= 6 ? k - 1 : k - 7);
    if (k <= 6)
        w[0] = (w[0] & ~(31u << s)) | (v << s);
    else
        w[1] = (w[1] & ~(31u << s)) | (v << s);
}
static_assert(kMaxN <= 4096, "upper-level pointers of levels up to 12");

// Lanes of one list: the whole warp (W = 32, one frame per warp) or one half of it (W = 16, two
// frames per warp, lists of at most 8 paths).  Path p of the list sits in lane base + p.  Every
// collective below is executed by all 32 lanes; with W = 16 the two halves compute their own
// results (shuffle offsets below 16 stay within a half).
template <int W>
struct Lanes {
    int lane, pl, base;
    __device__ __forceinline__ Lanes() : lane(threadIdx.x & 31), pl(lane & (W - 1)), base(lane & ~(W - 1)) {}
    __device__ __forceinline__ uint32_t ballot(bool p) const
    {
        const uint32_t b = __ballot_sync(0xffffffffu, p);
        return W == 32 ? b : (b >> base) & 0xffffu;
    }
    template <class V>
    __device__ __forceinline__ V shfl(V v, int p) const { return __shfl_sync(0xffffffffu, v, base + p); }
    // Reductions over the list: one redux.sync for a whole-warp list; for half-warp lists one per
    // half, each lane feeding the other half's reduction the identity, and keeping its own half's.
    __device__ __forceinline__ uint32_t red_or(uint32_t v) const
    {
        if constexpr (W == 32) {
            return __reduce_or_sync(0xffffffffu, v);
        } else {
            const uint32_t lo = __reduce_or_sync(0xffffffffu, base ? 0u : v);
            const uint32_t hi = __reduce_or_sync(0xffffffffu, base ? v : 0u);
            return base ? hi : lo;
        }
    }
    __device__ __forceinline__ uint32_t red_xor(uint32_t v) const
    {
        if constexpr (W == 32) {
            return __reduce_xor_sync(0xffffffffu, v);
        } else {
            const uint32_t lo = __reduce_xor_sync(0xffffffffu, base ? 0u : v);
            const uint32_t hi = __reduce_xor_sync(0xffffffffu, base ? v : 0u);
            return base ? hi : lo;
        }
    }
    __device__ __forceinline__ uint32_t red_max(uint32_t v) const
    {
        if constexpr (W == 32) {
            return __reduce_max_sync(0xffffffffu, v);
        } else {
            const uint32_t lo = __reduce_max_sync(0xffffffffu, base ? 0u : v);
            const uint32_t hi = __reduce_max_sync(0xffffffffu, base ? v : 0u);
            return base ? hi : lo;
        }
    }
    __device__ __forceinline__ uint32_t red_min(uint32_t v) const
    {
        if constexpr (W == 32) {
            return __reduce_min_sync(0xffffffffu, v);
        } else {
            const uint32_t lo = __reduce_min_sync(0xffffffffu, base ? 0xffffffffu : v);
            const uint32_t hi = __reduce_min_sync(0xffffffffu, base ? v : 0xffffffffu);
            return base ? hi : lo;
        }
    }
    __device__ __forceinline__ uint32_t match_any(uint32_t v) const
    {
        const uint32_t m = __match_any_sync(0xffffffffu, W == 32 ? v : v | ((uint32_t)base << 8));
        return W == 32 ? m : (m >> base) & 0xffffu;
    }
    // the larger of the two lists' values (W = 16), for loop bounds every lane must share
    __device__ __forceinline__ int both_max(int v) const
    {
        return W == 32 ? v : max(v, __shfl_xor_sync(0xffffffffu, v, 16));
    }
};

// A path about to rewrite level k that it shares takes a free array of that level (lane = path;
// `act` active paths; the lowest lane of each group of sharers keeps its array).  A list without
// sharing is left unchanged, so the call is safe for a list that does not need it.
template <int W>
__device__ __forceinline__ void scl_own(uint32_t (&w)[2], int k, int act, int L)
{
    const Lanes<W> sg;
    const bool on = sg.pl < act;
    const uint32_t mine = on ? fld(w, k) : 64u + sg.pl;
    const uint32_t same = sg.match_any(mine);
    const uint32_t below = (1u << sg.pl) - 1u;
    const bool need = on && (same & below) != 0u;
    const uint32_t used = sg.red_or(on ? (1u << mine) : 0u);
    uint32_t freem = ~used & (L >= 32 ? 0xffffffffu : ((1u << L) - 1u));
    const int r = __popc(sg.ballot(need) & below);
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

// The partial-sum step with the bit index r at run time (warp-uniform): kc = trailing ones of r
// levels fold in predicated steps, no jump (measured faster than dispatching leaf_psum<R> by a
// switch on r; the LLR step keeps the switch, which measured faster than its runtime form).
__device__ __forceinline__ uint32_t leaf_psum_rt(Leaf& f, uint32_t bitv, int r)
{
    if (!(r & 1)) {  // even bits (half of them): the bit itself is the level-0 partial sum
        f.c[0] = bitv;
        return bitv;
    }
    if (!(r & 2)) {  // bits 1 mod 4 (a quarter): one fold into level 1
        const uint32_t v1 = ((bitv ^ f.c[0]) & 0x1u) | ((bitv & 0x1u) << 1);
        f.c[1] = v1;
        return v1;
    }
    const int kc = __ffs(~r) - 1;
    uint32_t v = bitv;
    if (kc > 0) v = ((v ^ f.c[0]) & 0x1u) | ((v & 0x1u) << 1);
    if (kc > 1) v = ((v ^ f.c[1]) & 0x3u) | ((v & 0x3u) << 2);
    if (kc > 2) v = ((v ^ f.c[2]) & 0xFu) | ((v & 0xFu) << 4);
    if (kc > 3) v = ((v ^ f.c[3]) & 0xFFu) | ((v & 0xFFu) << 8);
    if (kc > 4) v = ((v ^ f.c[4]) & 0xFFFFu) | ((v & 0xFFFFu) << 16);
    if (kc == 0) f.c[0] = v;
    if (kc == 1) f.c[1] = v;
    if (kc == 2) f.c[2] = v;
    if (kc == 3) f.c[3] = v;
    if (kc == 4) f.c[4] = v;
    return v;
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

// List step of a half-warp list (W = 16, L <= 8, at most 16 candidates, one per lane): the same
// survivors as scl_list_step, computed with loop bounds shared by both halves -- the fast path is
// taken only when both lists qualify, and the ranks count over all 2L candidate slots with the
// unused ones at +inf.  Returns the survivor's parent path (within the list).
__device__ __forceinline__ int scl_list_step_half(float lam, float& pm, int& act, int L, uint8_t* selc,
                                                  uint32_t& bitv, bool& dup, bool& moved)
{
    const Lanes<16> sg;
    const int pl = sg.pl;
    const bool on = pl < act;
    const uint32_t hd_max = sg.red_max(on ? __float_as_uint(pm) : 0u);
    const uint32_t pen_min = sg.red_min(on ? __float_as_uint(__fadd_rn(pm, fabsf(lam))) : 0xffffffffu);
    const bool fast = act == L && hd_max < pen_min;
    if (__all_sync(0xffffffffu, fast || act == 0)) {
        bitv = lam < 0.0f ? 1u : 0u;
        dup = false;
        moved = false;
        return pl;
    }
    const int nc = 2 * act;
    const float inf = __int_as_float(0x7f800000);
    float cm0;
    {
        const float lp = sg.shfl(lam, (pl >> 1) & 15);
        const float pp = sg.shfl(pm, (pl >> 1) & 15);
        cm0 = ((uint32_t)(pl & 1) != (uint32_t)(lp < 0.0f)) ? __fadd_rn(pp, fabsf(lp)) : pp;
        if (pl >= nc) cm0 = inf;
    }
    int rank0 = 0;
    for (int c2 = 0; c2 < 2 * L; ++c2) {
        const float o = sg.shfl(cm0, c2);
        rank0 += (o < cm0) || (o == cm0 && c2 < pl);
    }
    const uint32_t below = (1u << pl) - 1u;
    const uint32_t km0 = sg.ballot(pl < nc && (nc <= L || rank0 < L));
    uint8_t* sel = selc + sg.base;
    if (km0 & (1u << pl)) sel[__popc(km0 & below)] = (uint8_t)pl;
    dup = (km0 & (km0 >> 1) & 0x55555555u) != 0u;
    const int nact = __popc(km0);
    __syncwarp();
    const int cq = pl < nact ? sel[pl] : 0;
    __syncwarp();
    const float m0 = sg.shfl(cm0, cq & 15);
    bitv = (uint32_t)(cq & 1);
    pm = pl < nact ? m0 : 0.0f;
    act = nact;
    moved = __any_sync(0xffffffffu, pl < nact && (cq >> 1) != pl);
    return cq >> 1;
}

// Decode one frame per list: the warp's frame (W = 32), or each half-warp's frame (W = 16; a
// half without a frame passes frame < 0 and decodes nothing).  TWO: L = 32, two candidates per
// lane.  MW: every warp of the CTA calls with the same frame; warp 0 holds the list and runs the
// bit loop, and all warps share the element-parallel upper-level updates (their path pointers
// and path count passed through `ptab`, 104 shared words), with CTA barriers around each level.
template <bool TWO, int W, bool MW = false>
__device__ void scl_decode_frame(const SCLArgs& a, const DevCode& C, int frame, const SCLWarp& S, uint8_t* selc,
                                 uint32_t* ptab = nullptr)
{
    static_assert(W == 32 || !TWO, "half-warp lists hold at most 8 paths");
    static_assert(!MW || W == 32, "the multi-warp form takes whole-warp lists");
    const bool lead = !MW || threadIdx.x < 32;
    const Lanes<W> sg;
    const int lane = sg.pl;  // path of this lane within its list
    const int N = C.N, n = C.n, L = a.L;
    const float* y = a.llr + (frame < 0 ? 0 : (a.llr_off ? a.llr_off[frame] : (long long)frame * N));
    uint32_t pA[2] = {0u, 0u}, pC[2] = {0u, 0u};  // upper-level pointer rows of path `lane`
    float pm = 0.0f;
    // CRC syndrome of the path's decided bits so far: XOR of the syndrome columns of the positions
    // decided 1 (frozen positions have column 0); survivors inherit their parent's
    uint32_t syn = 0u;
    int act = frame < 0 ? 0 : 1;
    uint32_t shA = 0u, shC = 0u;  // upper levels that may be shared since the last duplication
    Leaf lf;
#pragma unroll
    for (int k = 0; k < 5; ++k) lf.c[k] = 0u;
    const int nblocks = N >> 5;
    for (int blk = 0; blk < nblocks; ++blk) {
        // ------------------------------------------------ upper levels on entering the block
        const int t = blk == 0 ? n : 5 + __ffs(blk) - 1;
        const int top = blk == 0 ? n - 1 : t;
        const int act_both = sg.both_max(act);
        for (int k = top; k >= 5; --k) {
            // level 5 goes to the staging rows (indexed by path), levels >= 6 to their arrays
            const bool stage = k == 5;
            if (lead && !stage && __any_sync(0xffffffffu, (shA >> k) & 1u)) {
                scl_own<W>(pA, k, act, L);
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
            int nact = act, nact_both = act_both;
            if constexpr (MW) {
                if (lead) {
                    ptab[lane] = my_d;
                    ptab[32 + lane] = my_s;
                    ptab[64 + lane] = my_c;
                    if (lane == 0) ptab[96] = (uint32_t)act;
                }
                __syncthreads();
                nact = nact_both = (int)ptab[96];
            }
            const int cwk = scl_cs(k), total = nact << k, tmax = nact_both << k;
            // element stride of a round: the list's lanes, or every thread of the CTA
            const int TW = MW ? (int)blockDim.x : W, tix = MW ? (int)threadIdx.x : lane;
            // kSclUpRound elements per lane per round: all loads of a round are issued before any
            // store, so the L2 latency of the upper levels (global for long lists) is paid once per
            // round; the leaf registers are dead here and hold the round's values.  The loads are
            // unconditional (an element past the list's end reads a valid slot: its path index is
            // below L and its offset below len), so nothing but the stores is predicated and the
            // rounds' independent chains interleave.
            // CH: the level reads the channel row, whose values are staged as CA-SCL reads them
            auto rounds = [&](auto USE_G, auto FROM_CH) {
                constexpr bool G = decltype(USE_G)::value, CH = decltype(FROM_CH)::value;
                constexpr int U = kSclUpRound;
                for (int e0 = 0; e0 < tmax; e0 += U * TW) {
                    float va[U], vb[U];
                    uint32_t vw[U], pdv[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int e = e0 + TW * q + tix;
                        const int p = (e >> k) & (W - 1);
                        pdv[q] = MW ? ptab[p] : sg.shfl(my_d, p);
                        const uint32_t ps = MW ? ptab[32 + p] : sg.shfl(my_s, p);
                        const int j = e & (len - 1);
                        const float* src = srcb + ps * (2 * len);
                        va[q] = src[j];
                        vb[q] = src[j + len];
                        if constexpr (CH) {
                            va[q] = scl_stage(va[q]);
                            vb[q] = scl_stage(vb[q]);
                        }
                        if constexpr (G) vw[q] = cbk[(MW ? ptab[64 + p] : sg.shfl(my_c, p)) * cwk + (j >> 5)];
                    }
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int e = e0 + TW * q + tix;
                        const int j = e & (len - 1);
                        float r;
                        if constexpr (G)
                            r = scl_g(va[q], vb[q], (vw[q] >> (j & 31)) & 1u);
                        else
                            r = xmin(va[q], vb[q]);
                        if (e < total) dst[pdv[q] * dstride + j] = r;
                    }
                }
            };
            if (from_ch) {
                if (use_g)
                    rounds(std::true_type{}, std::true_type{});
                else
                    rounds(std::false_type{}, std::true_type{});
            } else if (use_g) {
                rounds(std::true_type{}, std::false_type{});
            } else {
                rounds(std::false_type{}, std::false_type{});
            }
            if constexpr (MW)
                __syncthreads();
            else
                __syncwarp();
        }
        if (!lead) continue;  // the helper warps only share the upper levels
        // level 5 of every path into its lane's registers (lanes past the list read row 0: the
        // staging area has L rows); the lower leaf levels and partial sums start afresh (every bit
        // of the block writes them before reading them), which also tells the compiler that their
        // registers were free during the upper-level rounds above
        {
            const float* row = S.stage + (lane < L ? lane : 0) * kSclStage;
#pragma unroll
            for (int j = 0; j < 32; ++j) lf.l5[j] = row[j];
#pragma unroll
            for (int j = 0; j < 16; ++j) lf.l4[j] = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) lf.l3[j] = 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) lf.l2[j] = 0.0f;
            lf.l1[0] = lf.l1[1] = 0.0f;
#pragma unroll
            for (int k = 0; k < 5; ++k) lf.c[k] = 0u;
        }
        // ------------------------------------------------ the 32 bits of the block
        // A runtime loop: one copy of the list step serves all 32 bits, and only the per-bit leaf
        // code (whose register indices are compile-time constants) is dispatched by the bit index.
        // Unrolling the block with a list step inlined per bit overflowed the instruction cache.
        const uint32_t fw = C.frozen_bits[blk], dw = C.decided_bits[blk];
        uint32_t v5 = 0u;
#pragma unroll 1
        for (int r = 0; r < 32; ++r) {
            const uint32_t col = C.colsyn[blk * 32 + r];
            float lam = 0.0f;
            if (r & 1) {
                // odd bits (half of them): one g from level 1, no dispatch
                lam = scl_g(lf.l1[0], lf.l1[1], lf.c[0] & 1u);
            } else if ((r & 3) == 2) {
                // bits 2 mod 4 (a quarter): g into level 1, then f
                leaf_g<2>(lf.l2, lf.l1, lf.c[1]);
                lam = xmin(lf.l1[0], lf.l1[1]);
            } else if ((r & 7) == 4) {
                // bits 4 mod 8 (an eighth): g into level 2, then f twice
                leaf_g<4>(lf.l3, lf.l2, lf.c[2]);
                leaf_f<2>(lf.l2, lf.l1);
                lam = xmin(lf.l1[0], lf.l1[1]);
            } else {
                switch (r) {
#define SCL_LEAF_LLR(R) \
    case 8 * (R): lam = leaf_llr<8 * (R)>(lf); break;
                    SCL_LEAF_LLR(0) SCL_LEAF_LLR(1) SCL_LEAF_LLR(2) SCL_LEAF_LLR(3)
#undef SCL_LEAF_LLR
                }
            }
            uint32_t bitv = 0u;
            bool moved = false;
            int parent = lane;
            if ((fw >> r) & 1u) {
                if (lane < act && lam < 0.0f) pm = __fadd_rn(pm, fabsf(lam));
            } else if ((dw >> r) & 1u) {
                // decision aiding: each path takes its hard decision, no branching, no metric
                bitv = lam < 0.0f ? 1u : 0u;
            } else {
                bool dup = false;
                if constexpr (W == 32)
                    parent = scl_list_step<TWO>(lam, pm, act, L, selc, bitv, dup, moved);
                else
                    parent = scl_list_step_half(lam, pm, act, L, selc, bitv, dup, moved);
                if (moved) {
                    const int src = sg.base + parent;
                    leaf_inherit_rt(lf, src, leaf_live_mask(r));
                    pA[0] = __shfl_sync(0xffffffffu, pA[0], src);
                    pA[1] = __shfl_sync(0xffffffffu, pA[1], src);
                    pC[0] = __shfl_sync(0xffffffffu, pC[0], src);
                    pC[1] = __shfl_sync(0xffffffffu, pC[1], src);
                    syn = __shfl_sync(0xffffffffu, syn, src);
                }
                if (dup) shA = shC = 0xffffffffu;
            }
            if (bitv) syn ^= col;
            v5 = leaf_psum_rt(lf, bitv, r);
        }
        // ------------------------------------------------ block complete: partial sums upward
        {
            const int i_last = blk * 32 + 31;
            const int kc = __ffs(~i_last) - 1;  // >= 5; n after the last block
            if (__any_sync(0xffffffffu, (shC >> kc) & 1u)) {
                scl_own<W>(pC, kc, act, L);
                shC &= ~(1u << kc);
            }
            uint32_t* dstl = S.Cl(kc);
            const int cwk = scl_cs(kc);
            if (lane < act) dstl[fld(pC, kc) * cwk] = v5;
            __syncwarp();
            const uint32_t my_dst = fld(pC, kc);
            const int act_both2 = sg.both_max(act);
            for (int k = 5; k < kc; ++k) {
                const int Wk = 1 << (k - 5), total = act * Wk, tmax = act_both2 * Wk;
                const uint32_t* ckb = S.Cl(k);
                const uint32_t my_k = fld(pC, k);
                if constexpr (W == 32) {
                    // four elements per lane and round, loads first and unconditional (an element
                    // past the list reads a word of a valid array), stores predicated
                    constexpr int UC = 4;
                    for (int e0 = 0; e0 < tmax; e0 += UC * W) {
                        uint32_t xv[UC], cv[UC], pdv[UC];
#pragma unroll
                        for (int q = 0; q < UC; ++q) {
                            const int e = e0 + W * q + lane;
                            const int p = (e >> (k - 5)) & (W - 1);
                            const int w = e & (Wk - 1);
                            pdv[q] = sg.shfl(my_dst, p);
                            xv[q] = dstl[pdv[q] * cwk + w];
                            cv[q] = ckb[sg.shfl(my_k, p) * scl_cs(k) + w];
                        }
#pragma unroll
                        for (int q = 0; q < UC; ++q) {
                            const int e = e0 + W * q + lane;
                            if (e < total) {
                                uint32_t* dst = dstl + pdv[q] * cwk;
                                const int w = e & (Wk - 1);
                                dst[Wk + w] = xv[q];
                                dst[w] = xv[q] ^ cv[q];
                            }
                        }
                    }
                } else {
                    // half-warp lists: one element per lane (the unrolled form measured slower
                    // with 2^16 frames, the two lists' registers)
                    for (int e0 = 0; e0 < tmax; e0 += W) {
                        const int e = e0 + lane;
                        const int p = (e >> (k - 5)) & (W - 1);
                        const uint32_t pd = sg.shfl(my_dst, p);
                        const uint32_t pk = sg.shfl(my_k, p);
                        if (e < total) {
                            const int w = e & (Wk - 1);
                            uint32_t* dst = dstl + pd * cwk;
                            const uint32_t x = dst[w];
                            dst[Wk + w] = x;
                            dst[w] = x ^ ckb[pk * scl_cs(k) + w];
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    if (!lead) return;
    // ------------------------------------------------------------------ CRC selection
    // Each path's syndrome was accumulated bit by bit; the chosen path's codeword (level-n array)
    // is turned into u = x G in place for the output.  The list's lanes hold the codeword's 32-bit
    // words lane + W h.
    constexpr int H = kMaxWords / W;  // words per lane
    const int words = N >> 5;
    uint32_t* xl = S.Cl(n);
    const uint32_t my_x = fld(pC, n);
    const uint32_t synd = lane < act ? syn : 0xffffffffu;  // lane p: syndrome of path p
    __syncwarp();
    // first CRC-passing path in (metric, index) order, else the best metric
    const bool ok_lane = lane < act && synd == 0u;
    const bool any_ok = sg.ballot(ok_lane) != 0u;
    const bool cand = any_ok ? ok_lane : lane < act;
    float key = cand ? pm : __int_as_float(0x7f800000);
    int who = cand ? lane : 64;
#pragma unroll
    for (int off = W / 2; off >= 1; off >>= 1) {
        const float ok2 = __shfl_xor_sync(0xffffffffu, key, off);
        const int ow = __shfl_xor_sync(0xffffffffu, who, off);
        if (ok2 < key || (ok2 == key && ow < who)) {
            key = ok2;
            who = ow;
        }
    }
    uint32_t* uw = xl + sg.shfl(my_x, who & (W - 1)) * scl_cs(n);
    {
        const bool live = frame >= 0;
        uint32_t w[H];
#pragma unroll
        for (int h = 0; h < H; ++h) w[h] = (live && lane + W * h < words) ? uw[lane + W * h] : 0u;
        const uint32_t m[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int e = 0; e < 5; ++e) w[h] ^= (w[h] >> (1 << e)) & m[e];
        for (int D = 1; D < W && D < words; D <<= 1) {
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, w[h], D);
                if (!(lane & D)) w[h] ^= o;
            }
        }
        for (int D = W; D < words; D <<= 1) {
            const int hd = D / W;
#pragma unroll
            for (int h = 0; h < H; ++h)
                if (!(h & hd) && (h | hd) < H) w[h] ^= w[h | hd];
        }
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (live && lane + W * h < words) uw[lane + W * h] = w[h];
        __syncwarp();
    }
    if (frame >= 0) {
        uint8_t* out = a.bits + (size_t)frame * a.row_bytes;
        for (int by = lane; by < a.row_bytes; by += W) {
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
    }
    __syncwarp();
}

// Decode `frame` (frame < 0: nothing, on this lane's list) by the calling warp with code `code_id`
// of a mixed batch (-1: the batch's single code): plan of the code, the list's shared words `ws`
// and global slot `slot` (null: every level in shared memory).  A list without a frame still walks
// the code's structure with no path, so both lists of a warp must be given the same code.
template <bool TWO, int W, bool MW = false>
__device__ __forceinline__ void scl_warp_frame(const SCLArgs& a, int frame, int code_id, uint32_t* ws, float* slot,
                                               uint8_t* selc, uint32_t* ptab = nullptr)
{
    constexpr int LISTS = 32 / W;
    const int L = a.L;
    const DevCode& C = code_id >= 0 ? *a.codes[code_id] : *a.code;
    SCLWarp S;
    S.L = L;
    if (a.code_of) {
        const SCLPlan p = scl_plan(C.N, L, slot == nullptr, LISTS);
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
    scl_decode_frame<TWO, W, MW>(a, C, frame, S, selc, ptab);
}

// W = 32: one frame per warp; W = 16: two (one per half-warp list), claimed together.  In a mixed
// batch (frames sorted by code) the two frames of a pair normally share their code; a pair whose
// codes differ is decoded one list after the other.
template <bool TWO, int W>
__global__ void __launch_bounds__(kSclWarpsPerCTA * 32) scl_kernel(const SCLArgs a)
{
    constexpr int LISTS = 32 / W;
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int li = lane / W;  // this lane's list
    uint32_t* wsw = smem + (size_t)wid * a.warp_words;
    uint32_t* ws = wsw + li * a.list_words;
    uint8_t* selc = reinterpret_cast<uint8_t*>(wsw + a.warp_words - 16);
    float* slot = a.scratch
        ? a.scratch + (((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * LISTS + li) * (size_t)a.slot_words
        : nullptr;
    const int count = a.count ? *a.count : a.B;
    if constexpr (W == 32) {
        // Few frames (at most one per CTA, single code): each CTA takes one frame at a time and
        // all its warps share the frame's upper-level updates (the words of warp 1, unused here,
        // hold the shared path pointers), which shortens the frame's decoding latency.
        if (!a.code_of && count <= (int)gridDim.x && blockDim.x >= 64) {
            uint32_t* ptab = smem + a.warp_words;
            // warp 0's list words, list-step scratch and global slot serve the CTA's frame
            float* slot0 = a.scratch ? a.scratch + (size_t)blockIdx.x * (blockDim.x >> 5) * (size_t)a.slot_words : nullptr;
            uint8_t* selc0 = reinterpret_cast<uint8_t*>(smem + a.warp_words - 16);
            for (;;) {
                if (threadIdx.x == 0) ptab[100] = (uint32_t)atomicAdd(a.next, 1);
                __syncthreads();
                const int idx = (int)ptab[100];
                __syncthreads();
                if (idx >= count) break;  // uniform over the CTA
                scl_warp_frame<TWO, W, true>(a, a.list ? a.list[idx] : idx, -1, smem, slot0, selc0, ptab);
                __syncthreads();
            }
            return;
        }
    }
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.next, LISTS);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;  // uniform over the warp
        const int k = idx + li;
        const int frame = k < count ? (a.list ? a.list[k] : k) : -1;
        if (!a.code_of) {
            scl_warp_frame<TWO, W>(a, frame, -1, ws, slot, selc);
            continue;
        }
        const int cf = frame >= 0 ? a.code_of[frame] : -1;
        if constexpr (LISTS == 2) {
            const int c0 = __shfl_sync(0xffffffffu, cf, 0), c1 = __shfl_sync(0xffffffffu, cf, 16);
            if (c0 >= 0 && c1 >= 0 && c0 != c1) {
                scl_warp_frame<TWO, W>(a, li == 0 ? frame : -1, c0, ws, slot, selc);
                scl_warp_frame<TWO, W>(a, li == 1 ? frame : -1, c1, ws, slot, selc);
            } else {
                scl_warp_frame<TWO, W>(a, frame, c0 >= 0 ? c0 : c1, ws, slot, selc);
            }
        } else {
            scl_warp_frame<TWO, W>(a, frame, cf, ws, slot, selc);
        }
    }
}

// Persistent launch: as many CTAs as fit on the device (bounded by the global slots and, when it
// is known on the host, by the work); returns cudaSuccess or the launch error.
cudaError_t scl_launch(SCLArgs a, int N, int L, cudaStream_t st, int warp_words_max, long long slot_words_max)
{
    const bool all_smem = a.scratch == nullptr;
    const int lists = scl_two_lists(L, all_smem) ? 2 : 1;
    const SCLPlan p = scl_plan(N, L, all_smem, lists);
    a.KS = p.KS;
    a.KC = p.KC;
    a.list_words = std::max(p.list_words, warp_words_max - 16);
    a.warp_words = lists * a.list_words + 16;
    a.slot_words = std::max(p.slot_words, slot_words_max);
    int W = kSclWarpsPerCTA;
    const size_t wb = (size_t)a.warp_words * 4;
    while (W > 1 && (size_t)W * wb > 200 * 1024) W >>= 1;
    const size_t smem = (size_t)W * wb;
    const bool two = L > 16;
    const void* fn = lists == 2 ? (const void*)scl_kernel<false, 16>
                                : (two ? (const void*)scl_kernel<true, 32> : (const void*)scl_kernel<false, 32>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, W * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int sms = scl_sm_count();
    long long grid = (long long)sms * per_sm;
    if (!all_smem) grid = std::min<long long>(grid, (long long)sms * kSclWarpsPerSM / (W * lists));
    if (!a.list) {
        // known work: whole-warp lists with at most one frame per CTA of the full grid get a CTA
        // per frame (its warps then share each frame's upper levels), otherwise no idle CTAs
        const long long need = (a.B + W * lists - 1) / (W * lists);
        grid = (lists == 1 && W > 1 && !a.code_of && a.B <= grid) ? std::max(a.B, 1) : std::min(grid, need);
    }
    if (grid < 1) grid = 1;
    if (lists == 2)
        scl_kernel<false, 16><<<(unsigned)grid, W * 32, smem, st>>>(a);
    else if (two)
        scl_kernel<true, 32><<<(unsigned)grid, W * 32, smem, st>>>(a);
    else
        scl_kernel<false, 32><<<(unsigned)grid, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

#endif  // POLAR_SCL_KERNELS

}  // namespace polar
