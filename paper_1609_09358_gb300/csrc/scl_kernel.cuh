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
// Lazy copy: every level k keeps L physical LLR arrays and L physical partial-sum arrays; a path
// holds one pointer per level.  A surviving child copies only its parent's pointer row.  Since a
// level is always rewritten whole, a path that is about to write a level it shares takes a free
// array of that level instead (the lowest-numbered sharer keeps the old one): no LLR or
// partial-sum data is ever copied.  A level is checked only if a list step duplicated a path since
// it was last written.
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
    float* scratch;    // per-warp LLR arrays when they do not fit shared memory
    int row_bytes;
};

__host__ __device__ inline int scl_cw(int k) { return k < 5 ? 1 : 1 << (k - 5); }  // words of a level-k C array
__host__ __device__ inline int scl_coff(int k, int L)  // word offset of level k's C arrays
{
    int s = 0;
    for (int q = 0; q < k; ++q) s += scl_cw(q);
    return s * L;
}
__host__ __device__ inline int scl_aoff(int k, int L) { return L * ((1 << k) - 2); }  // float offset, k >= 1

// per-warp shared memory: C arrays (levels 0..n) | pointer rows A and C [n+1][32] | candidate
// slots [64] | LLR arrays (levels 1..n-1) when resident
__host__ __device__ inline int scl_small_words(int n, int L) { return scl_coff(n + 1, L) + (2 * (n + 1) * 32 + 64) / 4; }
inline size_t scl_llr_bytes(int N, int L) { return (size_t)L * (N - 2) * sizeof(float); }
inline int log2_host(int v)
{
    int n = 0;
    while ((1 << n) < v) ++n;
    return n;
}
inline bool scl_fits_smem(int N, int L) { return scl_llr_bytes(N, L) <= 72 * 1024; }
inline size_t scl_warp_smem_bytes(int N, int L)
{
    size_t b = (size_t)scl_small_words(log2_host(N), L) * 4;
    b = (b + 15) / 16 * 16;
    if (scl_fits_smem(N, L)) b += scl_llr_bytes(N, L);
    return b;
}
constexpr int kSclGlobalWarpsPerSM = 8;
inline int scl_sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}
inline size_t scl_resident_warps(int N, int L) { return (size_t)scl_sm_count() * kSclGlobalWarpsPerSM; }
inline size_t scl_global_warp_bytes(int N, int L) { return scl_llr_bytes(N, L); }

// A path about to rewrite level row[] that it shares takes a free array of that level.  Lanes
// are paths; `active` paths.  The lowest lane of each group of sharers keeps its array.
__device__ __forceinline__ void scl_own(uint8_t* row, int active, int L)
{
    const int lane = threadIdx.x & 31;
    const bool act = lane < active;
    const int mine = act ? row[lane] : 64 + lane;
    const uint32_t same = __match_any_sync(0xffffffffu, mine);
    const bool need = act && (same & ((1u << lane) - 1u)) != 0u;
    const uint32_t used = __reduce_or_sync(0xffffffffu, act ? (1u << mine) : 0u);
    const uint32_t all = L >= 32 ? 0xffffffffu : ((1u << L) - 1u);
    uint32_t freem = ~used & all;
    const uint32_t needm = __ballot_sync(0xffffffffu, need);
    const int r = __popc(needm & ((1u << lane) - 1u));
    if (need) {
        for (int q = 0; q < r; ++q) freem &= freem - 1u;  // drop the r lowest free arrays
        row[lane] = (uint8_t)(__ffs(freem) - 1);
    }
    __syncwarp();
}

__device__ __forceinline__ float scl_g(float a, float b, uint32_t v) { return v ? __fsub_rn(b, a) : __fadd_rn(b, a); }

__device__ void scl_decode_frame(const SCLArgs& a, const DevCode& C, int frame, uint32_t* cb, uint8_t* ptrA,
                                 uint8_t* ptrC, uint8_t* selc, float* A)
{
    const int lane = threadIdx.x & 31;
    const int N = C.N, n = C.n, L = a.L;
    const float* y = a.llr + (size_t)frame * N;
    for (int k = 0; k <= n; ++k) {
        ptrA[k * 32 + lane] = 0;
        ptrC[k * 32 + lane] = 0;
    }
    __syncwarp();
    float pm = 0.0f, lam = 0.0f;
    int act = 1;
    uint32_t shA = 0u, shC = 0u;  // levels that may be shared since the last duplication
    for (int i = 0; i < N; ++i) {
        const int t = i == 0 ? n : __ffs(i) - 1;
        const int top = i == 0 ? n - 1 : t;
        for (int k = top; k >= 1; --k) {
            if ((shA >> k) & 1u) {
                scl_own(ptrA + k * 32, act, L);
                shA &= ~(1u << k);
            }
            const bool use_g = i != 0 && k == t;
            const int len = 1 << k;
            float* dstbase = A + scl_aoff(k, L);
            for (int e = lane; e < (act << k); e += 32) {
                const int p = e >> k, j = e & (len - 1);
                const float* src = (k + 1 == n) ? y : A + scl_aoff(k + 1, L) + ptrA[(k + 1) * 32 + p] * (2 * len);
                const float va = src[j], vb = src[j + len];
                float r;
                if (use_g) {
                    const uint32_t w = cb[scl_coff(k, L) + ptrC[k * 32 + p] * scl_cw(k) + (j >> 5)];
                    r = scl_g(va, vb, (w >> (j & 31)) & 1u);
                } else {
                    r = xmin(va, vb);
                }
                dstbase[ptrA[k * 32 + p] * len + j] = r;
            }
            __syncwarp();
        }
        // bit LLR (level 0), lane = path
        if (lane < act) {
            const float* src = A + scl_aoff(1, L) + ptrA[32 + lane] * 2;
            const float va = src[0], vb = src[1];
            if (i != 0 && t == 0)
                lam = scl_g(va, vb, cb[scl_coff(0, L) + ptrC[lane]] & 1u);
            else
                lam = xmin(va, vb);
        }
        uint32_t bitv = 0u;
        if (frozen_at(C.frozen_bits, i)) {
            if (lane < act && lam < 0.0f) pm = __fadd_rn(pm, fabsf(lam));
        } else {
            // ---------------------------------------------------------------- list step
            const int nc = 2 * act;
            const int cpl = nc > 32 ? 2 : 1;  // candidates per lane
            float cm[2];
            bool valid[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                const float lp = __shfl_sync(0xffffffffu, lam, (c >> 1) & 31);
                const float pp = __shfl_sync(0xffffffffu, pm, (c >> 1) & 31);
                valid[h] = h < cpl && c < nc;
                const uint32_t b = c & 1;
                cm[h] = (b != (uint32_t)(lp < 0.0f)) ? __fadd_rn(pp, fabsf(lp)) : pp;
            }
            int rank[2] = {0, 0};
            for (int c2 = 0; c2 < nc; ++c2) {
                const float o = __shfl_sync(0xffffffffu, c2 < 32 ? cm[0] : cm[1], c2 & 31);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h;
                    rank[h] += (o < cm[h]) || (o == cm[h] && c2 < c);
                }
            }
            const uint32_t km0 = __ballot_sync(0xffffffffu, valid[0] && rank[0] < L);
            const uint32_t km1 = __ballot_sync(0xffffffffu, valid[1] && rank[1] < L);
            const uint32_t below = (1u << lane) - 1u;
            if (km0 & (1u << lane)) selc[__popc(km0 & below)] = (uint8_t)lane;
            if (km1 & (1u << lane)) selc[__popc(km0) + __popc(km1 & below)] = (uint8_t)(lane + 32);
            const bool dup = ((km0 & (km0 >> 1) & 0x55555555u) | (km1 & (km1 >> 1) & 0x55555555u)) != 0u;
            const int nact = __popc(km0) + __popc(km1);
            __syncwarp();
            int cq = 0;
            if (lane < nact) cq = selc[lane];
            const float m0 = __shfl_sync(0xffffffffu, cm[0], cq & 31);
            const float m1 = __shfl_sync(0xffffffffu, cm[1], cq & 31);
            const int parent = cq >> 1;
            bitv = (uint32_t)(cq & 1);
            // pointer rows of the survivors: copies of their parents' rows
            uint8_t ra[12], rc[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                if (k <= n && lane < nact) {
                    ra[k] = ptrA[k * 32 + parent];
                    rc[k] = ptrC[k * 32 + parent];
                }
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                if (k <= n && lane < nact) {
                    ptrA[k * 32 + lane] = ra[k];
                    ptrC[k * 32 + lane] = rc[k];
                }
            }
            pm = lane < nact ? (cq < 32 ? m0 : m1) : 0.0f;
            act = nact;
            if (dup) shA = shC = 0xffffffffu;
            __syncwarp();
        }
        // -------------------------------------------------------------- partial sums
        const int kc = __ffs(~i) - 1;  // trailing ones of i; n after the last bit
        if ((shC >> kc) & 1u) {
            scl_own(ptrC + kc * 32, act, L);
            shC &= ~(1u << kc);
        }
        {
            // bottom five levels in one word per path (lane = path)
            uint32_t v = bitv;
            const int kw = kc < 5 ? kc : 5;
            if (lane < act) {
                for (int k = 0; k < kw; ++k) {
                    const uint32_t ck = cb[scl_coff(k, L) + ptrC[k * 32 + lane] * scl_cw(k)];
                    const uint32_t m = (1u << (1 << k)) - 1u;
                    v = ((v ^ ck) & m) | ((v & m) << (1 << k));
                }
                cb[scl_coff(kc, L) + ptrC[kc * 32 + lane] * scl_cw(kc)] = v;
            }
            __syncwarp();
            for (int k = 5; k < kc; ++k) {
                const int W = 1 << (k - 5);
                for (int e = lane; e < act * W; e += 32) {
                    const int p = e / W, w = e % W;
                    uint32_t* dst = cb + scl_coff(kc, L) + ptrC[kc * 32 + p] * scl_cw(kc);
                    const uint32_t ck = cb[scl_coff(k, L) + ptrC[k * 32 + p] * scl_cw(k) + w];
                    const uint32_t x = dst[w];
                    dst[W + w] = x;
                    dst[w] = x ^ ck;
                }
                __syncwarp();
            }
        }
    }
    // ------------------------------------------------------------------ CRC selection
    // u = x G on each path's N-bit codeword (level-n array), in place; syndrome of its
    // information bits
    const int words = N >> 5;
    uint32_t synd = 0xffffffffu;  // lane p: syndrome of path p
    for (int p = 0; p < act; ++p) {
        uint32_t* xw = cb + scl_coff(n, L) + ptrC[n * 32 + p] * scl_cw(n);
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
    const uint32_t* uw = cb + scl_coff(n, L) + ptrC[n * 32 + who] * scl_cw(n);
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

__global__ void __launch_bounds__(128) scl_kernel(const SCLArgs a, int llr_in_smem, int warp_words)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const DevCode& C = *a.code;
    const int N = C.N, n = C.n, L = a.L;
    uint32_t* cb = smem + (size_t)wid * warp_words;
    uint8_t* ptrA = reinterpret_cast<uint8_t*>(cb + scl_coff(n + 1, L));
    uint8_t* ptrC = ptrA + (n + 1) * 32;
    uint8_t* selc = ptrC + (n + 1) * 32;
    float* A;
    if (llr_in_smem) {
        A = reinterpret_cast<float*>(cb + ((scl_small_words(n, L) + 3) & ~3));
    } else {
        A = a.scratch + ((size_t)blockIdx.x * (blockDim.x >> 5) + wid) * (size_t)L * (N - 2);
    }
    const int count = a.count ? *a.count : a.B;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(a.next, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;
        const int frame = a.list ? a.list[idx] : idx;
        scl_decode_frame(a, C, frame, cb, ptrA, ptrC, selc, A);
    }
}

// Persistent launch: as many CTAs as fit on the device (bounded by the work when it is known on
// the host); returns cudaSuccess or the launch error.
inline cudaError_t scl_launch(const SCLArgs& a, int N, int L, cudaStream_t st)
{
    const bool in_smem = scl_fits_smem(N, L);
    const size_t wb = scl_warp_smem_bytes(N, L);
    int W = 4;
    while (W > 1 && (size_t)W * wb > 200 * 1024) W >>= 1;
    const size_t smem = (size_t)W * wb;
    cudaError_t e = cudaFuncSetAttribute(scl_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scl_kernel, W * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int sms = scl_sm_count();
    long long grid = (long long)sms * per_sm;
    if (!in_smem) grid = std::min<long long>(grid, (long long)sms * kSclGlobalWarpsPerSM / W);
    if (!a.list) grid = std::min<long long>(grid, (a.B + W - 1) / W);
    if (grid < 1) grid = 1;
    const int warp_words = (int)(wb / 4);
    scl_kernel<<<(unsigned)grid, W * 32, smem, st>>>(a, in_smem ? 1 : 0, warp_words);
    return cudaGetLastError();
}

}  // namespace polar
