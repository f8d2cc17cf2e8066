// encode_kernels.cuh -- CRC + polar encoder (Sec. II, x = u G) and the seeded workload
// generator (payload bits and BPSK-AWGN channel LLRs from Philox4x32-10).
#pragma once

#include "polar_common.cuh"

namespace polar {

// One warp per frame.  Lane l owns the 32-bit words l + 32 h (h < kMaxWords / 32) of the N-bit
// vectors.
// CRC: XOR of the syndrome columns x^(K-1-k) mod g of the payload bits set (k < P), which is the
// remainder of payload(x) x^c; its bits go to the last c information positions, MSB first.
// Transform: the Fig. 1 butterflies x_j ^= x_{j+d} (bit log2 d of j clear) -- in-word with shifts
// for d < 32, across words with shuffles for 32 <= d < 1024 and within the lane for d >= 1024.
__global__ void encode_kernel(const DevCode* __restrict__ code, const uint8_t* __restrict__ payload,
                              int B, int pay_bytes, uint8_t* __restrict__ codeword)
{
    const int lane = threadIdx.x & 31;
    const int frame = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (frame >= B) return;
    const DevCode& C = *code;
    const int N = C.N, P = C.P, c = C.c, K = C.K, words = N >> 5;
    const uint8_t* pay = payload + (size_t)frame * pay_bytes;
    uint32_t crc = 0;
    for (int p = lane; p < P; p += 32)
        if ((pay[p >> 3] >> (p & 7)) & 1) crc ^= C.colsyn[C.info_idx[p]];
    crc = __reduce_xor_sync(0xffffffffu, crc);
    constexpr int H = kMaxWords / 32;
    uint32_t w[H];
#pragma unroll
    for (int h = 0; h < H; ++h) w[h] = 0u;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int wi = lane + 32 * h;
        if (wi >= words) break;
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            const int j = wi * 32 + b;
            if (frozen_at(C.frozen_bits, j)) continue;
            const int p = C.paypos[j];
            uint32_t bit;
            if (p >= 0) {
                bit = (pay[p >> 3] >> (p & 7)) & 1u;
            } else {
                // CRC node: its information index k >= P, CRC bit k - P, MSB first
                int k = P;
                while (C.info_idx[k] != j) ++k;
                bit = (crc >> (c - 1 - (k - P))) & 1u;
            }
            v |= bit << b;
        }
        w[h] = v;
    }
    (void)K;
    const uint32_t m[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
        for (int e = 0; e < 5; ++e) w[h] ^= (w[h] >> (1 << e)) & m[e];
    for (int D = 1; D < 32 && D < words; D <<= 1) {
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const uint32_t other = __shfl_xor_sync(0xffffffffu, w[h], D);
            if (!(lane & D)) w[h] ^= other;
        }
    }
#pragma unroll
    for (int hd = 1; hd < H; hd <<= 1)
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (!(h & hd) && 32 * (h | hd) < words) w[h] ^= w[h | hd];
    uint8_t* out = codeword + (size_t)frame * (N >> 3);
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int wi = lane + 32 * h;
        if (wi < words) reinterpret_cast<uint32_t*>(out)[wi] = w[h];
    }
}

// ------------------------------------------------------------------------------ Philox4x32-10
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// One thread per Philox block (128 payload bits) of one frame.
__global__ void random_payload_kernel(int B, int P, uint64_t seed, uint64_t frame0, uint8_t* __restrict__ out)
{
    const int nwords = (P + 31) >> 5, nblocks = (nwords + 3) >> 2, bytes = (P + 7) >> 3;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)B * nblocks) return;
    const int b = (int)(gid / nblocks), blk = (int)(gid % nblocks);
    const uint64_t f = frame0 + (uint64_t)b;
    const U4 r = philox4x32_10(U4{(uint32_t)blk, (uint32_t)f, 0u, (uint32_t)(f >> 32)}, (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
    uint8_t* row = out + (size_t)b * bytes;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int word = blk * 4 + q;
#pragma unroll
        for (int by = 0; by < 4; ++by) {
            const int byte = word * 4 + by;
            if (byte >= bytes) continue;
            uint8_t v = (uint8_t)(wv[q] >> (8 * by));
            const int valid = P - byte * 8;  // clear the pad bits of the last byte
            if (valid < 8) v &= (uint8_t)((1u << valid) - 1u);
            row[byte] = v;
        }
    }
}

// One thread per Philox block (4 nodes) of one frame: Box-Muller on (w0, w1) and (w2, w3).
__global__ void awgn_llr_kernel(const uint8_t* __restrict__ codeword, int B, int N, float sigma_all,
                                const float* __restrict__ sigmas, uint64_t seed, uint64_t frame0,
                                float* __restrict__ llr)
{
    const int nblocks = N >> 2;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)B * nblocks) return;
    const int b = (int)(gid / nblocks), blk = (int)(gid % nblocks);
    const float sigma = sigmas ? sigmas[b] : sigma_all;
    const uint64_t f = frame0 + (uint64_t)b;
    const U4 r = philox4x32_10(U4{(uint32_t)blk, (uint32_t)f, 1u, (uint32_t)(f >> 32)}, (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    const float scale = 2.0f / (sigma * sigma);
    const uint32_t e[2] = {r.x, r.z}, o[2] = {r.y, r.w};
    const uint8_t xb = codeword[(size_t)b * (N >> 3) + (blk >> 1)] >> ((blk & 1) * 4);
    float4 v;
    float* vp = &v.x;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float u1 = (float)((e[p] >> 8) + 1u) * (1.0f / 16777216.0f);
        const float u2 = (float)(o[p] >> 8) * (1.0f / 16777216.0f);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        const float z[2] = {rad * cs, rad * sn};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int i = 2 * p + q;
            const float s = ((xb >> i) & 1) ? -1.0f : 1.0f;
            vp[i] = scale * (s + sigma * z[q]);
        }
    }
    reinterpret_cast<float4*>(llr + (size_t)b * N)[blk] = v;
}

}  // namespace polar
