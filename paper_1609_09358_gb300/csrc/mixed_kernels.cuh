// mixed_kernels.cuh -- one persistent BP launch over frames of several codes (block lengths
// 128..2048 and rates mixed in one batch), plus the bucketing of frames by code.
//
// Frames are bucketed by code on the device (count, scan, scatter), so nothing in a mixed decode
// waits for the host and the whole sequence can be captured in a CUDA graph.  The BP launch is a
// persistent grid of CTAs of BLOCK threads.  A CTA works on one code at a time: it splits into
// BLOCK / T frame groups of that code's plan (T threads each), and every group pulls frames from
// the code's queue until it is empty; then the CTA moves to the next code.  CTA b starts at code
// b mod ncodes, so the codes are worked on in parallel and drained queues are skipped.  Each code
// has a plan variant (the register-blocking factor b of its BP plan, hence T and the number of
// frames per CTA), chosen on the host by the autotuner.
#pragma once

#include "bp_kernel.cuh"

namespace polar {

constexpr int kMixMaxCodes = 32;
constexpr int kMixBlock = 256;

// plan variants: id -> (log2 N, b)
//   0: (7,2)  1: (8,3)  2: (8,2)  3: (9,3)  4: (9,2)  5: (10,3)  6: (11,3)  7: (10,2)
constexpr int kMixVariants = 8;
__host__ __device__ inline int mix_variant_logn(int v)
{
    return v == 0 ? 7 : v <= 2 ? 8 : v <= 4 ? 9 : v == 5 || v == 7 ? 10 : 11;
}
__host__ __device__ inline int mix_variant_logr(int v) { return (v == 0 || v == 2 || v == 4 || v == 7) ? 2 : 3; }

struct MixedArgs {
    BPArgs base;                 // llr + llr_off, outputs (fixed row stride), limits, fail list
    const DevCode* code[kMixMaxCodes];
    int variant[kMixMaxCodes];
    int ncodes;
    const int* order;            // frames bucketed by code
    const int* start;            // [ncodes + 1] bucket starts
    int* qnext;                  // [ncodes] queue counters, zero before the launch
};

template <class P>
__host__ __device__ constexpr int mix_cta_words()
{
    return (kMixBlock / P::T) * bp_slot_words<P>();
}

// Defined in mixed_launch.cu: the kernel of a precision, and the bucketing by code.
const void* bp_mixed_fn(int precision, bool packed_syndrome);
cudaError_t mix_bucketing(const int* code_of, int B, int ncodes, int* counts, int* start, int* cursor, int* order,
                          cudaStream_t st);
// the first *count entries of list (frame indices, *count <= cap) sorted into `sorted` by the rank
// of their code (rank.r[code]: a permutation of 0 .. ncodes-1)
struct MixRank {
    int r[kMixMaxCodes];
};
cudaError_t mix_sort_list(const int* list, const int* count, int cap, const int* code_of, int ncodes, MixRank rank,
                          int* counts, int* start, int* cursor, int* sorted, cudaStream_t st);

inline size_t mix_smem_bytes(int variant)
{
    switch (variant) {
        case 0: return 4 * (size_t)mix_cta_words<BPPlan<7, 2>>();
        case 1: return 4 * (size_t)mix_cta_words<BPPlan<8, 3>>();
        case 2: return 4 * (size_t)mix_cta_words<BPPlan<8, 2>>();
        case 3: return 4 * (size_t)mix_cta_words<BPPlan<9, 3>>();
        case 4: return 4 * (size_t)mix_cta_words<BPPlan<9, 2>>();
        case 5: return 4 * (size_t)mix_cta_words<BPPlan<10, 3>>();
        case 7: return 4 * (size_t)mix_cta_words<BPPlan<10, 2>>();
        default: return 4 * (size_t)mix_cta_words<BPPlan<11, 3>>();
    }
}

#ifdef POLAR_MIXED_KERNELS
template <class P, class MSG, bool SYNP>
__device__ __forceinline__ void mix_run(const MixedArgs& m, int c, uint32_t* smem)
{
    constexpr int G = kMixBlock / P::T;  // frame groups in the CTA
    const int slot = threadIdx.x / P::T, t = threadIdx.x % P::T;
    QueueSource src{m.order + m.start[c], m.start[c + 1] - m.start[c], m.qnext + c};
    bp_run_group<P, MSG, false, (G > 1), QueueSource, SYNP>(m.base, *m.code[c], slot, t,
                                                            smem + slot * bp_slot_words<P>(), src);
}

// Two resident CTAs per SM (the register cap costs a few bytes of spill); the half2 kernel whose
// codes have CRCs of at most 16 bits keeps both frames' syndromes in one word (SYNP)
template <class MSG, bool SYNP>
__global__ void __launch_bounds__(kMixBlock, (std::is_same<MSG, float>::value || SYNP) ? 2 : 1)
    bp_mixed_kernel(const MixedArgs m)
{
    extern __shared__ uint32_t smem[];
    for (int k = 0; k < m.ncodes; ++k) {
        const int c = (blockIdx.x + k) % m.ncodes;
        // Every thread enters (control flow stays uniform over the CTA: a group's threads must all
        // reach its barriers); a group whose first fetch finds the queue empty returns at once.
        switch (m.variant[c]) {
            case 0: mix_run<BPPlan<7, 2>, MSG, SYNP>(m, c, smem); break;
            case 1: mix_run<BPPlan<8, 3>, MSG, SYNP>(m, c, smem); break;
            case 2: mix_run<BPPlan<8, 2>, MSG, SYNP>(m, c, smem); break;
            case 3: mix_run<BPPlan<9, 3>, MSG, SYNP>(m, c, smem); break;
            case 4: mix_run<BPPlan<9, 2>, MSG, SYNP>(m, c, smem); break;
            case 5: mix_run<BPPlan<10, 3>, MSG, SYNP>(m, c, smem); break;
            case 7: mix_run<BPPlan<10, 2>, MSG, SYNP>(m, c, smem); break;
            default: mix_run<BPPlan<11, 3>, MSG, SYNP>(m, c, smem); break;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ bucketing by code
// counts[c] = number of frames of code c; start = exclusive scan; order = frames by code.
// A frame whose code id is outside [0, ncodes) is left out of every bucket (not decoded).
__global__ void mix_count_kernel(const int* __restrict__ code_of, int B, int ncodes, int* counts)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        const int c = code_of[b];
        if (c >= 0 && c < ncodes) atomicAdd(&counts[c], 1);
    }
}

__global__ void mix_scan_kernel(const int* counts, int ncodes, int* start, int* cursor)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < ncodes; ++c) {
            start[c] = acc;
            cursor[c] = acc;
            acc += counts[c];
        }
        start[ncodes] = acc;
    }
}

__global__ void mix_scatter_kernel(const int* __restrict__ code_of, int B, int ncodes, int* cursor, int* order)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        const int c = code_of[b];
        if (c >= 0 && c < ncodes) order[atomicAdd(&cursor[c], 1)] = b;
    }
}

// The same three steps over the entries of a list (the frames CA-SCL decodes).
__global__ void mix_count_list_kernel(const int* __restrict__ list, const int* count, const int* __restrict__ code_of,
                                      int ncodes, MixRank rank, int* counts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *count) {
        const int c = code_of[list[i]];
        if (c >= 0 && c < ncodes) atomicAdd(&counts[rank.r[c]], 1);
    }
}
__global__ void mix_scatter_list_kernel(const int* __restrict__ list, const int* count, const int* __restrict__ code_of,
                                        int ncodes, MixRank rank, int* cursor, int* sorted)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < *count) {
        const int f = list[i];
        const int c = code_of[f];
        if (c >= 0 && c < ncodes) sorted[atomicAdd(&cursor[rank.r[c]], 1)] = f;
    }
}

#endif  // POLAR_MIXED_KERNELS

}  // namespace polar
