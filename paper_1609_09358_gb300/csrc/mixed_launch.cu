// mixed_launch.cu -- translation unit of the mixed-batch BP kernel and the bucketing kernels
// (see mixed_kernels.cuh).
#define POLAR_MIXED_KERNELS
#include "mixed_kernels.cuh"

namespace polar {

const void* bp_mixed_fn(int precision, bool packed_syndrome)
{
    if (precision != POLAR_FP16) return (const void*)bp_mixed_kernel<float, false>;
    return packed_syndrome ? (const void*)bp_mixed_kernel<__half2, true> : (const void*)bp_mixed_kernel<__half2, false>;
}

cudaError_t mix_sort_list(const int* list, const int* count, int cap, const int* code_of, int ncodes, MixRank rank,
                          int* counts, int* start, int* cursor, int* sorted, cudaStream_t st)
{
    if (cap <= 0) return cudaSuccess;
    const int tb = 256, nb = (cap + tb - 1) / tb;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)ncodes, st);
    if (e != cudaSuccess) return e;
    mix_count_list_kernel<<<nb, tb, 0, st>>>(list, count, code_of, ncodes, rank, counts);
    mix_scan_kernel<<<1, 1, 0, st>>>(counts, ncodes, start, cursor);
    mix_scatter_list_kernel<<<nb, tb, 0, st>>>(list, count, code_of, ncodes, rank, cursor, sorted);
    return cudaGetLastError();
}

cudaError_t mix_bucketing(const int* code_of, int B, int ncodes, int* counts, int* start, int* cursor, int* order,
                          cudaStream_t st)
{
    const int tb = 256, nb = (B + tb - 1) / tb;
    mix_count_kernel<<<nb, tb, 0, st>>>(code_of, B, ncodes, counts);
    mix_scan_kernel<<<1, 1, 0, st>>>(counts, ncodes, start, cursor);
    mix_scatter_kernel<<<nb, tb, 0, st>>>(code_of, B, ncodes, cursor, order);
    return cudaGetLastError();
}

}  // namespace polar
