// bp_launch_fp16.cu -- translation unit of the half2 BP kernels.
#include "bp_launch.cuh"
namespace polar {
BPKernelInfo bp_kernel_info_fp16(int logn, int weighted, bool packed_syndrome)
{
    return bp_kernel_info_t<__half2>(logn, weighted, packed_syndrome);
}
cudaError_t wms_prepare_fp16(int logn, const float* w, int iters, void* out, cudaStream_t st)
{
    return wms_prepare_t<__half>(logn, w, iters, out, st);
}
}  // namespace polar
