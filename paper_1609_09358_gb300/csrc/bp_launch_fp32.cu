// bp_launch_fp32.cu -- translation unit of the FP32 BP kernels.
#include "bp_launch.cuh"
namespace polar {
BPKernelInfo bp_kernel_info_fp32(int logn, int weighted, bool packed_syndrome)
{
    return bp_kernel_info_t<float>(logn, weighted, packed_syndrome);
}
cudaError_t wms_prepare_fp32(int logn, const float* w, int iters, void* out, cudaStream_t st)
{
    return wms_prepare_t<float>(logn, w, iters, out, st);
}
}  // namespace polar
