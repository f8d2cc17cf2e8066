// bp_launch_fp32.cu -- translation unit of the FP32 BP kernels.
#include "bp_launch.cuh"
namespace polar {
BPKernelInfo bp_kernel_info_fp32(int logn, bool weighted) { return bp_kernel_info_t<float>(logn, weighted); }
}  // namespace polar
