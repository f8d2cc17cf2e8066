// bp_launch_fp16.cu -- translation unit of the half2 BP kernels.
#include "bp_launch.cuh"
namespace polar {
BPKernelInfo bp_kernel_info_fp16(int logn, bool weighted) { return bp_kernel_info_t<__half2>(logn, weighted); }
}  // namespace polar
