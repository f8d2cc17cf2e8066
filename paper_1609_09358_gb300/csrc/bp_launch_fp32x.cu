// bp_launch_fp32x.cu -- translation unit of the FP32 BP kernels with the exact PE function and/or
// the re-encoding stop (Sec. II-B), compiled apart from the min-sum kernels.
#include "bp_launch.cuh"
namespace polar {
BPKernelInfo bp_kernel_info_fp32_var(int logn, int var)
{
    switch (var) {
        case 1: return bp_kernel_info_var_t<1>(logn);
        case 2: return bp_kernel_info_var_t<2>(logn);
        default: return bp_kernel_info_var_t<3>(logn);
    }
}
}  // namespace polar
