// scl_launch.cu -- translation unit of the CA-SCL kernels (see scl_kernel.cuh).
#define POLAR_SCL_KERNELS
#include "scl_kernel.cuh"
