// pipe_rates.cu -- issue-rate microbenchmark of the instructions the BP roofline is built on
// (measurement only; not a step of the paper's method).
//
// Each thread runs kChains independent dependency chains of one instruction for `iters` rounds,
// so that with 32 warps per SM the pipe, not the latency, limits the rate.  Every CTA brackets its
// loop with clock64() after a barrier; all CTAs of the grid are resident at once (4 CTAs of 256
// threads per SM, few registers), so the SM-cycles of a CTA are cycles in which the SM runs all of
// its CTAs.  Rate = instructions (per lane, i.e. results of one lane; an f16x2 instruction counts
// once) completed on an SM / that SM's cycles = sum over the SM's CTAs of their instructions / the
// longest of their cycle counts.
#include <cstdint>
#include <vector>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "polar_gb300.h"

namespace polar {

constexpr int kChains = 8;
constexpr int kRateThreads = 256;
constexpr int kRateCtasPerSm = 4;

template <int OP>
__device__ __forceinline__ uint32_t rate_op(uint32_t x, uint32_t c)
{
    uint32_t d;
    if constexpr (OP == POLAR_RATE_MINXORSIGN_F32)
        asm volatile("min.xorsign.abs.f32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_MINXORSIGN_F16X2)
        asm volatile("min.xorsign.abs.f16x2 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_ADD_F32)
        asm volatile("add.rn.f32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_ADD_F16X2)
        asm volatile("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_MUL_F16X2)
        asm volatile("mul.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_MIN_F32)
        asm volatile("min.f32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(c));
    else if constexpr (OP == POLAR_RATE_EX2_F32)
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=r"(d) : "r"(x));
    else if constexpr (OP == POLAR_RATE_LG2_F32)
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=r"(d) : "r"(x));
    else if constexpr (OP == POLAR_RATE_PRMT)
        asm volatile("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(d) : "r"(x), "r"(c));
    else
        d = x;
    return d;
}

// `out[blockIdx.x]` = (instructions of the CTA, its SM cycles, its SM id)
template <int OP>
__global__ void __launch_bounds__(kRateThreads) pipe_rate_kernel(int iters, uint32_t seed, unsigned long long* out)
{
    uint32_t x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 0x3C003C00u ^ (seed + (uint32_t)(threadIdx.x * kChains + i));
    const uint32_t c = 0x3F800000u ^ (seed & 0xFFu);  // an ordinary value whatever the instruction's type
    __syncthreads();
    const long long t0 = clock64();
    for (int r = 0; r < iters; ++r) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = rate_op<OP>(x[i], c);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc ^= x[i];
    __syncthreads();
    const long long t1 = clock64();
    if (acc == 0x12345678u) out[3 * gridDim.x] = acc;  // keeps the chains live (never true in practice)
    if (threadIdx.x == 0) {
        uint32_t sm;
        asm("mov.u32 %0, %%smid;" : "=r"(sm));
        out[3 * blockIdx.x] = (unsigned long long)iters * kChains * blockDim.x;
        out[3 * blockIdx.x + 1] = (unsigned long long)(t1 - t0);
        out[3 * blockIdx.x + 2] = sm;
    }
}

using RateKernel = void (*)(int, uint32_t, unsigned long long*);

static RateKernel rate_kernel(int op)
{
    switch (op) {
        case POLAR_RATE_MINXORSIGN_F32: return pipe_rate_kernel<POLAR_RATE_MINXORSIGN_F32>;
        case POLAR_RATE_MINXORSIGN_F16X2: return pipe_rate_kernel<POLAR_RATE_MINXORSIGN_F16X2>;
        case POLAR_RATE_ADD_F32: return pipe_rate_kernel<POLAR_RATE_ADD_F32>;
        case POLAR_RATE_ADD_F16X2: return pipe_rate_kernel<POLAR_RATE_ADD_F16X2>;
        case POLAR_RATE_MUL_F16X2: return pipe_rate_kernel<POLAR_RATE_MUL_F16X2>;
        case POLAR_RATE_MIN_F32: return pipe_rate_kernel<POLAR_RATE_MIN_F32>;
        case POLAR_RATE_EX2_F32: return pipe_rate_kernel<POLAR_RATE_EX2_F32>;
        case POLAR_RATE_LG2_F32: return pipe_rate_kernel<POLAR_RATE_LG2_F32>;
        case POLAR_RATE_PRMT: return pipe_rate_kernel<POLAR_RATE_PRMT>;
        default: return nullptr;
    }
}

}  // namespace polar

extern "C" size_t polar_pipe_rate_scratch_bytes(void)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return (3 * (size_t)sms * polar::kRateCtasPerSm + 1) * sizeof(unsigned long long);
}

extern "C" int polar_pipe_rate(int32_t op, int32_t iters, void* scratch, size_t scratch_bytes, double* per_sm_clock,
                               void* stream)
{
    using namespace polar;
    const RateKernel k = rate_kernel(op);
    if (!k || iters < 1 || !per_sm_clock || !scratch) return POLAR_ERR_ARG;
    const size_t need = polar_pipe_rate_scratch_bytes();
    if (need == 0) return POLAR_ERR_CUDA;
    if (scratch_bytes < need) return POLAR_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = (int)((need / sizeof(unsigned long long) - 1) / 3);
    unsigned long long* d = static_cast<unsigned long long*>(scratch);
    std::vector<unsigned long long> h(need / sizeof(unsigned long long));
    k<<<grid, kRateThreads, 0, st>>>(iters, 0x9E3779B9u, d);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), d, need, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return POLAR_ERR_CUDA;
    // per SM (by %smid): instructions of its CTAs over the longest of their cycle counts; mean
    // over the SMs that ran CTAs
    unsigned long long max_sm = 0;
    for (int b = 0; b < grid; ++b) max_sm = h[3 * b + 2] > max_sm ? h[3 * b + 2] : max_sm;
    std::vector<unsigned long long> ops((size_t)max_sm + 1, 0ull), cyc((size_t)max_sm + 1, 0ull);
    for (int b = 0; b < grid; ++b) {
        const size_t sm = (size_t)h[3 * b + 2];
        ops[sm] += h[3 * b];
        cyc[sm] = h[3 * b + 1] > cyc[sm] ? h[3 * b + 1] : cyc[sm];
    }
    double rate_sum = 0.0;
    int used = 0;
    for (size_t sm = 0; sm <= (size_t)max_sm; ++sm)
        if (cyc[sm]) {
            rate_sum += (double)ops[sm] / (double)cyc[sm];
            ++used;
        }
    *per_sm_clock = used ? rate_sum / used : 0.0;
    return POLAR_OK;
}
