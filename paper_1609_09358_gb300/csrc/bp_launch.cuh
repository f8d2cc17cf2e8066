// bp_launch.cuh -- per-length BP kernel selection, compiled once per message type
// (bp_launch_fp32.cu, bp_launch_fp16.cu).
#pragma once

#include "bp_kernel.cuh"

namespace polar {

struct BPKernelInfo {
    const void* fn;
    int threads;
    size_t smem;
    int groups_per_cta;  // frame groups (frames, or frame pairs for half2) per CTA
};

// kernel of (log2 N, weighted) for the message type of this translation unit (weighted: 0 plain,
// 1 learned scales, 2 learned scales within [-1, 1] with both frames of a half2 register on the
// same iteration -- FP32 takes the form-1 kernel for 2); plain kernels come in a variant for
// crc_len <= 16 that packs the CRC syndrome into 16-bit halves (half2: both frames' syndromes in
// one word; FP32: the columns of two nodes in one word)
BPKernelInfo bp_kernel_info_fp32(int logn, int weighted, bool packed_syndrome);
// FP32 unweighted kernel of a BP variant: bit 0 exact PE function, bit 1 re-encoding stop
BPKernelInfo bp_kernel_info_fp32_var(int logn, int var);
BPKernelInfo bp_kernel_info_fp16(int logn, int weighted, bool packed_syndrome);
// natural-layout learned weights [iters][2][n][N] -> the prepared layout of the length's plan
cudaError_t wms_prepare_fp32(int logn, const float* w, int iters, void* out, cudaStream_t st);
cudaError_t wms_prepare_fp16(int logn, const float* w, int iters, void* out, cudaStream_t st);

template <class E>
cudaError_t wms_prepare_t(int logn, const float* w, int iters, void* out, cudaStream_t st)
{
    auto go = [&](auto LOGN_C) -> cudaError_t {
        constexpr int LOGN = decltype(LOGN_C)::value;
        using P = typename BPConfig<LOGN>::Plan;
        const size_t total = (size_t)iters * 2 * P::LOGN * P::N;
        if (total == 0) return cudaSuccess;
        const unsigned grid = (unsigned)((total + 255) / 256);
        wms_prepare_kernel<P, E><<<grid, 256, 0, st>>>(w, iters, static_cast<E*>(out));
        return cudaGetLastError();
    };
    switch (logn) {
        case 7: return go(std::integral_constant<int, 7>{});
        case 8: return go(std::integral_constant<int, 8>{});
        case 9: return go(std::integral_constant<int, 9>{});
        case 10: return go(std::integral_constant<int, 10>{});
        default: return go(std::integral_constant<int, 11>{});
    }
}

template <class MSG>
BPKernelInfo bp_kernel_info_t(int logn, int weighted, bool packed_syndrome = false)
{
    auto pick = [&](auto LOGN_C) -> BPKernelInfo {
        constexpr int LOGN = decltype(LOGN_C)::value;
        using Cfg = BPConfig<LOGN>;
        using P = typename Cfg::Plan;
        constexpr int TH = Cfg::F * P::T;
        const size_t smem = (size_t)Cfg::F * bp_slot_words<P>() * 4;
        const void* fn;
        // the plain kernels' own plan
        using KP = BPKernelPlan<LOGN, 0, 0, MsgTraits<MSG>::FPT>;
        using P0 = typename KP::Plan;
        constexpr int TH0 = KP::F * P0::T;
        const size_t smem0 = (size_t)KP::F * bp_slot_words<P0>() * 4;
        if (weighted) {
            // learned weights: N <= 2048 (no weighted kernel is built for longer codes)
            if constexpr (LOGN > 11)
                return BPKernelInfo{nullptr, TH, smem, Cfg::F};
            else if constexpr (std::is_same<MSG, __half2>::value)
                return BPKernelInfo{weighted == 2 ? (const void*)bp_kernel<LOGN, MSG, 2, TH>
                                                  : (const void*)bp_kernel<LOGN, MSG, 1, TH>,
                                    TH, smem, Cfg::F};
            else
                return BPKernelInfo{(const void*)bp_kernel<LOGN, MSG, 1, TH>, TH, smem, Cfg::F};
        }
        fn = packed_syndrome ? (const void*)bp_kernel<LOGN, MSG, 0, TH0, true>
                             : (const void*)bp_kernel<LOGN, MSG, 0, TH0>;
        return {fn, TH0, smem0, KP::F};
    };
    switch (logn) {
        case 7: return pick(std::integral_constant<int, 7>{});
        case 8: return pick(std::integral_constant<int, 8>{});
        case 9: return pick(std::integral_constant<int, 9>{});
        case 10: return pick(std::integral_constant<int, 10>{});
        case 11: return pick(std::integral_constant<int, 11>{});
        default: return pick(std::integral_constant<int, 12>{});
    }
}

template <int VAR>
BPKernelInfo bp_kernel_info_var_t(int logn)
{
    auto pick = [&](auto LOGN_C) -> BPKernelInfo {
        constexpr int LOGN = decltype(LOGN_C)::value;
        using KP = BPKernelPlan<LOGN, 0, VAR, 1>;
        using P = typename KP::Plan;
        constexpr int TH = KP::F * P::T;
        const size_t smem = (size_t)KP::F * bp_slot_words<P>() * 4;
        return {(const void*)bp_kernel<LOGN, float, 0, TH, false, VAR>, TH, smem, KP::F};
    };
    switch (logn) {
        case 7: return pick(std::integral_constant<int, 7>{});
        case 8: return pick(std::integral_constant<int, 8>{});
        case 9: return pick(std::integral_constant<int, 9>{});
        case 10: return pick(std::integral_constant<int, 10>{});
        case 11: return pick(std::integral_constant<int, 11>{});
        default: return pick(std::integral_constant<int, 12>{});
    }
}

}  // namespace polar
