// fengine_sub.cu -- F-engine launches of the members of a batch (corr_batch_*): the kernels of the
// single-integration launches (fengine.cu), in variants that read their parameters from the
// batch's device table when they run.  A graph captured once then serves every replay, each
// with new sample pointers and frame counters written into the table by a copy node of the same
// graph.  A translation unit of its own, so that these instantiations compile beside fengine.cu.
#include "fengine_wfft.cuh"

namespace gbx {
namespace {

template <int M, int MODE>
cudaError_t launch_w_sub(const FeBatch* tab, int sub, int n_int, cudaStream_t s) {
    using P = WPlan<M>;
    const size_t smem = WSmem<M>::total;
    cudaError_t e = w_launch_ok(fengine_w_tab_kernel<M, MODE>);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fengine_w_tab_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (n_int + P::F - 1) / P::F;
    fengine_w_tab_kernel<M, MODE><<<grid, kWThreads, smem, s>>>(tab, sub);
    return cudaGetLastError();
}

// n_fft = 4096: 4-frame CTAs, in 2-CTA clusters where the output is fp16 (Epi::kPair)
template <int MODE>
cudaError_t launch_t_sub(const FeBatch* tab, int sub, int n_int, cudaStream_t s) {
    constexpr int M = 2048;
    using P = Plan<M>;
    const size_t smem = Smem<M>::total;
    cudaError_t e = cudaFuncSetAttribute(fengine_tab_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (n_int + P::F - 1) / P::F;
    if constexpr (Epi<M, MODE>::kPair) {
        if (grid % 2) return cudaErrorInvalidValue;   // n_int is a multiple of 16: whole pairs
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, fengine_tab_kernel<M, MODE>, tab, sub);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    fengine_tab_kernel<M, MODE><<<grid, kThreads, smem, s>>>(tab, sub);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_sub_w(const FeBatch* tab, int sub, int n_chan, int n_int, cudaStream_t s) {
    switch (n_chan) {
        case 32: return launch_w_sub<32, MODE>(tab, sub, n_int, s);
        case 64: return launch_w_sub<64, MODE>(tab, sub, n_int, s);
        case 128: return launch_w_sub<128, MODE>(tab, sub, n_int, s);
        case 256: return launch_w_sub<256, MODE>(tab, sub, n_int, s);
        case 512: return launch_w_sub<512, MODE>(tab, sub, n_int, s);
        case 1024: return launch_w_sub<1024, MODE>(tab, sub, n_int, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fengine_sub(const FeBatch* tab, int sub, int n_chan, int n_int, int mode, cudaStream_t s) {
    if (!tab || sub < 0 || sub >= kMaxSub) return cudaErrorInvalidValue;
    if (n_chan == 2048) {
        switch (mode) {
            case OUT_FP32: return launch_t_sub<OUT_FP32>(tab, sub, n_int, s);
            case OUT_I8: return launch_t_sub<OUT_I8>(tab, sub, n_int, s);
            case OUT_F16: return launch_t_sub<OUT_F16>(tab, sub, n_int, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case OUT_FP32: return launch_sub_w<OUT_FP32>(tab, sub, n_chan, n_int, s);
        case OUT_F16: return launch_sub_w<OUT_F16>(tab, sub, n_chan, n_int, s);
        case OUT_I8B: return launch_sub_w<OUT_I8B>(tab, sub, n_chan, n_int, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbx
