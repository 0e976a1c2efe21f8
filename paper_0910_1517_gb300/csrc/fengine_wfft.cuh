// fengine_wfft.cuh -- the F-engine for n_chan <= 1024 (n_fft <= 2048): warp-specialised, one
// warp per FFT group, two radix-32 passes; included by fengine.cu after fengine_impl.cuh.
//
// Same work and outputs as the kernel of fengine_impl.cuh (Sec. 2.1 FX chain, Eq. 2 phasor,
// Sec. 2.2 beams), organised to cut instructions and shared-memory traffic and to keep both
// halves of the work in flight at once:
//   * a CTA owns F = 8192 / M consecutive frames and walks over every input (the beams need
//     every antenna of a frame in one CTA);
//   * warps 0-7 (the FFT group, 104 registers a thread) transform the frames of input it:
//     the M-point complex FFT of a frame (z[n] = x[2n] + i x[2n+1], M = 32 P) is a four-step
//     FFT inside one warp -- lane l takes column n = l + 32 m of each of the warp's G = 32 / P
//     frames, P-point DFTs in registers straight from the int8 staging buffer, the twiddle
//     W_M^(l k1), one transpose through the warp's own shared-memory region (__syncwarp), then
//     lane (g, k1) a 32-point DFT in registers: Z[k1 + P k2] -- and leave the results in the
//     region in natural order;
//   * warps 8-15 (the epilogue group, 152 registers a thread) meanwhile take input it - 1: each
//     thread owns 8 frames of two channel pairs (k, M - k) for the real split, the Eq. 2 phasor,
//     the beams (accumulated in its registers over all inputs) and the K-block stores;
//   * the regions, the antenna tables and the staging buffer are double-buffered; mbarriers
//     hand a region set from the FFT group to the epilogue group (full) and back (empty).
//     Every wait is bounded: on a timeout the error word is set, the CTA's abort flag stops
//     both groups, and the copies still in flight are waited for before the CTA exits.
#pragma once

#include "fengine_impl.cuh"

namespace gbx {
namespace {

constexpr int kWThreads = 512;
constexpr int kWFftWarps = 8;                  // warps 0-7: FFT group (warpgroups 0, 1)
constexpr int kWEpiThreads = 256;              // warps 8-15: epilogue group (warpgroups 2, 3)
constexpr int kWRegFft = 104, kWRegEpi = 152;  // 256 x 104 + 256 x 152 = 512 x 128 registers

template <int M>
struct WPlan {
    static_assert(M >= 32 && M <= 1024 && (M & (M - 1)) == 0, "32 <= M <= 1024, a power of two");
    static constexpr int P = M / 32;               // pass-1 points per lane and frame
    static constexpr int G = 32 / P;               // frames per FFT warp
    static constexpr int F = kWFftWarps * G;       // frames per CTA (8192 / M)
    static constexpr int N = 2 * M;                // real FFT size
    static constexpr int S = 33 * P;               // float2 stride of a frame in a warp region
    static constexpr int RS = 34;                  // float2 per transpose row (16-byte aligned rows)
    static constexpr int REG = 32 * RS;            // float2 per warp region
    static constexpr int STAGE = F * N + 32;       // staging bytes per buffer
    static constexpr int L = 8;                    // frames per epilogue thread
    static constexpr int SLOTS = M / 4;            // pair slots per frame group (two pairs each)
    static constexpr int NFG = kWEpiThreads / SLOTS;   // frame groups
    static_assert(NFG * L == F && G * S <= REG && STAGE % 16 == 0, "plan");
};

template <int M>
struct WSmem {
    using P = WPlan<M>;
    static constexpr int kTw1 = P::P * 32;         // inter-pass twiddles [k1 / 2][l][k1 % 2]
    static constexpr int kTwN = M / 2 + 1;         // real-split twiddles
    static constexpr int kTab = 2 * M + P::F;      // [pf M | wcoh M | ff F] of one antenna
    static constexpr size_t stage = 0;
    static constexpr size_t X = stage + 2 * static_cast<size_t>(P::STAGE);
    static constexpr size_t tw = X + 2 * sizeof(float2) * kWFftWarps * P::REG;
    static constexpr size_t tab = ((tw + sizeof(float2) * (kTw1 + kTwN) + 127) / 128) * 128;
    static constexpr size_t total = tab + 2 * sizeof(float2) * kTab;
    static_assert(total <= 232448 - 1024, "F-engine shared memory exceeds 227 KB");
    static_assert(X % 16 == 0 && tab % 16 == 0 && (sizeof(float2) * kTab) % 16 == 0, "bulk-copy targets");
};

struct WCtl {
    uint64_t bar[2];           // staging buffer b landed
    uint64_t tbar[2];          // antenna tables b landed
    uint64_t full[2];          // region set b transformed (FFT warps -> epilogue)
    uint64_t empty[2];         // region set b and tables b consumed (epilogue warps -> FFT group)
    int abort_flag;
    int Ds[kMaxAnt];
};

template <int N_REG>
__device__ __forceinline__ void reg_dealloc() { asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N_REG)); }
template <int N_REG>
__device__ __forceinline__ void reg_alloc() { asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N_REG)); }

template <int M, int MODE>
__global__ void __launch_bounds__(kWThreads, 1) fengine_w_kernel(const FeParams p) {
#include "fengine_wfft_body.cuh"
}

// One member of a batch: the parameters are read from the batch's device table when the kernel
// runs, so that a captured graph takes new sample pointers and frame counters on every replay.
template <int M, int MODE>
__global__ void __launch_bounds__(kWThreads, 1) fengine_w_tab_kernel(const FeBatch* __restrict__ batch, int sub) {
    __shared__ FeParams ps;
    if (threadIdx.x == 0) ps = batch->p[sub];
    __syncthreads();
    const FeParams& p = ps;
#include "fengine_wfft_body.cuh"
}

// the register split (setmaxnreg) hands the FFT group's registers to the epilogue group: it
// needs exactly the 512 x 128 registers of the launch, or the epilogue warps would wait for
// registers that never come
template <typename K>
cudaError_t w_launch_ok(K kern) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.numRegs * kWThreads != kWRegFft * kWFftWarps * 32 + kWRegEpi * kWEpiThreads) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

template <int M, int MODE>
cudaError_t launch_w(const FeParams& p, cudaStream_t s) {
    using P = WPlan<M>;
    const size_t smem = WSmem<M>::total;
    cudaError_t e = w_launch_ok(fengine_w_kernel<M, MODE>);   // refuse a launch with the wrong register count
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fengine_w_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (p.n_int + P::F - 1) / P::F;
    fengine_w_kernel<M, MODE><<<grid, kWThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_w_mode(const FeParams& p, cudaStream_t s) {
    if constexpr (MODE == OUT_F32Q || MODE == OUT_I8B) {   // n_chan 32 .. 1024 only
        switch (p.n_chan) {
            case 32: return launch_w<32, MODE>(p, s);
            case 64: return launch_w<64, MODE>(p, s);
            case 128: return launch_w<128, MODE>(p, s);
            case 256: return launch_w<256, MODE>(p, s);
            case 512: return launch_w<512, MODE>(p, s);
            case 1024: return launch_w<1024, MODE>(p, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (p.n_chan) {
        case 32: return launch_w<32, MODE>(p, s);
        case 64: return launch_w<64, MODE>(p, s);
        case 128: return launch_w<128, MODE>(p, s);
        case 256: return launch_w<256, MODE>(p, s);
        case 512: return launch_w<512, MODE>(p, s);
        case 1024: return launch_w<1024, MODE>(p, s);
        case 2048: return launch_t<2048, MODE>(p, s);   // 4-frame CTAs: the kernel of fengine_impl.cuh
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace gbx
