// multibeam.cu -- several phased-array beams with full-polar products or voltages (Sec. 2.2:
// the coherent beamformer also gives the voltage cross products for the Stokes parameters;
// Sec. 5: multiple phased beams covering different directions in the primary beam), from the
// F-engine's FP32 spectra:
//   U_bp[t][k] = sum_a w[k][b][a] Y_{a,p}[t][k]     (FP32 complex multiply-adds)
//   full polar (products 0): mean over `avg` frames of |U_b0|^2, |U_b1|^2, Re U_b0 conj U_b1,
//                            Im U_b0 conj U_b1
//   voltages   (products 1, avg 1): Re U_b0, Im U_b0, Re U_b1, Im U_b1
//
// One CTA takes channel k and max(64, avg) frames, staged 64 at a time: the FP32 K-blocks of a
// stage arrive by one bulk copy each (padded apart, so the 32 frames a warp reads hit distinct
// banks), the channel's weights [beam][antenna] by another (once).  Lanes are consecutive frames and
// warps beam groups (beams w, w + 8, ...), so every weight read is a broadcast and each sample
// is read once for all of a thread's beams.  A window of `avg` frames is summed by shuffles
// across its lanes (avg <= 32) and then across passes in registers, in a fixed order.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

constexpr int kMbThreads = 256;
constexpr int kMbWarps = kMbThreads / 32;
constexpr int kMbMaxBeams = 64;                 // beams per launch (kMbMaxBeams / kMbWarps per thread)
constexpr int kMbPad = 4;                       // floats between K-blocks in shared memory
constexpr int kMbFrames = 64;                   // frames per shared-memory stage

struct MbShared {
    uint64_t bar;
};

template <int BPT>   // beams per thread
__global__ void __launch_bounds__(kMbThreads) multibeam_kernel(const float* __restrict__ spec, int n_ant, int n_pol,
                                                               int n_chan, int n_int, const float2* __restrict__ w,
                                                               int wstride, int n_beams, int products, int avg,
                                                               float4* __restrict__ out, unsigned* err) {
    extern __shared__ __align__(16) float sm[];
    __shared__ MbShared ms;
    const int n_in = n_ant * n_pol;
    const int tb = tb_fp32(n_chan), Rp = rows_fp32(n_in);
    const int kb_per = kMbFrames / tb, blk = Rp * tb, pitch = blk + kMbPad;
    float2* ws = reinterpret_cast<float2*>(sm + kb_per * pitch);   // [beam][antenna] of channel k
    float4* acc = reinterpret_cast<float4*>(ws + wstride);          // per-beam window sums (avg > 32)
    const int fcta = avg > kMbFrames ? avg : kMbFrames;             // frames of this CTA
    const int k = blockIdx.x, t0 = blockIdx.y * fcta;
    const int64_t ntb = n_int / tb;
    if (threadIdx.x == 0) {
        mbar_init(&ms.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n_out = n_int / avg;
    bool ok = true;
    int last_sub = 0;
    for (int sub = 0; sub < fcta / kMbFrames && ok; ++sub) {
        last_sub = sub;
        const int ts = t0 + sub * kMbFrames;                        // first frame of this sub-chunk
        if (threadIdx.x == 0) {
            const uint32_t wbytes = sub == 0 ? static_cast<uint32_t>(wstride) * sizeof(float2) : 0u;
            mbar_arrive_expect_tx(&ms.bar, kb_per * blk * 4 + wbytes);
            for (int j = 0; j < kb_per; ++j)
                bulk_g2s(sm + j * pitch, spec + (static_cast<int64_t>(k) * ntb + ts / tb + j) * blk, blk * 4, &ms.bar);
            if (sub == 0) bulk_g2s(ws, w + static_cast<int64_t>(k) * wstride, wbytes, &ms.bar);
        }
        ok = __syncthreads_and(mbar_wait(&ms.bar, sub & 1, err, ERR_WAIT_STAGE));   // one decision for all
        for (int pass = 0; pass < kMbFrames / 32 && ok; ++pass) {
            const int f = pass * 32 + lane;                         // frame within the sub-chunk
            const float* kb = sm + (f / tb) * pitch;
            const int e = f % tb;
            float ur[BPT][2], ui[BPT][2];
#pragma unroll
            for (int q = 0; q < BPT; ++q) ur[q][0] = ur[q][1] = ui[q][0] = ui[q][1] = 0.0f;
            for (int a = 0; a < n_ant; ++a)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    if (p >= n_pol) break;
                    const int i = a * n_pol + p;
                    const float yr = kb[fp32_off(2 * i, e, tb)], yi = kb[fp32_off(2 * i + 1, e, tb)];
#pragma unroll
                    for (int q = 0; q < BPT; ++q) {
                        const int b = warp + q * kMbWarps;
                        const float2 wv = ws[(b < n_beams ? b : 0) * n_ant + a];
                        ur[q][p] = fmaf(wv.x, yr, fmaf(-wv.y, yi, ur[q][p]));
                        ui[q][p] = fmaf(wv.x, yi, fmaf(wv.y, yr, ui[q][p]));
                    }
                }
            const int gpass = sub * (kMbFrames / 32) + pass;        // 32-frame pass of the CTA
#pragma unroll
            for (int q = 0; q < BPT; ++q) {
                const int b = warp + q * kMbWarps;
                if (b >= n_beams) break;
                if (products == 1) {
                    out[(static_cast<int64_t>(b) * n_out + ts + f) * n_chan + k] =
                        make_float4(ur[q][0], ui[q][0], ur[q][1], ui[q][1]);
                    continue;
                }
                float4 v = make_float4(ur[q][0] * ur[q][0] + ui[q][0] * ui[q][0],
                                       ur[q][1] * ur[q][1] + ui[q][1] * ui[q][1],
                                       ur[q][0] * ur[q][1] + ui[q][0] * ui[q][1],
                                       ui[q][0] * ur[q][1] - ur[q][0] * ui[q][1]);
                // sum over the window's lanes (avg <= 32), or over the warp (avg > 32), fixed order
                const int span = avg < 32 ? avg : 32;
                for (int off = 1; off < span; off <<= 1) {
                    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
                    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
                    v.z += __shfl_xor_sync(0xffffffffu, v.z, off);
                    v.w += __shfl_xor_sync(0xffffffffu, v.w, off);
                }
                const float sc = 1.0f / avg;
                if (avg <= 32) {
                    if (lane % span == 0)
                        out[(static_cast<int64_t>(b) * n_out + (ts + f) / avg) * n_chan + k] =
                            make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
                } else if (lane == 0) {                             // passes of one window, in order
                    float4 a4 = gpass == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[b];
                    a4 = make_float4(a4.x + v.x, a4.y + v.y, a4.z + v.z, a4.w + v.w);
                    acc[b] = a4;
                    if (gpass == fcta / 32 - 1)
                        out[(static_cast<int64_t>(b) * n_out + t0 / avg) * n_chan + k] =
                            make_float4(a4.x * sc, a4.y * sc, a4.z * sc, a4.w * sc);
                }
            }
        }
        __syncthreads();                                            // the stage is read: the next may land
    }
    if (!ok && threadIdx.x == 0)        // the copies of the stage whose wait ran out land before the CTA exits
        mbar_wait(&ms.bar, last_sub & 1, nullptr, 0);
}

}  // namespace

int multibeam_max_beams() { return kMbMaxBeams; }

size_t multibeam_smem(int n_in, int n_chan, int n_beams, int n_ant) {
    const int tb = tb_fp32(n_chan), blk = rows_fp32(n_in) * tb;
    const int wstride = ((n_beams * n_ant + 1) / 2) * 2;
    return sizeof(float) * (static_cast<size_t>(kMbFrames / tb) * (blk + kMbPad)) + sizeof(float2) * wstride +
           sizeof(float4) * n_beams;
}

int multibeam_wstride(int n_beams, int n_ant) { return ((n_beams * n_ant + 1) / 2) * 2; }

cudaError_t launch_multibeam(const float* spec, int n_ant, int n_pol, int n_chan, int n_int, const float2* w,
                             int n_beams, int products, int avg, float4* out, unsigned* err, cudaStream_t s) {
    const int fcta = avg > kMbFrames ? avg : kMbFrames;
    if (n_beams < 1 || n_beams > kMbMaxBeams || avg < 1 || (avg & (avg - 1)) || n_int % fcta ||
        (products != 0 && products != 1) || (products == 1 && avg != 1))
        return cudaErrorInvalidValue;
    const size_t smem = multibeam_smem(n_ant * n_pol, n_chan, n_beams, n_ant);
    const int wstride = multibeam_wstride(n_beams, n_ant);
    const dim3 grid(n_chan, n_int / fcta);
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        kern<<<grid, kMbThreads, smem, s>>>(spec, n_ant, n_pol, n_chan, n_int, w, wstride, n_beams, products, avg, out,
                                            err);
        return cudaGetLastError();
    };
    const int bpt = (n_beams + kMbWarps - 1) / kMbWarps;
    if (bpt <= 1) return go(multibeam_kernel<1>);
    if (bpt <= 2) return go(multibeam_kernel<2>);
    if (bpt <= 4) return go(multibeam_kernel<4>);
    return go(multibeam_kernel<8>);
}

}  // namespace gbx
