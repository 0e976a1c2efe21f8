// multibeam.cu -- several phased-array beams with full-polar products or voltages (Sec. 2.2:
// the coherent beamformer also gives the voltage cross products for the Stokes parameters;
// Sec. 5: multiple phased beams covering different directions in the primary beam), from the
// F-engine's FP32 spectra:
//   U_bp[t][k] = sum_a w[k][b][a] Y_{a,p}[t][k]     (FP32 complex multiply-adds)
//   full polar (products 0): mean over `avg` frames of |U_b0|^2, |U_b1|^2, Re U_b0 conj U_b1,
//                            Im U_b0 conj U_b1
//   voltages   (products 1, avg 1): Re U_b0, Im U_b0, Re U_b1, Im U_b1
//
// One CTA takes channel k and up to 512 frames, staged 64 at a time through two buffers (one
// bulk copy per stage, the next stages in flight): each stage's FP32 K-blocks are transposed
// once into planes Yr[i][f], Yi[i][f].  Lanes are consecutive frames (two per lane) and warps
// beam groups (beams w, w + 8, ...), so every weight read is a broadcast, shared by two frames,
// and each sample is read once for all of a thread's beams.  A window of `avg` frames is summed
// by shuffles across its lanes (avg <= 32) and then across 32-frame passes in order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

constexpr int kMbThreads = 256;
constexpr int kMbWarps = kMbThreads / 32;
constexpr int kMbMaxBeams = 64;                 // beams per launch (kMbMaxBeams / kMbWarps per thread)
constexpr int kMbFrames = 64;                   // frames per shared-memory stage (a lane takes 2)
constexpr int kMbMaxIn = 128;
constexpr int kMbTcMinBeams = 24;               // more beams than this: the tensor-core form

struct MbShared {
    uint64_t bar[2];
};

// Shared memory: two raw stages (the FP32 K-blocks of 64 frames), the stage transposed into
// planes Yr[i][f], Yi[i][f], the channel's weights and the window accumulators.
__host__ __device__ constexpr size_t mb_raw_floats(int n_in, int n_chan) {
    return static_cast<size_t>(rows_fp32(n_in)) * kMbFrames;
}

template <int BPT>   // beams per thread
__global__ void __launch_bounds__(kMbThreads) multibeam_kernel(const float* __restrict__ spec, int n_ant, int n_pol,
                                                               int n_chan, int n_int, const float2* __restrict__ w,
                                                               int wstride, int n_beams, int products, int avg,
                                                               int span, float4* __restrict__ out, unsigned* err) {
    extern __shared__ __align__(16) float sm[];
    __shared__ MbShared ms;
    const int n_in = n_ant * n_pol;
    const int tb = tb_fp32(n_chan), Rp = rows_fp32(n_in);
    const int raw_f = static_cast<int>(mb_raw_floats(n_in, n_chan));
    float* yr = sm + 2 * raw_f;                                     // raw stages: sm + (st & 1) * raw_f                                     // [n_in][64]
    float* yi = yr + n_in * kMbFrames;
    float2* ws = reinterpret_cast<float2*>(yi + n_in * kMbFrames);  // [beam][antenna] of channel k
    float4* acc = reinterpret_cast<float4*>(ws + wstride);          // per (beam, frame half) window sums
    const int k = blockIdx.x, t0 = blockIdx.y * span;
    const int64_t ntb = n_int / tb;
    const int n_stage = span / kMbFrames;
    const uint32_t stage_bytes = static_cast<uint32_t>(raw_f) * 4;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    auto issue = [&](int st) {   // thread 0: stage st's K-blocks (contiguous) into raw[st & 1]
        const uint32_t wbytes = st == 0 ? static_cast<uint32_t>(wstride) * sizeof(float2) : 0u;
        mbar_arrive_expect_tx(&ms.bar[st & 1], stage_bytes + wbytes);
        bulk_g2s(sm + (st & 1) * raw_f, spec + (static_cast<int64_t>(k) * ntb + (t0 + st * kMbFrames) / tb) * Rp * tb,
                 stage_bytes, &ms.bar[st & 1]);
        if (st == 0) bulk_g2s(ws, w + static_cast<int64_t>(k) * wstride, wbytes, &ms.bar[0]);
    };
    if (tid == 0) {
        mbar_init(&ms.bar[0], 1);
        mbar_init(&ms.bar[1], 1);
        fence_mbar_init();
        issue(0);
        if (n_stage > 1) issue(1);
    }
    __syncthreads();
    const int n_out = n_int / avg;
    bool ok = true;
    int st = 0;
    for (; st < n_stage && ok; ++st) {
        ok = __syncthreads_and(mbar_wait(&ms.bar[st & 1], (st >> 1) & 1, err, ERR_WAIT_STAGE));
        if (!ok) break;
        // transpose: granule q of the stage = 4 frames of one row (the FP32 layout's XOR placement undone)
        const float* rs = sm + (st & 1) * raw_f;
        const int gpb = Rp * tb / 4;                                // granules per K-block
        for (int q = tid; q < (kMbFrames / tb) * gpb; q += kMbThreads) {
            const int kb = q / gpb, pos = q % gpb;
            const int G = pos / (2 * tb), gs = (pos % (2 * tb)) ^ (G & 7);
            const int r = G * 8 + gs / (tb / 4), f0 = kb * tb + (gs % (tb / 4)) * 4;
            if (r >= 2 * n_in) continue;                            // padding rows
            const float4 v = reinterpret_cast<const float4*>(rs)[q];
            *reinterpret_cast<float4*>(((r & 1) ? yi : yr) + (r >> 1) * kMbFrames + f0) = v;
        }
        __syncthreads();                                            // the raw stage read, planes written
        if (tid == 0 && st + 2 < n_stage) issue(st + 2);
        // beams: lane takes frames lane and lane + 32 of the stage, warp the beams warp + 8 q
        float ur[BPT][2][2], ui[BPT][2][2];                         // [beam][frame half][pol]
#pragma unroll
        for (int q = 0; q < BPT; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) ur[q][h][0] = ur[q][h][1] = ui[q][h][0] = ui[q][h][1] = 0.0f;
        for (int a = 0; a < n_ant; ++a)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                if (p >= n_pol) break;
                const int i = a * n_pol + p;
                const float r0 = yr[i * kMbFrames + lane], i0 = yi[i * kMbFrames + lane];
                const float r1 = yr[i * kMbFrames + lane + 32], i1 = yi[i * kMbFrames + lane + 32];
#pragma unroll
                for (int q = 0; q < BPT; ++q) {
                    const int b = warp + q * kMbWarps;
                    const float2 wv = ws[(b < n_beams ? b : 0) * n_ant + a];
                    ur[q][0][p] = fmaf(wv.x, r0, fmaf(-wv.y, i0, ur[q][0][p]));
                    ui[q][0][p] = fmaf(wv.x, i0, fmaf(wv.y, r0, ui[q][0][p]));
                    ur[q][1][p] = fmaf(wv.x, r1, fmaf(-wv.y, i1, ur[q][1][p]));
                    ui[q][1][p] = fmaf(wv.x, i1, fmaf(wv.y, r1, ui[q][1][p]));
                }
            }
        const int ts = t0 + st * kMbFrames;                         // first frame of the stage
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int b = warp + q * kMbWarps;
            if (b >= n_beams) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = h * 32 + lane;
                if (products == 1) {
                    out[(static_cast<int64_t>(b) * n_out + ts + f) * n_chan + k] =
                        make_float4(ur[q][h][0], ui[q][h][0], ur[q][h][1], ui[q][h][1]);
                    continue;
                }
                float4 v = make_float4(ur[q][h][0] * ur[q][h][0] + ui[q][h][0] * ui[q][h][0],
                                       ur[q][h][1] * ur[q][h][1] + ui[q][h][1] * ui[q][h][1],
                                       ur[q][h][0] * ur[q][h][1] + ui[q][h][0] * ui[q][h][1],
                                       ui[q][h][0] * ur[q][h][1] - ur[q][h][0] * ui[q][h][1]);
                // sum over the window's lanes (avg <= 32), or over the warp (avg > 32), fixed order
                const int sp = avg < 32 ? avg : 32;
                for (int off = 1; off < sp; off <<= 1) {
                    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
                    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
                    v.z += __shfl_xor_sync(0xffffffffu, v.z, off);
                    v.w += __shfl_xor_sync(0xffffffffu, v.w, off);
                }
                const float sc = 1.0f / avg;
                if (avg <= 32) {
                    if (lane % sp == 0)
                        out[(static_cast<int64_t>(b) * n_out + (ts + f) / avg) * n_chan + k] =
                            make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
                } else if (lane == 0) {                             // 32-frame passes of one window, in order
                    const int gpass = (ts + f - t0) / 32;           // pass index within the CTA
                    const int per = avg / 32;
                    float4 a4 = gpass % per == 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : acc[b];
                    a4 = make_float4(a4.x + v.x, a4.y + v.y, a4.z + v.z, a4.w + v.w);
                    acc[b] = a4;
                    if (gpass % per == per - 1)
                        out[(static_cast<int64_t>(b) * n_out + (ts + f) / avg) * n_chan + k] =
                            make_float4(a4.x * sc, a4.y * sc, a4.z * sc, a4.w * sc);
                }
            }
        }
        __syncthreads();                                            // planes read: the next transpose may write
    }
    if (!ok && tid == 0) {   // copies in flight land before the CTA exits (bounded)
        for (int q = st; q < n_stage && q < st + 2; ++q) mbar_wait(&ms.bar[q & 1], (q >> 1) & 1, nullptr, 0);
    }
}

}  // namespace

int multibeam_max_beams() { return kMbMaxBeams; }

size_t multibeam_smem(int n_in, int n_chan, int n_beams, int n_ant) {
    const int wstride = ((n_beams * n_ant + 1) / 2) * 2;
    return sizeof(float) * (2 * mb_raw_floats(n_in, n_chan) + 2 * static_cast<size_t>(n_in) * kMbFrames) +
           sizeof(float2) * wstride + sizeof(float4) * n_beams;
}

int multibeam_wstride(int n_beams, int n_ant) { return ((n_beams * n_ant + 1) / 2) * 2; }

cudaError_t launch_multibeam(const float* spec, int n_ant, int n_pol, int n_chan, int n_int, const float2* w,
                             int n_beams, int products, int avg, float4* out, unsigned* err, cudaStream_t s) {
    if (n_beams < 1 || n_beams > kMbMaxBeams || avg < 1 || (avg & (avg - 1)) || n_int % (avg > 64 ? avg : 64) ||
        (products != 0 && products != 1) || (products == 1 && avg != 1) || n_ant * n_pol > kMbMaxIn)
        return cudaErrorInvalidValue;
    // frames per CTA: a multiple of 64 and of avg dividing n_int, up to 512 (more stages per CTA
    // hide the copies; fewer CTAs per channel leave enough of them)
    int span = avg > 64 ? avg : 64;
    while (span < 512 && n_int % (2 * span) == 0) span *= 2;
    const int wstride = multibeam_wstride(n_beams, n_ant);
    // the tensor-core form for many beams: its time hardly depends on the beam count (5.0 ms for
    // 16 and 5.1 ms for 64 beams at GMRT scale), the CUDA-core kernel's grows with it (3.4 ms for
    // 16, 13.0 ms for 64); they cross near 24 beams
    if (n_beams > kMbTcMinBeams && multibeam_tc_supported(n_ant, n_pol, n_chan, n_int)) {
        int e = -8;
        for (int n = 2 * n_chan; n > 1; n >>= 1) ++e;
        return launch_multibeam_tc(spec, n_ant, n_pol, n_chan, n_int, w, wstride, n_beams, products, avg,
                                   ldexpf(1.0f, -e), out, err, s);
    }
    const size_t smem = multibeam_smem(n_ant * n_pol, n_chan, n_beams, n_ant);
    const dim3 grid(n_chan, n_int / span);
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        kern<<<grid, kMbThreads, smem, s>>>(spec, n_ant, n_pol, n_chan, n_int, w, wstride, n_beams, products, avg,
                                            span, out, err);
        return cudaGetLastError();
    };
    const int bpt = (n_beams + kMbWarps - 1) / kMbWarps;
    if (bpt <= 1) return go(multibeam_kernel<1>);
    if (bpt <= 2) return go(multibeam_kernel<2>);
    if (bpt <= 4) return go(multibeam_kernel<4>);
    return go(multibeam_kernel<8>);
}

}  // namespace gbx
