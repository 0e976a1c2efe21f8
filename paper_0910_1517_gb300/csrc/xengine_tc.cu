// xengine_tc.cu -- X-engine on the tcgen05 tensor cores (sm_103a).
//
// Per channel k the visibilities are one dense contraction.  With the 2 n_in
// real rows A[r][t], r = 2i + c (c = 0 real, 1 imaginary part of Y_i[t]),
// the real Gram G = A A^T (M = N = 128 rows, K = n_int frames) holds every
// product:  Re V_ij = G[2i][2j] + G[2i+1][2j+1],  Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// A is the F-engine's K-block layout, which already is the no-swizzle K-major
// canonical operand layout (core matrices of 8 rows x 16 bytes), so one
// TMA-engine bulk copy per stage lands a ready operand tile and the same shared
// memory tile is passed as both A and B.
//
// Roles (6 warps): warp 0 streams stages in (and owns the TMEM allocation),
// warp 1 issues tcgen05.mma from one thread, warps 2-5 drain the accumulators.
// Accumulation is chunked: every 512 frames the FP32 accumulator (double
// buffered in TMEM) is drained and added into a running sum kept in TMEM.  For
// int8-valued operands every product is an integer below 2^14 and a chunk sum
// stays below 2^23, so the FP32 accumulator is exact and the running sum is
// kept as int32: the result equals the integer MAC bit for bit.
#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
namespace {

constexpr int kWarps = 6;
constexpr int kThreads = kWarps * 32;
constexpr int kStages = 8;
constexpr int kFramesPerStage = 64;           // 8 K-blocks of 8 frames, 4 MMAs of K = 16
constexpr int kStagesPerChunk = 8;            // 512 frames per exact FP32 chunk
constexpr int kRowsMax = 128;
constexpr int kStageBytes = (kFramesPerStage / kTbHalf) * kRowsMax * 16;   // 16 KB
constexpr int kStageStride = kStageBytes + 2048;                           // rows past R stay in bounds
constexpr int kTailSlack = 32768;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColRun = 256;             // running-sum columns

struct Shared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accf[2];
    uint64_t acce[2];
    uint32_t taddr;
    int abort_flag;
    int consumed;
};

__global__ void __launch_bounds__(kThreads, 1) xengine_tc_kernel(const XParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Shared sh;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int R = 2 * p.n_in;
    const int NP = ((R + 15) / 16) * 16;           // MMA N
    const int ntb = p.n_int / kTbHalf;
    const int n_stage_ch = (p.n_int + kFramesPerStage - 1) / kFramesPerStage;
    const int n_ch_mine = (p.n_chan - static_cast<int>(blockIdx.x) + gridDim.x - 1) / gridDim.x;
    const int n_chunk_ch = (n_stage_ch + kStagesPerChunk - 1) / kStagesPerChunk;
    const __half* spec = static_cast<const __half*>(p.spec);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh.accf[b], 1);
            mbar_init(&sh.acce[b], 128);
        }
        fence_mbar_init();
        sh.abort_flag = 0;
        sh.consumed = 0;
    }
    if (warp == 0) {
        tmem_alloc(&sh.taddr, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.taddr;
    volatile int* abort_flag = &sh.abort_flag;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int g = 0;
            for (int c = 0; c < n_ch_mine && !*abort_flag; ++c) {
                const int k = blockIdx.x + c * gridDim.x;
                for (int st = 0; st < n_stage_ch; ++st, ++g) {
                    const int slot = g % kStages;
                    if (!mbar_wait(&sh.empty[slot], ((g / kStages) & 1) ^ 1, p.err, ERR_WAIT_MMA)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int kb0 = st * (kFramesPerStage / kTbHalf);
                    const int nkb = min(kFramesPerStage / kTbHalf, ntb - kb0);
                    const uint32_t bytes = static_cast<uint32_t>(nkb) * R * 16;
                    const __half* src = spec + (static_cast<int64_t>(k) * ntb + kb0) * R * kTbHalf;
                    mbar_arrive_expect_tx(&sh.full[slot], bytes);
                    bulk_g2s(smem + slot * kStageStride, src, bytes, &sh.full[slot]);
                }
            }
            // let every issued copy land before the CTA can exit
            for (int q = sh.consumed; q < g; ++q)
                mbar_wait(&sh.full[q % kStages], (q / kStages) & 1, nullptr, 0);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16_f32(128, NP);
            const uint32_t lbo = static_cast<uint32_t>(R) * 16, sbo = 128;
            int g = 0, cc = 0;
            for (int c = 0; c < n_ch_mine && !*abort_flag; ++c) {
                for (int chunk = 0; chunk < n_chunk_ch && !*abort_flag; ++chunk, ++cc) {
                    const int b = cc & 1;
                    if (!mbar_wait(&sh.acce[b], ((cc >> 1) & 1) ^ 1, p.err, ERR_WAIT_EPI)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dcol = tmem + b * 128;
                    const int st0 = chunk * kStagesPerChunk;
                    const int st1 = min(n_stage_ch, st0 + kStagesPerChunk);
                    bool first = true;
                    for (int st = st0; st < st1; ++st, ++g) {
                        const int slot = g % kStages;
                        if (!mbar_wait(&sh.full[slot], (g / kStages) & 1, p.err, ERR_WAIT_STAGE)) {
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const int nkb = min(kFramesPerStage / kTbHalf, ntb - st * (kFramesPerStage / kTbHalf));
                        const uint32_t base = smem_u32(smem + slot * kStageStride);
                        for (int kk = 0; kk < nkb / 2; ++kk) {
                            const uint64_t d = smem_desc_noswizzle(base + kk * 2 * lbo, lbo, sbo);
                            umma_f16(dcol, d, d, idesc, first ? 0u : 1u);
                            first = false;
                        }
                        umma_commit(&sh.empty[slot]);   // frees the stage once these MMAs finish
                        sh.consumed = g + 1;
                    }
                    if (*abort_flag) break;
                    umma_commit(&sh.accf[b]);           // chunk complete
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..5)
        const int q = warp & 3;                   // TMEM lane quarter this warp may access
        const int row = 32 * q + lane;            // Gram row = TMEM lane
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const int n_bl = p.n_ant * (p.n_ant + 1) / 2, npp = p.n_pol * p.n_pol;
        int cc = 0;
        for (int c = 0; c < n_ch_mine && !*abort_flag; ++c) {
            const int k = blockIdx.x + c * gridDim.x;
            for (int chunk = 0; chunk < n_chunk_ch; ++chunk, ++cc) {
                const int b = cc & 1;
                if (!mbar_wait(&sh.accf[b], (cc >> 1) & 1, p.err, ERR_WAIT_MMA)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const bool last = chunk == n_chunk_ch - 1;
                for (int j0 = 0; j0 < NP; j0 += 32) {
                    uint32_t v[32], run[32];
                    tmem_ld32(tmem + lane_off + b * 128 + j0, v);
                    if (chunk > 0) tmem_ld32(tmem + lane_off + kColRun + j0, run);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (p.exact) {
                            const int x = __float2int_rn(__uint_as_float(v[e]));
                            run[e] = chunk > 0 ? static_cast<uint32_t>(static_cast<int>(run[e]) + x)
                                               : static_cast<uint32_t>(x);
                        } else {
                            const float x = __uint_as_float(v[e]);
                            run[e] = __float_as_uint(chunk > 0 ? __uint_as_float(run[e]) + x : x);
                        }
                    }
                    if (!last) {
                        tmem_st32(tmem + lane_off + kColRun + j0, run);
                    } else {
                        // final sums of columns j0..j0+31: pair rows 2i and 2i+1 (adjacent lanes)
                        uint32_t other[32];
#pragma unroll
                        for (int e = 0; e < 32; ++e) other[e] = __shfl_xor_sync(0xffffffffu, run[e], 1);
                        const bool odd = row & 1;
                        const int i = row >> 1;
                        // even lane: j' = 0..7 of this slice, odd lane: j' = 8..15
#pragma unroll
                        for (int jh = 0; jh < 8; ++jh) {
                            const int jp = jh + (odd ? 8 : 0);
                            const int j = (j0 >> 1) + jp;
                            // row 2i values and row 2i+1 values at columns 2jp, 2jp+1
                            const uint32_t g_r0c0 = odd ? other[2 * jp] : run[2 * jp];
                            const uint32_t g_r0c1 = odd ? other[2 * jp + 1] : run[2 * jp + 1];
                            const uint32_t g_r1c0 = odd ? run[2 * jp] : other[2 * jp];
                            const uint32_t g_r1c1 = odd ? run[2 * jp + 1] : other[2 * jp + 1];
                            if (i >= p.n_in || j >= p.n_in) continue;
                            const int a = i / p.n_pol, pp = i % p.n_pol, a2 = j / p.n_pol, qq = j % p.n_pol;
                            if (a > a2) continue;
                            const int bl = a * p.n_ant - a * (a - 1) / 2 + (a2 - a);
                            const int64_t o = (static_cast<int64_t>(k) * n_bl + bl) * npp + pp * p.n_pol + qq;
                            const float d = p.scale[static_cast<int64_t>(i) * p.n_chan + k] *
                                            p.scale[static_cast<int64_t>(j) * p.n_chan + k];
                            if (p.exact) {
                                const int re = static_cast<int>(g_r0c0) + static_cast<int>(g_r1c1);
                                const int im = static_cast<int>(g_r1c0) - static_cast<int>(g_r0c1);
                                if (p.vis_int) p.vis_int[o] = make_int2(re, im);
                                p.vis[o] = make_float2(static_cast<float>(re) / d, static_cast<float>(im) / d);
                            } else {
                                const float re = __uint_as_float(g_r0c0) + __uint_as_float(g_r1c1);
                                const float im = __uint_as_float(g_r1c0) - __uint_as_float(g_r0c1);
                                p.vis[o] = make_float2(re / d, im / d);
                            }
                        }
                    }
                }
                if (!last) tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&sh.acce[b]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

bool xengine_tc_supported(int n_in) { return n_in >= 1 && 2 * n_in <= kRowsMax; }

cudaError_t launch_xengine_tc(const XParams& p, int n_sm, cudaStream_t s) {
    if (!xengine_tc_supported(p.n_in) || p.n_int % 16 != 0) return cudaErrorInvalidValue;
    const size_t smem = static_cast<size_t>(kStages) * kStageStride + kTailSlack;
    cudaError_t e = cudaFuncSetAttribute(xengine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(p.n_chan, n_sm));
    xengine_tc_kernel<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace gbx
