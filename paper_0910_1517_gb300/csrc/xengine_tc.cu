// xengine_tc.cu -- X-engine on the tcgen05 tensor cores (sm_103a).
//
// Per channel k the visibilities are one dense contraction.  With the 2 n_in
// real rows A[r][t], r = 2i + c (c = 0 real, 1 imaginary part of Y_i[t]),
// the real Gram G = A A^T (K = n_int frames) holds every product:
//   Re V_ij = G[2i][2j] + G[2i+1][2j+1],  Im V_ij = G[2i+1][2j] - G[2i][2j+1].
// A is the F-engine's K-block layout, which already is the no-swizzle K-major
// canonical operand layout (core matrices of 8 rows x 16 bytes), so one
// TMA-engine bulk copy per stage lands a ready operand tile and the same shared
// memory tile serves as both A and B.
//
// Work items are (sub-array, channel, row block): 128 Gram rows a0..a0+127 against
// columns b0..b0+N-1.  Up to 128 rows need one item (N <= 128, the rest of the 128
// rows is ignored); 256 rows need two (rows 0-127 x columns 0-255, rows 128-255 x
// columns 128-255).  A persistent CTA walks a cost-ordered item list; several
// sub-arrays of different sizes share one launch.
//
// Roles (6 warps): warp 0 streams stages in (and owns the TMEM allocation),
// warp 1 issues tcgen05.mma from one thread, warps 2-5 drain the accumulators.
// Accumulation is chunked: every 1024 frames the FP32 accumulator is drained
// and added into a running sum in TMEM (columns 256-511).  Items with N <= 128
// double-buffer the accumulator (columns 0-127 / 128-255), wider ones use one
// buffer of N columns.  For int8-valued operands every product is an integer of
// magnitude at most 127^2 = 16129 and a chunk sum at most 1024 * 16129 =
// 16,516,096 < 2^24, so the FP32 accumulator is exact and the running sum is kept
// as int32: the result equals the integer MAC.
#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
namespace {

constexpr int kWarps = 6;
constexpr int kThreads = kWarps * 32;
constexpr int kStages = 5;
constexpr int kChunk = 1024;                  // frames per exact FP32 chunk
constexpr int kSlot = kStageMaxBytes + 2048;  // rows past R stay in bounds
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

struct ItemGeo {
    int sub, k, a0, b0, N, R, ntb, n_stage, n_chunk, nkb_stage;
    bool dbl;
};

__device__ __forceinline__ ItemGeo item_geo(const XtBatch& t, int it) {
    ItemGeo g;
    const int4 e = t.items[it];
    g.sub = e.x;
    g.k = e.y;
    const XtSub& s = t.sub[g.sub];
    g.R = 2 * s.n_in;
    g.a0 = 128 * e.z;
    g.b0 = (g.R > 128) ? g.a0 : 0;
    g.N = ((g.R - g.b0 + 15) / 16) * 16;
    g.dbl = g.N <= 128;
    g.ntb = s.n_int / kTbHalf;
    g.nkb_stage = s.ks / kTbHalf;
    g.n_stage = (s.n_int + s.ks - 1) / s.ks;
    g.n_chunk = (s.n_int + kChunk - 1) / kChunk;
    return g;
}

__global__ void __launch_bounds__(kThreads, 1) xengine_tc_kernel(const XtBatch* __restrict__ tab) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Shared sh;
    const XtBatch& t = *tab;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

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
            for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
                const ItemGeo ig = item_geo(t, it);
                const XtSub& s = t.sub[ig.sub];
                for (int st = 0; st < ig.n_stage; ++st, ++g) {
                    const int slot = g % kStages;
                    if (!mbar_wait(&sh.empty[slot], ((g / kStages) & 1) ^ 1, t.err, ERR_WAIT_MMA)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int kb0 = st * ig.nkb_stage;
                    const int nkb = min(ig.nkb_stage, ig.ntb - kb0);
                    const uint32_t bytes = static_cast<uint32_t>(nkb) * ig.R * 16;
                    const __half* src = s.spec + (static_cast<int64_t>(ig.k) * ig.ntb + kb0) * ig.R * kTbHalf;
                    mbar_arrive_expect_tx(&sh.full[slot], bytes);
                    bulk_g2s(smem + slot * kSlot, src, bytes, &sh.full[slot]);
                }
            }
            // let every issued copy land before the CTA can exit
            for (int q = *(volatile int*)&sh.consumed; q < g; ++q)
                mbar_wait(&sh.full[q % kStages], (q / kStages) & 1, nullptr, 0);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int g = 0, cc = 0, use0 = 0, use1 = 0;
            int prev_dbl = -1;
            for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
                const ItemGeo ig = item_geo(t, it);
                const XtSub& s = t.sub[ig.sub];
                const uint32_t idesc = idesc_f16_f32(128, ig.N);
                const uint32_t lbo = static_cast<uint32_t>(ig.R) * 16, sbo = 128;
                const int stages_per_chunk = kChunk / s.ks;
                for (int chunk = 0; chunk < ig.n_chunk && !*abort_flag; ++chunk, ++cc) {
                    const int b = ig.dbl ? (cc & 1) : 0;
                    // a single-buffered item, or a change of buffering, needs every earlier drain done
                    bool ok = true;
                    if (!ig.dbl || prev_dbl != static_cast<int>(ig.dbl)) {
                        ok = mbar_wait(&sh.acce[0], (use0 & 1) ^ 1, t.err, ERR_WAIT_EPI) &&
                             mbar_wait(&sh.acce[1], (use1 & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    } else {
                        ok = mbar_wait(&sh.acce[b], ((b ? use1 : use0) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    }
                    prev_dbl = ig.dbl;
                    if (!ok) {
                        *abort_flag = 1;
                        break;
                    }
                    if (b) ++use1; else ++use0;
                    tc_fence_after();
                    const uint32_t dcol = tmem + (ig.dbl ? b * 128 : 0);
                    const int st0 = chunk * stages_per_chunk;
                    const int st1 = min(ig.n_stage, st0 + stages_per_chunk);
                    bool first = true;
                    for (int st = st0; st < st1; ++st, ++g) {
                        const int slot = g % kStages;
                        if (!mbar_wait(&sh.full[slot], (g / kStages) & 1, t.err, ERR_WAIT_STAGE)) {
                            *abort_flag = 1;
                            break;
                        }
                        tc_fence_after();
                        const int nkb = min(ig.nkb_stage, ig.ntb - st * ig.nkb_stage);
                        const uint32_t base = smem_u32(smem + slot * kSlot);
                        for (int kk = 0; kk < nkb / 2; ++kk) {
                            const uint32_t kbase = base + kk * 2 * lbo;
                            const uint64_t da = smem_desc_noswizzle(kbase + ig.a0 * 16, lbo, sbo);
                            const uint64_t db = smem_desc_noswizzle(kbase + ig.b0 * 16, lbo, sbo);
                            umma_f16(dcol, da, db, idesc, first ? 0u : 1u);
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
        const int lrow = 32 * q + lane;           // row within the item's 128 rows = TMEM lane
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        int cc = 0, use0 = 0, use1 = 0;
        for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
            const ItemGeo ig = item_geo(t, it);
            const XtSub& s = t.sub[ig.sub];
            const int n_bl = s.n_ant * (s.n_ant + 1) / 2, npp = s.n_pol * s.n_pol;
            const int row = ig.a0 + lrow;
            for (int chunk = 0; chunk < ig.n_chunk; ++chunk, ++cc) {
                const int b = ig.dbl ? (cc & 1) : 0;
                const int use = b ? use1 : use0;
                if (!mbar_wait(&sh.accf[b], use & 1, t.err, ERR_WAIT_MMA)) {
                    *abort_flag = 1;
                    break;
                }
                if (b) ++use1; else ++use0;
                tc_fence_after();
                const bool last = chunk == ig.n_chunk - 1;
                const uint32_t acol = ig.dbl ? b * 128 : 0;
                for (int j0 = 0; j0 < ig.N; j0 += 32) {
                    uint32_t v[32], run[32];
                    tmem_ld32(tmem + lane_off + acol + j0, v);
                    if (chunk > 0) tmem_ld32(tmem + lane_off + kColRun + j0, run);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (s.exact) {
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
                            const int j = ((ig.b0 + j0) >> 1) + jp;
                            const uint32_t g_r0c0 = odd ? other[2 * jp] : run[2 * jp];
                            const uint32_t g_r0c1 = odd ? other[2 * jp + 1] : run[2 * jp + 1];
                            const uint32_t g_r1c0 = odd ? run[2 * jp] : other[2 * jp];
                            const uint32_t g_r1c1 = odd ? run[2 * jp + 1] : other[2 * jp + 1];
                            if (i >= s.n_in || j >= s.n_in) continue;
                            const int a = i / s.n_pol, pp = i % s.n_pol, a2 = j / s.n_pol, qq = j % s.n_pol;
                            if (a > a2) continue;
                            const int bl = a * s.n_ant - a * (a - 1) / 2 + (a2 - a);
                            const int64_t o = (static_cast<int64_t>(ig.k) * n_bl + bl) * npp + pp * s.n_pol + qq;
                            const float d = s.scale[static_cast<int64_t>(i) * s.n_chan + ig.k] *
                                            s.scale[static_cast<int64_t>(j) * s.n_chan + ig.k];
                            if (s.exact) {
                                const int re = static_cast<int>(g_r0c0) + static_cast<int>(g_r1c1);
                                const int im = static_cast<int>(g_r1c0) - static_cast<int>(g_r0c1);
                                if (s.vis_int) s.vis_int[o] = make_int2(re, im);
                                s.vis[o] = make_float2(static_cast<float>(re) / d, static_cast<float>(im) / d);
                            } else {
                                const float re = __uint_as_float(g_r0c0) + __uint_as_float(g_r1c1);
                                const float im = __uint_as_float(g_r1c0) - __uint_as_float(g_r0c1);
                                s.vis[o] = make_float2(re / d, im / d);
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

bool xengine_tc_supported(int n_in) { return n_in >= 1 && 2 * n_in <= 256; }

int xengine_tc_max_ks(int n_in) {
    int ks = 512;                                  // stages of at most 512 frames
    while (ks > 16 && (ks / kTbHalf) * 2 * n_in * 16 > kStageMaxBytes) ks /= 2;
    return ks;
}

size_t xengine_tc_smem() { return static_cast<size_t>(kStages) * kSlot + kTailSlack; }

cudaError_t launch_xengine_tc_table(const XtBatch* dtab, int n_items, int n_sm, cudaStream_t s) {
    const size_t smem = xengine_tc_smem();
    cudaError_t e = cudaFuncSetAttribute(xengine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(n_items, n_sm));
    xengine_tc_kernel<<<grid, kThreads, smem, s>>>(dtab);
    return cudaGetLastError();
}

}  // namespace gbx
