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
// Roles (10 warps): warp 0 streams stages in (and owns the TMEM allocation),
// warp 1 issues tcgen05.mma from one thread, warps 2-9 drain the accumulators
// (warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. Gram rows, and the column half
// (w - 2) / 4 of them).
// Accumulation is chunked: every `chunk` frames the FP32 accumulator is drained
// and added into a running sum.  Items with N <= 128 rotate over four 128-column
// accumulators (the MMAs run up to three chunks ahead of the drain) and keep the
// running sums in the draining threads' registers (one Gram row per thread);
// wider items use one accumulator of N columns and a running sum in TMEM
// (columns 256-511).  For int8-valued operands (chunk 1024) every product is an
// integer of magnitude at most 127^2 = 16129 and a chunk sum at most 1024 * 16129 =
// 16,516,096 < 2^24, so the FP32 accumulator is exact and the running sum is kept
// as int32: the result equals the integer MAC.
//
// Two-plane FP32 form: each FP32 value v (scaled by a power of two) arrives as
// fp16 hi + lo with |v - hi - lo| <= 2^-22 |v|.  Every stage carries both planes
// and each 16-frame step issues three MMAs, H H^T + H L^T + L H^T (the dropped
// L L^T is below 2^-22 of the product).  fp16 x fp16 products are exact in FP32,
// but the tensor core's FP32 accumulation drops low bits of every partial sum, a
// loss that grows with the accumulator's size and the number of steps.  So the
// dominant H H^T term is accumulated in 128-frame chunks that the CUDA cores add
// in FP32, while the cross terms, 2^-11 of it, go to a separate accumulator
// (columns 384-511) over the whole integration: narrow items then rotate over
// three chunk accumulators.
#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
namespace {

constexpr int kWarps = 10;
constexpr int kEpiThreads = (kWarps - 2) * 32;
constexpr int kThreads = kWarps * 32;
constexpr int kStages = 5;
constexpr int kSlot = kStageMaxBytes + 2048;  // rows past R stay in bounds
constexpr int kTailSlack = 32768;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColRun = 256;             // running-sum columns of wide items
constexpr int kAccBufs = 4;                   // 128-column accumulators of narrow items
constexpr uint32_t kColX = 384;               // two-plane narrow items: the cross-term accumulator
constexpr int kXBit = 4;                      // its parity bit in the phase words

struct Shared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accf[kAccBufs];
    uint64_t acce[kAccBufs];
    uint64_t xf;                  // cross-term accumulator complete (MMA -> epilogue)
    uint64_t xe;                  // cross-term accumulator drained (epilogue -> MMA)
    uint32_t taddr;
    int abort_flag;
    int consumed;
};

struct ItemGeo {
    int sub, k, a0, b0, N, R, ntb, n_stage, n_chunk, nkb_stage;
    bool dbl;      // N <= 128: rotating 128-column accumulators, running sums in registers
    bool sep;      // dbl and two planes: cross terms in their own accumulator
    int nbuf;      // accumulators the item rotates over
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
    g.sep = g.dbl && s.spec_lo != nullptr;
    g.nbuf = !g.dbl ? 1 : (g.sep ? 3 : kAccBufs);
    g.ntb = s.n_int / kTbHalf;
    g.nkb_stage = s.ks / kTbHalf;
    g.n_stage = (s.n_int + s.ks - 1) / s.ks;
    g.n_chunk = (s.n_int + s.chunk - 1) / s.chunk;
    return g;
}

// running sum + chunk sum: int32 for int8-valued operands (the FP32 chunk sum is an exact
// integer), FP32 otherwise
__device__ __forceinline__ uint32_t chunk_add(int exact, bool have, uint32_t run, uint32_t v) {
    if (exact) {
        const int x = __float2int_rn(__uint_as_float(v));
        return have ? static_cast<uint32_t>(static_cast<int>(run) + x) : static_cast<uint32_t>(x);
    }
    const float x = __uint_as_float(v);
    return __float_as_uint(have ? __uint_as_float(run) + x : x);
}

// Final sums of Gram row `row`, columns b0 + j0 .. b0 + j0 + 31 (every lane of the warp calls it):
// rows 2i and 2i+1 sit in adjacent lanes.  The even lane writes input pairs (i, j) for the first 8
// column pairs of the piece and the odd lane for the last 8; per column pair each lane sends its
// partner the two sums the partner lacks.
__device__ __forceinline__ void write_piece(const XtSub& s, const ItemGeo& ig, int row, int j0,
                                            const uint32_t (&run)[32]) {
    const int n_bl = s.n_ant * (s.n_ant + 1) / 2, npp = s.n_pol * s.n_pol;
    const bool odd = row & 1;
    const int i = row >> 1;
#pragma unroll
    for (int jh = 0; jh < 8; ++jh) {
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, odd ? run[2 * jh] : run[2 * jh + 16], 1);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, odd ? run[2 * jh + 1] : run[2 * jh + 17], 1);
        const int jp = jh + (odd ? 8 : 0);
        const int j = ((ig.b0 + j0) >> 1) + jp;
        // G[2i][2j], G[2i][2j+1], G[2i+1][2j], G[2i+1][2j+1]
        const uint32_t g_r0c0 = odd ? r0 : run[2 * jh];
        const uint32_t g_r0c1 = odd ? r1 : run[2 * jh + 1];
        const uint32_t g_r1c0 = odd ? run[2 * jh + 16] : r0;
        const uint32_t g_r1c1 = odd ? run[2 * jh + 17] : r1;
        if (i >= s.n_in || j >= s.n_in) continue;
        const int a = i / s.n_pol, pp = i % s.n_pol, a2 = j / s.n_pol, qq = j % s.n_pol;
        if (a > a2) continue;
        const int bl = a * s.n_ant - a * (a - 1) / 2 + (a2 - a);
        const int64_t o = (static_cast<int64_t>(ig.k) * n_bl + bl) * npp + pp * s.n_pol + qq;
        if (s.exact) {
            const float d = s.scale[static_cast<int64_t>(i) * s.n_chan + ig.k] *
                            s.scale[static_cast<int64_t>(j) * s.n_chan + ig.k];
            const int re = static_cast<int>(g_r0c0) + static_cast<int>(g_r1c1);
            const int im = static_cast<int>(g_r1c0) - static_cast<int>(g_r0c1);
            if (s.vis_int) s.vis_int[o] = make_int2(re, im);
            s.vis[o] = make_float2(static_cast<float>(re) / d, static_cast<float>(im) / d);
        } else {
            const float re = __uint_as_float(g_r0c0) + __uint_as_float(g_r1c1);
            const float im = __uint_as_float(g_r1c0) - __uint_as_float(g_r0c1);
            if (s.spec_lo) {
                s.vis[o] = make_float2(re * s.descale, im * s.descale);
            } else {
                const float d = s.scale[static_cast<int64_t>(i) * s.n_chan + ig.k] *
                                s.scale[static_cast<int64_t>(j) * s.n_chan + ig.k];
                s.vis[o] = make_float2(re / d, im / d);
            }
        }
    }
}

// One chunk of a wide item (N > 128, one accumulator at column 0): add this thread's alternate
// 32-column pieces into the running sums at kColRun, or write the final sums after the last
// chunk.  Kept out of line: its registers are not allocated together with the narrow path's.
__device__ __noinline__ void drain_wide(const XtSub& s, const ItemGeo ig, uint32_t tm, int row, int half,
                                        int chunk) {
    const bool last = chunk == ig.n_chunk - 1;
    for (int j0 = 32 * half; j0 < ig.N; j0 += 64) {   // alternate 32-column pieces
        uint32_t v[32], rs[32];
        tmem_ld32(tm + j0, v);
        if (chunk > 0) tmem_ld32(tm + kColRun + j0, rs);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) rs[e] = chunk_add(s.exact, chunk > 0, rs[e], v[e]);
        if (!last) tmem_st32(tm + kColRun + j0, rs);
        else write_piece(s, ig, row, j0, rs);
    }
    if (!last) tmem_wait_st();
}

// run[0..63] (+)= this thread's 64 columns of the accumulator at TMEM address `col`
__device__ __forceinline__ void drain64(uint32_t (&run)[64], uint32_t col, bool have, int exact) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {           // two 32-column loads
        uint32_t v[32];
        tmem_ld32(col + 32 * h, v);
        tmem_wait_ld();
        if (!have) {
#pragma unroll
            for (int e = 0; e < 32; ++e) run[32 * h + e] = chunk_add(exact, false, 0u, v[e]);
        } else if (exact) {
#pragma unroll
            for (int e = 0; e < 32; ++e) run[32 * h + e] = chunk_add(1, true, run[32 * h + e], v[e]);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) run[32 * h + e] = chunk_add(0, true, run[32 * h + e], v[e]);
        }
    }
}

// All chunks of a narrow item (N <= 128): chunk c (global chunk count cc + c) sits in accumulator
// (cc + c) % nbuf; the running sums of this thread's row and 64-column half stay in registers,
// the cross terms of a two-plane item are added at the end, then the sums are written.  `par`
// holds the accumulators' phase bits; the updated bits are returned.  Kept out of line so that
// its registers are allocated apart from the wide path's.
__device__ __noinline__ uint32_t drain_narrow(Shared& sh, const XtSub& s, const ItemGeo ig, uint32_t tm, int row,
                                              int half, int cc, uint32_t par, unsigned* err) {
    const int c0 = 64 * half;
    uint32_t run[64];
#pragma unroll
    for (int e = 0; e < 64; ++e) run[e] = 0u;
    for (int chunk = 0; chunk < ig.n_chunk; ++chunk) {
        const int b = (cc + chunk) % ig.nbuf;
        if (!mbar_wait(&sh.accf[b], (par >> b) & 1, err, ERR_WAIT_MMA)) {
            sh.abort_flag = 1;
            return par;
        }
        par ^= 1u << b;
        tc_fence_after();
        if (c0 < ig.N) drain64(run, tm + b * 128 + c0, chunk > 0, s.exact);
        tc_fence_before();
        mbar_arrive(&sh.acce[b]);             // the accumulator goes back to the MMA issuer
    }
    if (ig.sep) {                             // add the cross terms of the whole integration
        if (!mbar_wait(&sh.xf, (par >> kXBit) & 1, err, ERR_WAIT_MMA)) {
            sh.abort_flag = 1;
            return par;
        }
        par ^= 1u << kXBit;
        tc_fence_after();
        if (c0 < ig.N) drain64(run, tm + kColX + c0, true, 0);
        tc_fence_before();
        mbar_arrive(&sh.xe);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (c0 + 32 * j < ig.N) {
            uint32_t piece[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) piece[e] = run[32 * j + e];
            write_piece(s, ig, row, c0 + 32 * j, piece);
        }
    }
    return par;
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
        for (int b = 0; b < kAccBufs; ++b) {
            mbar_init(&sh.accf[b], 1);
            mbar_init(&sh.acce[b], kEpiThreads);
        }
        mbar_init(&sh.xf, 1);
        mbar_init(&sh.xe, kEpiThreads);
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
                    const int64_t off = (static_cast<int64_t>(ig.k) * ig.ntb + kb0) * ig.R * kTbHalf;
                    mbar_arrive_expect_tx(&sh.full[slot], s.spec_lo ? 2 * bytes : bytes);
                    bulk_g2s(smem + slot * kSlot, s.spec + off, bytes, &sh.full[slot]);
                    if (s.spec_lo)   // the lo plane right after a full stage of hi
                        bulk_g2s(smem + slot * kSlot + ig.nkb_stage * ig.R * 16, s.spec_lo + off, bytes,
                                 &sh.full[slot]);
                }
            }
            // let every issued copy land before the CTA can exit
            for (int q = *(volatile int*)&sh.consumed; q < g; ++q)
                mbar_wait(&sh.full[q % kStages], (q / kStages) & 1, nullptr, 0);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int g = 0, cc = 0;
            uint32_t par = 0;                     // bit b: parity of accumulator b's uses so far
            int prev_nbuf = -1;
            for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
                const ItemGeo ig = item_geo(t, it);
                const XtSub& s = t.sub[ig.sub];
                const uint32_t idesc = idesc_f16_f32(128, ig.N);
                const uint32_t lbo = static_cast<uint32_t>(ig.R) * 16, sbo = 128;
                const int stages_per_chunk = s.chunk / s.ks;
                const bool two = s.spec_lo != nullptr;
                const uint32_t lo_off = static_cast<uint32_t>(ig.nkb_stage) * ig.R * 16;
                bool xfirst = true;                   // next cross-term MMA starts the accumulator
                if (ig.sep) {                         // the previous item's cross terms are drained
                    if (!mbar_wait(&sh.xe, ((par >> kXBit) & 1) ^ 1, t.err, ERR_WAIT_EPI)) {
                        *abort_flag = 1;
                        break;
                    }
                    par ^= 1u << kXBit;
                }
                for (int chunk = 0; chunk < ig.n_chunk && !*abort_flag; ++chunk, ++cc) {
                    const int b = cc % ig.nbuf;
                    // a single-buffered item, or a change of buffering, needs every earlier drain done
                    bool ok = true;
                    if (!ig.dbl || prev_nbuf != ig.nbuf) {
                        for (int q = 0; q < kAccBufs && ok; ++q)
                            ok = mbar_wait(&sh.acce[q], ((par >> q) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                        // (columns 384-511 may have held cross terms; a sep item already waited)
                        if (ok && !ig.sep)
                            ok = mbar_wait(&sh.xe, ((par >> kXBit) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    } else {
                        ok = mbar_wait(&sh.acce[b], ((par >> b) & 1) ^ 1, t.err, ERR_WAIT_EPI);
                    }
                    prev_nbuf = ig.nbuf;
                    if (!ok) {
                        *abort_flag = 1;
                        break;
                    }
                    par ^= 1u << b;
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
                            if (two) {
                                const uint64_t la = smem_desc_noswizzle(kbase + lo_off + ig.a0 * 16, lbo, sbo);
                                const uint64_t lb = smem_desc_noswizzle(kbase + lo_off + ig.b0 * 16, lbo, sbo);
                                const uint32_t xcol = ig.sep ? tmem + kColX : dcol;
                                umma_f16(xcol, da, lb, idesc, (ig.sep && xfirst) ? 0u : 1u);   // H L^T
                                umma_f16(xcol, la, db, idesc, 1u);                              // L H^T
                                xfirst = false;
                            }
                        }
                        umma_commit(&sh.empty[slot]);   // frees the stage once these MMAs finish
                        sh.consumed = g + 1;
                    }
                    if (*abort_flag) break;
                    umma_commit(&sh.accf[b]);           // chunk complete
                }
                if (*abort_flag) break;
                if (ig.sep) umma_commit(&sh.xf);        // cross terms complete
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        const int q = warp & 3;                   // TMEM lane quarter this warp may access
        const int lrow = 32 * q + lane;           // row within the item's 128 rows = TMEM lane
        const int half = (warp - 2) >> 2;         // column half: 64-column halves / alternate 32-column pieces
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        int cc = 0;
        uint32_t par = 0;                         // bit b: parity of accumulator b's uses so far
        for (int it = blockIdx.x; it < t.n_items && !*abort_flag; it += gridDim.x) {
            const ItemGeo ig = item_geo(t, it);
            const XtSub& s = t.sub[ig.sub];
            if (ig.dbl) {
                par = drain_narrow(sh, s, ig, tmem + lane_off, ig.a0 + lrow, half, cc, par, t.err);
                cc += ig.n_chunk;
            } else {
                for (int chunk = 0; chunk < ig.n_chunk; ++chunk, ++cc) {
                    if (!mbar_wait(&sh.accf[0], par & 1, t.err, ERR_WAIT_MMA)) {
                        sh.abort_flag = 1;
                        break;
                    }
                    par ^= 1u;
                    tc_fence_after();
                    drain_wide(s, ig, tmem + lane_off, ig.a0 + lrow, half, chunk);
                    tc_fence_before();
                    mbar_arrive(&sh.acce[0]);
                }
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

int xengine_tc_max_ks(int n_in, int planes) {
    int ks = 512;                                  // stages of at most 512 frames
    while (ks > 16 && planes * (ks / kTbHalf) * 2 * n_in * 16 > kStageMaxBytes) ks /= 2;
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
