// fengine_wfft.cuh -- the F-engine for n_chan <= 1024 (n_fft <= 2048): warp-specialised, one
// warp per FFT group, two radix-32 passes; included by fengine.cu after fengine_impl.cuh.
//
// Same work and outputs as the kernel of fengine_impl.cuh (Sec. 2.1 FX chain, Eq. 2 phasor,
// Sec. 2.2 beams), organised to cut instructions and shared-memory traffic and to keep both
// halves of the work in flight at once:
//   * a CTA owns F = 8192 / M consecutive frames and walks over every input (the beams need
//     every antenna of a frame in one CTA);
//   * warps 0-7 (the FFT group, 104 or 80 registers a thread, WRegs) transform the frames of input it:
//     the M-point complex FFT of a frame (z[n] = x[2n] + i x[2n+1], M = 32 P) is a four-step
//     FFT inside one warp -- lane l takes column n = l + 32 m of each of the warp's G = 32 / P
//     frames, P-point DFTs in registers straight from the int8 staging buffer, the twiddle
//     W_M^(l k1), one transpose through the warp's own shared-memory region (__syncwarp), then
//     lane (g, k1) a 32-point DFT in registers: Z[k1 + P k2] -- and leave the results in the
//     region in natural order;
//   * warps 8-15 (the epilogue group, 152 or 176 registers a thread) meanwhile take input it - 1: each
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
constexpr int kWRegs = 128;                    // registers a thread at launch (512 x 128)

// Registers a thread of each group after setmaxnreg, for 256 + 256 threads = 512 x kWRegs: the
// 1024-point FFT group takes 104 (with 80 the int8 GMRT-scale kernel ran 15 % slower, though
// spill-free); below that 80 / 176, which removes the 60-200 bytes a thread the smaller sizes'
// epilogues spilled with 104 / 152 (measured 4-7 % faster at 256 and 512 points)
template <int M, int MODE>
struct WRegs {
    static constexpr bool kWide = M == 1024;
    static constexpr int FFT = kWide ? 104 : 80;
    static constexpr int EPI = kWide ? 152 : 176;
    static_assert(FFT * kWFftWarps * 32 + EPI * kWEpiThreads == kWRegs * kWThreads, "the launch's registers, split");
};

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
    using P = WPlan<M>;
    using S = WSmem<M>;
    constexpr int PP = P::P, G = P::G, F = P::F, N = P::N, L = P::L;
    constexpr int TB = (MODE == OUT_FP32) ? tb_fp32(M) : kTbHalf;
    static_assert(TB == 8, "8-frame K-block runs");
    static_assert(MODE != OUT_F32Q || M >= 32, "channel quads");
    __shared__ __align__(8) WCtl ctl;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage0 = smem + S::stage;
    float2* Xbuf = reinterpret_cast<float2*>(smem + S::X);          // [2][8 warps][REG]
    float2* tw1 = reinterpret_cast<float2*>(smem + S::tw);         // [P / 2][32][2]
    float2* twN = tw1 + S::kTw1;                                    // [M/2 + 1]
    float2* tab = reinterpret_cast<float2*>(smem + S::tab);        // 2 x [pf | wcoh | ff]
    volatile int* abort_flag = &ctl.abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t0 = blockIdx.x * F;
    const int n_fr = min(F, p.n_int - t0);
    const int n_iter = p.n_in;                // polarisation-major: it = pol * n_ant + a

    const float2* twsrc = p.tw + fengine_tw_wfft_offset(N);
    for (int m = tid; m < S::kTw1 + S::kTwN; m += kWThreads) tw1[m] = twsrc[m];
    for (int m = tid; m < p.n_ant; m += kWThreads) ctl.Ds[m] = p.D[m];
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl.bar[b], 1);
            mbar_init(&ctl.tbar[b], 1);
            mbar_init(&ctl.full[b], kWFftWarps);
            mbar_init(&ctl.empty[b], kWEpiThreads / 32);
        }
        fence_mbar_init();
        ctl.abort_flag = 0;
    }
    __syncthreads();

    if (warp < kWFftWarps) {
        // ================================================================ FFT group
        reg_dealloc<WRegs<M, MODE>::FFT>();
        // lane 0 of warp 0 issues the bulk copy of the F frames of input `it` (offset by its
        // integer delay); bytes past the last 16-byte boundary are copied by the lanes only when
        // rounding the copy up would read past the row's readable samples
        auto issue = [&](int it) {
            const int pol = it / p.n_ant, a = it % p.n_ant;
            const int i = a * p.n_pol + pol;
            unsigned char* dst = stage0 + (it & 1) * P::STAGE;
            const int64_t s0 = static_cast<int64_t>(t0) * N + ctl.Ds[a];
            const int64_t aligned = s0 & ~static_cast<int64_t>(15);
            const int64_t end = s0 + static_cast<int64_t>(n_fr) * N;
            const int64_t up = (end + 15) & ~static_cast<int64_t>(15);
            const int64_t bulk_end = up <= p.n_avail ? up : (end & ~static_cast<int64_t>(15));
            const uint32_t bulk = static_cast<uint32_t>(bulk_end - aligned);
            const int8_t* row = p.x + static_cast<int64_t>(i) * p.ld;
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&ctl.bar[it & 1], bulk);
                bulk_g2s(dst, row + aligned, bulk, &ctl.bar[it & 1]);
            }
            const int64_t q = bulk_end + lane;
            if (q < end) dst[q - aligned] = static_cast<unsigned char>(row[q]);
        };
        // phasor, beam-weight and fringe rows of the antenna of input `it` (n_fr * 8 bytes of
        // fringe phasors: a multiple of 16 since n_fr is a multiple of 16 or F)
        auto issue_tab = [&](int it) {
            const int a = it % p.n_ant;
            float2* dst = tab + (it & 1) * S::kTab;
            uint64_t* tb = &ctl.tbar[it & 1];
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(tb, (2 * M + n_fr) * sizeof(float2));
            bulk_g2s(dst, p.pf + static_cast<int64_t>(a) * M, M * sizeof(float2), tb);
            bulk_g2s(dst + M, p.wcoh + static_cast<int64_t>(a) * M, M * sizeof(float2), tb);
            bulk_g2s(dst + 2 * M, p.ff + static_cast<int64_t>(a) * p.n_int + t0, n_fr * sizeof(float2), tb);
        };
        if (warp == 0) issue(0);
        int staged = 1, tabbed = 0;           // copies issued so far (staging buffers, tables)
        for (int it = 0; it < n_iter; ++it) {
            const int b = it & 1;
            // every FFT warp is done with input it - 1: its staging buffer takes input it + 1.  The
            // barrier also takes the decision to stop (the OR of every FFT thread's view of the abort
            // flag), so that the whole group leaves together.
            if (named_bar_or(1, kWFftWarps * 32, *abort_flag != 0)) break;
            if (warp == 0 && it + 1 < n_iter) {
                issue(it + 1);
                staged = it + 2;
            }
            // region set b and tables b: the epilogue has finished input it - 2
            bool ok = it < 2 || mbar_wait(&ctl.empty[b], ((it - 2) >> 1) & 1, p.err, ERR_WAIT_EPI);
            if (ok && tid == 0) {
                issue_tab(it);
                tabbed = it + 1;
            }
            ok = ok && mbar_wait(&ctl.bar[b], (it >> 1) & 1, p.err, ERR_WAIT_STAGE);
            // a timed-out wait stops the CTA at the next barrier; this pass runs on whatever the
            // buffers hold (every address is data-independent), so no thread leaves the group alone
            if (!ok) *abort_flag = 1;
            const int a = it % p.n_ant;
            const int64_t s0 = static_cast<int64_t>(t0) * N + ctl.Ds[a];
            float2* Rw = Xbuf + b * (kWFftWarps * P::REG) + warp * P::REG;   // this warp's region
            // ---- pass 1: lane = column l of each of the warp's G frames, P-point DFTs
            const unsigned char* st = stage0 + b * P::STAGE + (s0 & 15) + warp * G * N;
            float2 v[32];
            if ((s0 & 1) == 0) {               // pairs are 2-byte aligned: one load each
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const uint16_t* s16 = reinterpret_cast<const uint16_t*>(st + g * N);
#pragma unroll
                    for (int m = 0; m < PP; ++m) v[g * PP + m] = pair_u16(s16[lane + 32 * m]);
                }
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int m = 0; m < PP; ++m) {
                        const unsigned char* q = st + g * N + 2 * (lane + 32 * m);
                        v[g * PP + m] = pair_u16(q[0] | (static_cast<uint32_t>(q[1]) << 8));
                    }
            }
            // the twiddle W_M^(l k1), k1 >= 1 (pairs of k1 in one 16-byte load), then the transpose
            // through the warp's region (row r = g P + k1, column l; rows of 34 points, so a lane
            // reads its row 16 bytes at a time without bank conflicts)
            auto twiddle_transpose = [&]() {
#pragma unroll
                for (int j = 0; 2 * j + 1 < PP; ++j) {   // (P = 1: no twiddle)
                    const float4 w = reinterpret_cast<const float4*>(tw1)[j * 32 + lane];
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        if (j > 0) v[g * PP + 2 * j] = cmul(make_float2(w.x, w.y), v[g * PP + 2 * j]);
                        if (2 * j + 1 < PP) v[g * PP + 2 * j + 1] = cmul(make_float2(w.z, w.w), v[g * PP + 2 * j + 1]);
                    }
                }
#pragma unroll
                for (int r = 0; r < 32; ++r) Rw[r * P::RS + lane] = v[r];
                __syncwarp();
                const float4* row = reinterpret_cast<const float4*>(Rw + lane * P::RS);
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const float4 q = row[n];
                    v[2 * n] = make_float2(q.x, q.y);
                    v[2 * n + 1] = make_float2(q.z, q.w);
                }
                __syncwarp();
            };
            {
#pragma unroll
                for (int g = 0; g < G; ++g) Dft<PP>::template run<1>(v + g * PP);
                twiddle_transpose();
                // ---- pass 2: lane = (g, k1), 32-point DFT over the columns: Z_g[k1 + P k2]
                Dft<32>::template run<1>(v);
            }
            float2* o = Rw + (lane / PP) * P::S + (lane % PP);
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) o[PP * k2] = v[k2];
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl.full[b]);
        }
        if (*abort_flag && tid == 0) {
            // copies issued and not yet seen to land must land before the CTA exits
            for (int q = max(0, staged - 2); q < staged; ++q) mbar_wait(&ctl.bar[q & 1], (q >> 1) & 1, nullptr, 0);
            for (int q = max(0, tabbed - 2); q < tabbed; ++q) mbar_wait(&ctl.tbar[q & 1], (q >> 1) & 1, nullptr, 0);
        }
    } else {
        // ================================================================ epilogue group
        reg_alloc<WRegs<M, MODE>::EPI>();
        const int e = tid - kWFftWarps * 32;
        const int fg = e / P::SLOTS, ps = e % P::SLOTS;
        const bool live = fg * L < n_fr;      // n_fr is a multiple of 8: whole frame groups
        const int R = 2 * p.n_in;
        const int64_t ntb = p.n_int / TB;
        const int kb_run = (t0 + fg * L) / TB;
        const int64_t blk_elems = static_cast<int64_t>((MODE == OUT_FP32) ? rows_fp32(p.n_in) : R) * TB;
        // channels of this thread: pairs (ps, M - ps) (pair 0 = (0, M/2)) and (ps + M/4, M - ps - M/4)
        int chs[4];
        chs[0] = ps;
        chs[1] = (ps == 0) ? M / 2 : M - ps;
        chs[2] = ps + M / 4;
        chs[3] = M - ps - M / 4;
        // Frames go in pairs: a float2 holds one component (real or imaginary part) of frames
        // 2j and 2j + 1, so one packed FP32x2 instruction does the arithmetic of both frames.
        // -i W_N^k of the two pairs (the real split below works on 2 X), as broadcast pairs
        float2 wnx[2], wny[2], nwny[2];        // -i W_N^k = (w.y, -w.x), w = W_N^k
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float2 w = twN[chs[2 * q]];
            wnx[q] = make_float2(w.y, w.y);
            wny[q] = make_float2(-w.x, -w.x);
            nwny[q] = make_float2(w.x, w.x);
        }
        constexpr int LP = L / 2;              // frame pairs per thread
        float2 incr[LP][4];                    // incoherent beam
        float2 cre[LP][4], cim[LP][4];         // coherent sum of the current polarisation
#pragma unroll
        for (int j = 0; j < LP; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                incr[j][c] = make_float2(0.0f, 0.0f);
                cre[j][c] = make_float2(0.0f, 0.0f);
                cim[j][c] = make_float2(0.0f, 0.0f);
            }
        for (int it = 0; it < n_iter; ++it) {
            const int b = it & 1;
            const int pol = it / p.n_ant, a = it % p.n_ant;
            const int i = a * p.n_pol + pol;
            const float g2 = p.ginc[a];
            const float2 g22 = make_float2(g2, g2);
            float scv[4];                      // requantisation scales of this thread's channels
            if constexpr (MODE == OUT_F16 || MODE == OUT_I8B) {
#pragma unroll
                for (int c = 0; c < 4; ++c) scv[c] = p.scale[static_cast<int64_t>(i) * M + chs[c]];
            }
            // every lane waits; the warp goes on only if all of them saw both copies land and no
            // abort (a warp-uniform decision: the stores below trade values between lanes)
            bool ok = *abort_flag == 0 && mbar_wait(&ctl.full[b], (it >> 1) & 1, p.err, ERR_WAIT_EPI) &&
                      mbar_wait(&ctl.tbar[b], (it >> 1) & 1, p.err, ERR_WAIT_STAGE);
            if (!__all_sync(0xffffffffu, ok)) {
                *abort_flag = 1;
                break;
            }
            const float2* Xi = Xbuf + b * (kWFftWarps * P::REG);
            const float2* pfa = tab + b * S::kTab;
            const float2* wa = pfa + M;
            const float2* fra = pfa + 2 * M;   // fringe phasors of the CTA's frames
            const bool detect = a == p.n_ant - 1;   // this polarisation's coherent sums are complete
            // every lane computes (the FP32 stores trade values between lanes, and `live` is not
            // warp-uniform when a warp spans several frame groups); only live lanes write
            constexpr int PG = TB / 2;
            const int Gr = (2 * i) >> 3, sgr = Gr & 7;
            const int pstart = Gr * 8 * TB + ((((i & 3) ^ (sgr / PG)) * PG) << 2);   // floats from the block start
            // y of frame l, channel slot: real / imaginary part
            auto comp = [](const float2 (&v)[LP], int l) { return (l & 1) ? v[l >> 1].y : v[l >> 1].x; };
            auto emit = [&](int c, const float2 (&yr)[LP], const float2 (&yi)[LP]) {
                const float2 w = wa[chs[c]];
                const float2 wx = make_float2(w.x, w.x), wy = make_float2(w.y, w.y), nwy = make_float2(-w.y, -w.y);
#pragma unroll
                for (int j = 0; j < LP; ++j) {
                    incr[j][c] = __ffma2_rn(g22, __ffma2_rn(yr[j], yr[j], __fmul2_rn(yi[j], yi[j])), incr[j][c]);
                    cre[j][c] = __ffma2_rn(nwy, yi[j], __ffma2_rn(wx, yr[j], cre[j][c]));
                    cim[j][c] = __ffma2_rn(wy, yr[j], __ffma2_rn(wx, yi[j], cim[j][c]));
                }
                if (detect) {                  // detect, add the polarisations, start the next sum
#pragma unroll
                    for (int j = 0; j < LP; ++j) {
                        const float2 pw = __ffma2_rn(cim[j][c], cim[j][c], __fmul2_rn(cre[j][c], cre[j][c]));
                        cre[j][c] = make_float2(0.0f, 0.0f);
                        cim[j][c] = make_float2(0.0f, 0.0f);
                        if (live) {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float* bc = p.beams + (static_cast<int64_t>(p.n_int) + t0 + fg * L + 2 * j + h) * M + chs[c];
                                const float v = h ? pw.y : pw.x;
                                *bc = (pol == 0) ? v : *bc + v;
                            }
                        }
                    }
                }
                if constexpr (MODE == OUT_F32Q) {
                    // the channel-quad layout: this lane's own 64-byte piece, two 32-byte stores; the lanes
                    // of consecutive channels fill whole 256-byte quads
                    float* o = static_cast<float*>(p.spec) + f32q_piece(chs[c], kb_run, i, ntb, p.n_in);
                    uint32_t u[8];
#pragma unroll
                    for (int l = 0; l < 8; ++l) u[l] = __float_as_uint(comp(yr, l));
                    if (live) st_global_v8(o, u);
#pragma unroll
                    for (int l = 0; l < 8; ++l) u[l] = __float_as_uint(comp(yi, l));
                    if (live) st_global_v8(o + 8, u);
                } else if constexpr (MODE == OUT_I8B) {
                    // rows 2i (real) and 2i + 1 (imaginary) of the K-block, 8 int8 frames each: one
                    // 16-byte piece of the channel-quad byte layout (the lanes of consecutive channels
                    // fill whole 64-byte runs)
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {   // h = 2 comp + half: frames 4 (h & 1) .. + 3
                        int qv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int l = 4 * (h & 1) + e;
                            const float x = ((h >> 1) ? comp(yi, l) : comp(yr, l)) * scv[c];
                            qv[e] = max(-127, min(127, __float2int_rn(x)));
                        }
                        w[h] = __byte_perm(__byte_perm(qv[0], qv[1], 0x0040), __byte_perm(qv[2], qv[3], 0x0040), 0x5410);
                    }
                    int8_t* o = static_cast<int8_t*>(p.spec) + i8q_piece(chs[c], kb_run, i, ntb, p.n_in);
                    if (live) *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
                } else if constexpr (MODE == OUT_FP32) {
                    // 64-byte piece of (channel, input): granule slot (2 comp + half) ^ (sgr & 3); each lane
                    // pair writes one piece per instruction, trading the component each needs by a shuffle
                    float* spec = static_cast<float*>(p.spec);
                    const bool odd = ps & 1;
                    const int cA = (sgr >> 1) & 1;
                    const bool hswap = sgr & 1;
                    const int chp = __shfl_xor_sync(0xffffffffu, chs[c], 1);
                    const int csend = odd ? cA : 1 - cA;
                    float mine[8], recv[8];
#pragma unroll
                    for (int l = 0; l < 8; ++l) {
                        const float own_keep = (odd ? 1 - cA : cA) ? comp(yi, l) : comp(yr, l);
                        const float own_send = csend ? comp(yi, l) : comp(yr, l);
                        mine[l] = own_keep;
                        recv[l] = __shfl_xor_sync(0xffffffffu, own_send, 1);
                    }
                    auto put = [&](int ch, const float (&v)[8]) {
                        uint32_t u[8];
#pragma unroll
                        for (int l = 0; l < 4; ++l) {
                            u[l] = __float_as_uint(hswap ? v[4 + l] : v[l]);
                            u[4 + l] = __float_as_uint(hswap ? v[l] : v[4 + l]);
                        }
                        if (live)
                            st_global_v8(spec + (static_cast<int64_t>(ch) * ntb + kb_run) * blk_elems + pstart + (odd ? 8 : 0), u);
                    };
                    float d0[8], d1[8];
#pragma unroll
                    for (int l = 0; l < 8; ++l) {
                        d0[l] = odd ? recv[l] : mine[l];
                        d1[l] = odd ? mine[l] : recv[l];
                    }
                    put(odd ? chp : chs[c], d0);
                    put(odd ? chs[c] : chp, d1);
                } else {
                    __half hr[L], hi[L];
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        const float xr = comp(yr, l) * scv[c], xi = comp(yi, l) * scv[c];
                        hr[l] = __float2half_rn(xr);
                        hi[l] = __float2half_rn(xi);
                    }
                    __half* o = static_cast<__half*>(p.spec) + (static_cast<int64_t>(chs[c]) * ntb + kb_run) * blk_elems +
                                2 * i * TB;
                    uint32_t u[8];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        u[m] = pack_half2(hr[2 * m], hr[2 * m + 1]);
                        u[4 + m] = pack_half2(hi[2 * m], hi[2 * m + 1]);
                    }
                    if (live) st_global_v8(o, u);
                }
            };
            // ---- real split and Eq. 2 phasor.  With zk = Z[k], zm = Z[M - k]:
            //   2 X[k] = E + Q, 2 X[M - k] = conj(E - Q), E = zk + conj(zm), Q = (-i W_N^k)(zk - conj(zm));
            //   Y = X pf fr = ((2 X) (pf / 2)) fr.  Pair 0: 2 X[0] = 2 (Re + Im of Z[0]), 2 X[M/2] = 2 conj(Z[M/2]).
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = chs[2 * q], kc = chs[2 * q + 1];
                const float2 hk = pfa[k], hm = pfa[kc];
                const float2 pkx = make_float2(0.5f * hk.x, 0.5f * hk.x), pky = make_float2(0.5f * hk.y, 0.5f * hk.y);
                const float2 npky = make_float2(-0.5f * hk.y, -0.5f * hk.y);
                const float2 pmx = make_float2(0.5f * hm.x, 0.5f * hm.x), pmy = make_float2(0.5f * hm.y, 0.5f * hm.y);
                const float2 npmy = make_float2(-0.5f * hm.y, -0.5f * hm.y);
                float2 ykr[LP], yki[LP], ymr[LP], ymi[LP];
#pragma unroll
                for (int j = 0; j < LP; ++j) {
                    const int f0 = fg * L + 2 * j, f1 = f0 + 1;
                    const float2* X0 = Xi + (f0 / G) * P::REG + (f0 % G) * P::S;
                    const float2* X1 = Xi + (f1 / G) * P::REG + (f1 % G) * P::S;
                    const float2 a0 = X0[k], a1 = X1[k], b0 = X0[kc], b1 = X1[kc];
                    const float2 zkr = make_float2(a0.x, a1.x), zki = make_float2(a0.y, a1.y);
                    const float2 zmr = make_float2(b0.x, b1.x), zmi = make_float2(b0.y, b1.y);
                    float2 xkr, xki, xmr, xmi;     // 2 X[k], 2 X[M - k]
                    if (q == 0 && ps == 0) {
                        xkr = __fmul2_rn(make_float2(2.0f, 2.0f), __fadd2_rn(zkr, zki));     // DC
                        xki = make_float2(0.0f, 0.0f);
                        xmr = __fmul2_rn(make_float2(2.0f, 2.0f), zmr);                     // channel M/2
                        xmi = __fmul2_rn(make_float2(-2.0f, -2.0f), zmi);
                    } else {
                        const float2 er = __fadd2_rn(zkr, zmr), ei = psub(zki, zmi);
                        const float2 dr = psub(zkr, zmr), di = __fadd2_rn(zki, zmi);
                        const float2 qr = __ffma2_rn(nwny[q], di, __fmul2_rn(wnx[q], dr));
                        const float2 qi = __ffma2_rn(wny[q], dr, __fmul2_rn(wnx[q], di));
                        xkr = __fadd2_rn(er, qr);
                        xki = __fadd2_rn(ei, qi);
                        xmr = psub(er, qr);
                        xmi = psub(qi, ei);
                    }
                    // u = (2 X) (pf / 2), then y = u fr
                    const float2 ukr = __ffma2_rn(npky, xki, __fmul2_rn(pkx, xkr));
                    const float2 uki = __ffma2_rn(pky, xkr, __fmul2_rn(pkx, xki));
                    const float2 umr = __ffma2_rn(npmy, xmi, __fmul2_rn(pmx, xmr));
                    const float2 umi = __ffma2_rn(pmy, xmr, __fmul2_rn(pmx, xmi));
                    const float2 r0 = fra[f0], r1 = fra[f1];
                    const float2 frr = make_float2(r0.x, r1.x), fri = make_float2(r0.y, r1.y);
                    const float2 nfri = make_float2(-r0.y, -r1.y);
                    ykr[j] = __ffma2_rn(uki, nfri, __fmul2_rn(ukr, frr));
                    yki[j] = __ffma2_rn(uki, frr, __fmul2_rn(ukr, fri));
                    ymr[j] = __ffma2_rn(umi, nfri, __fmul2_rn(umr, frr));
                    ymi[j] = __ffma2_rn(umi, frr, __fmul2_rn(umr, fri));
                }
                emit(2 * q, ykr, yki);
                emit(2 * q + 1, ymr, ymi);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl.empty[b]);   // region set b and tables b may be reused
        }
        // incoherent beam of this thread's points
        if (!*abort_flag && live) {
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    p.beams[static_cast<int64_t>(t0 + fg * L + l) * M + chs[c]] = (l & 1) ? incr[l >> 1][c].y : incr[l >> 1][c].x;
        }
    }
}

template <int M, int MODE>
cudaError_t launch_w(const FeParams& p, cudaStream_t s) {
    using P = WPlan<M>;
    const size_t smem = WSmem<M>::total;
    // the register split (setmaxnreg) hands the FFT group's registers to the epilogue group: it
    // needs exactly the 512 x 128 registers of the launch, or the epilogue warps would wait for
    // registers that never come -- refuse to launch otherwise
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fengine_w_kernel<M, MODE>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != kWRegs) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(fengine_w_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (p.n_int + P::F - 1) / P::F;
    fengine_w_kernel<M, MODE><<<grid, kWThreads, smem, s>>>(p);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_w_mode(const FeParams& p, cudaStream_t s) {
    if constexpr (MODE == OUT_F32Q || MODE == OUT_I8B) {   // n_chan 32 .. 1024 (int8 bytes: .. 2048)
        switch (p.n_chan) {
            case 32: return launch_w<32, MODE>(p, s);
            case 64: return launch_w<64, MODE>(p, s);
            case 128: return launch_w<128, MODE>(p, s);
            case 256: return launch_w<256, MODE>(p, s);
            case 512: return launch_w<512, MODE>(p, s);
            case 1024: return launch_w<1024, MODE>(p, s);
            case 2048:   // 4-frame CTAs in cluster pairs: the kernel of fengine_impl.cuh
                if constexpr (MODE == OUT_I8B) return launch_t<2048, MODE>(p, s);
                return cudaErrorInvalidValue;
            default: return cudaErrorInvalidValue;
        }
    } else {
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
}

}  // namespace
}  // namespace gbx
