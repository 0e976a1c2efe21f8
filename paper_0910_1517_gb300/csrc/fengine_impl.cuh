// fengine_impl.cuh -- the F-engine kernel for 4096-point FFTs (n_chan 2048; smaller FFTs run
// the warp-FFT kernel of fengine_wfft.cuh) and its launcher, included by fengine_wfft.cuh.
//
// One CTA owns a block of F = 4 consecutive frames (F * n_chan = 8192 complex
// channel-frames) and walks over every input (antenna x polarisation) in turn:
//   1. the F frames of input i, offset by its integer delay D_a (Sec. 2.1,
//      Sec. 2.3.2: the read pointer is moved, no data is shifted), arrive in
//      shared memory through one TMA-engine bulk copy, double-buffered so the
//      next input streams in while this one is transformed;
//   2. each frame is an n_fft-point real FFT computed as an M = n_fft/2-point
//      complex FFT of (x[2n] + i x[2n+1]) -- Stockham radix-16/16/R passes, 16
//      points per thread in registers, shared memory between passes -- followed
//      by the even/odd real split; channels 0..M-1 are kept (Nyquist dropped);
//   3. every channel is multiplied by the post-FFT phasor of Eq. 2, the FSTC
//      term exp(+2 pi i k tau_f / N) times the fringe term exp(-i phi_a(g));
//   4. the incoherent beam (sum of g_a^2 |Y|^2) and the coherent voltage sum
//      (sum of g_a e^{i theta} Y, detected once per polarisation) accumulate in
//      the registers of the thread that owns each (frame, channel) point, since
//      this CTA sees every antenna of its frames (Sec. 2.2) -- no atomics;
//   5. each thread writes its (channel, input) pieces of the layout the X-engines
//      read: FP32 4-frame K-blocks straight from registers, or -- FP16 values or
//      requantised int8 bytes, in 8-frame pieces -- through the 2-CTA cluster
//      exchange with the CTA of the neighbouring 4 frames.
#pragma once
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "fengine.cuh"
#include "fft_smem.cuh"

namespace gbx {
namespace {

constexpr int kThreads = 512;
constexpr int kE = 16;                      // complex points per thread per FFT
constexpr int kChanFrames = 8192;           // F * M per CTA
constexpr int kMaxAnt = 128;

template <int M>
struct Plan {
    static constexpr int T = M / kE;                           // threads per FFT
    static constexpr int F = kThreads / T;                     // frames per CTA
    static constexpr int N = 2 * M;                            // real FFT size
    static constexpr int R1 = 16;
    static constexpr int R2 = (M / 16 >= 16) ? 16 : M / 16;
    static constexpr int R3 = M / (R1 * R2);                   // 1 when two passes suffice
    static constexpr int PADM = M + M / 16;                    // padded frame length (float2)
    static constexpr int STAGE = F * N + 32;                   // staging bytes per buffer
    static_assert(F * M == kChanFrames, "CTA covers 8192 channel-frames");
};

// Stockham pass of radix R over span Ns for one frame: read X[b + r*M/R], twiddle by
// W_{Ns R}^{(b mod Ns) r}, DFT, write X[(b/Ns)*Ns*R + b%Ns + r*Ns].  The pass's twiddles are
// tabulated as tw[r*Ns + j] so that a warp's consecutive j read consecutive words.
template <int M, int R, int Ns>
__device__ __forceinline__ void pass_load(const float2* __restrict__ src, const float2* __restrict__ tw, int t,
                                          float2 (&v)[kE]) {
    constexpr int T = M / kE, NB = M / R, PER = kE / R;
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int b = t + m * T;
        if constexpr (NB % 16 == 0) {            // pad16(b + r NB) = pad16(b) + r (NB + NB / 16)
            const float2* s0 = src + pad16(b);
#pragma unroll
            for (int r = 0; r < R; ++r) v[m * R + r] = s0[r * (NB + NB / 16)];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[m * R + r] = src[pad16(b + r * NB)];
        }
        const int j = b % Ns;
#pragma unroll
        for (int r = 1; r < R; ++r) v[m * R + r] = cmul(tw[r * Ns + j], v[m * R + r]);
        Dft<R>::template run<1>(v + m * R);
    }
}

template <int M, int R, int Ns>
__device__ __forceinline__ void pass_store(float2* __restrict__ dst, int t, const float2 (&v)[kE]) {
    constexpr int T = M / kE, PER = kE / R;
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int b = t + m * T;
        const int base = (b / Ns) * Ns * R + (b % Ns);
        if constexpr (Ns % 16 == 0 || (Ns == 1 && R == 16)) {
            // Ns % 16 == 0: pad16(base + r Ns) = pad16(base) + r (Ns + Ns / 16);
            // Ns == 1, R == 16: base = 16 b, so pad16(base + r) = pad16(base) + r
            float2* d0 = dst + pad16(base);
            constexpr int step = (Ns % 16 == 0) ? Ns + Ns / 16 : 1;
#pragma unroll
            for (int r = 0; r < R; ++r) d0[r * step] = v[m * R + r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) dst[pad16(base + r * Ns)] = v[m * R + r];
        }
    }
}

// Split / epilogue geometry: after the FFT every thread takes L consecutive frames (8, or all
// F when fewer) of NP channel pairs (k, M - k), a whole number of K-block runs (TB frames per
// 16-byte row), so that it holds whole (channel, input) pieces of the K-block layout and
// writes each run as one 32-byte sector straight from registers -- no transposition buffer.
// The TPG = L * T threads of a frame group are exactly the FFT groups of its L frames.
template <int M, int MODE>
struct Epi {
    using P = Plan<M>;
    static constexpr int TB = (MODE == OUT_FP32) ? tb_fp32(M) : kTbHalf;
    static constexpr int L = (P::F < 8) ? P::F : 8;      // frames per thread
    // fp16 runs of 8 frames from 4-frame CTAs (n_chan 2048): the two CTAs of a cluster (consecutive
    // frame blocks) trade halves of their channels through distributed shared memory, so that each
    // writes whole 32-byte pieces (8 frames x re, im) of its half of the channels
    static constexpr bool kPair = (M == 2048 && MODE != OUT_FP32);
    static_assert(M == 2048 && L == 4, "this kernel runs the 4096-point FFTs (4-frame CTAs); smaller ones run fengine_wfft.cuh's");
    static_assert(MODE != OUT_F32Q, "the channel-quad FP32 layout comes from the warp-FFT kernel");
    static_assert(L % TB == 0 || L < TB, "whole K-block runs, or part of one when F < TB");
    static constexpr int NP = kE / (2 * L);                // channel pairs per thread
    static constexpr int TPG = L * P::T;                   // threads per frame group
    static_assert(2 * NP * L == kE && NP * TPG == M / 2, "split covers every channel of every frame once");
};

template <int M>
struct Smem {
    using P = Plan<M>;
    static constexpr int kTw = P::R2 * 16 + (P::R3 > 1 ? P::R3 * 16 * P::R2 : 0) + M / 2 + 1;
    static constexpr int kTab = 2 * M + P::F;                          // [pf M | wcoh M | ff F] of one antenna
    static constexpr size_t stage = 0;
    static constexpr size_t X = stage + 2 * static_cast<size_t>(P::STAGE);
    static constexpr size_t tw = X + sizeof(float2) * P::F * P::PADM;
    static constexpr size_t tab = ((tw + sizeof(float2) * kTw + 127) / 128) * 128;   // 2 bulk-copy targets
    // cluster-pair exchange buffer (n_chan 2048): [4 slots (re, im) x (rank 0, 1)][M/2 channels] of 4
    // fp16 frames (8 bytes): a warp's writes and reads of consecutive channels are conflict-free
    static constexpr size_t xch = ((tab + 2 * sizeof(float2) * kTab + 127) / 128) * 128;
    static constexpr size_t total = xch + (M == 2048 ? static_cast<size_t>(M / 2) * 32 : 0);
    static_assert(total <= 232448, "F-engine shared memory exceeds 227 KB");
    static_assert(X % 16 == 0 && tab % 16 == 0 && (sizeof(float2) * kTab) % 16 == 0 && P::STAGE % 16 == 0,
                  "bulk-copy targets are 16-byte aligned");
};

// Per-CTA control words kept in static shared memory by the kernel that runs the body.
struct FeCtl {
    uint64_t bar[2];
    uint64_t tbar[2];
    int abort_flag;
    uint64_t xfull;            // paired CTAs: the partner's half of this input's exchange has landed
    uint64_t xempty;           // paired CTAs: the partner has read its exchange buffer (we may write it)
    int Ds[kMaxAnt];           // integer delays, read every iteration
};

__device__ __forceinline__ uint32_t pack_half2(__half lo, __half hi) {
    return static_cast<uint32_t>(__half_as_ushort(lo)) | (static_cast<uint32_t>(__half_as_ushort(hi)) << 16);
}

// The F-engine work of one CTA: frame block `block` of the integration described by p.
template <int M, int MODE>
__device__ __forceinline__ void fengine_cta(const FeParams& p, int block, FeCtl& ctl) {
    using P = Plan<M>;
    using S = Smem<M>;
    using E = Epi<M, MODE>;
    constexpr int T = P::T, F = P::F, N = P::N;
    constexpr int Ns3 = P::R1 * P::R2;
    constexpr int TB = E::TB, L = E::L, NP = E::NP, TPG = E::TPG;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage0 = smem + S::stage;
    float2* X = reinterpret_cast<float2*>(smem + S::X);           // F * PADM
    float2* tw2 = reinterpret_cast<float2*>(smem + S::tw);       // [R2][16]
    float2* tw3 = tw2 + P::R2 * 16;                               // [R3][Ns3]
    float2* twN = tw3 + (P::R3 > 1 ? P::R3 * Ns3 : 0);            // [M/2 + 1]
    float2* tab = reinterpret_cast<float2*>(smem + S::tab);      // 2 x [pf | wcoh | ff] of one antenna
    uint64_t* bar = ctl.bar;
    uint64_t* tbar = ctl.tbar;
    int& abort_flag = ctl.abort_flag;
    int* Ds = ctl.Ds;

    const int tid = threadIdx.x;
    const int f = tid / T;            // frame of this thread's FFT group
    const int t = tid % T;            // thread within the FFT group
    const int fg = tid / TPG;         // frame group of the split: frames fg*L .. fg*L + L - 1
    const int kk = tid % TPG;         // channel pairs kk + q*TPG, q < NP
    const int t0 = block * F;
    if (t0 >= p.n_int) return;        // no frames left (never in a cluster-paired launch)
    const int n_fr = min(F, p.n_int - t0);
    const bool live = fg * L < n_fr;  // n_fr is a multiple of L: whole frame groups are live or not
    constexpr bool kPair = E::kPair;
    unsigned char* xch = smem + S::xch;
    const uint32_t rank = kPair ? cluster_ctarank() : 0;   // frames 4 rank .. of the pair's 8
    const int R = 2 * p.n_in;
    const int64_t ntb = p.n_int / TB;

    // this thread's channels, fixed for the CTA; the K-block of its frames starts at element
    // (ch * ntb + kb) * rows * TB of the spectra
    int chs[2 * NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const int k = kk + q * TPG;
        chs[2 * q] = k;
        chs[2 * q + 1] = (k == 0) ? M / 2 : M - k;
    }
    const int kb_run = (t0 + fg * L) / TB;
    const int64_t blk_elems = static_cast<int64_t>((MODE == OUT_FP32) ? rows_fp32(p.n_in) : R) * TB;

    // beam accumulators of this thread's L x 2 NP points: the incoherent sum over every input,
    // and the coherent voltage sum of the current polarisation.  Frames go in pairs: a float2
    // holds one component of frames 2j and 2j + 1, so one packed FP32x2 instruction does both.
    constexpr int LP = L / 2;
    float2 incr[LP][2 * NP];
    float2 cre[LP][2 * NP], cim[LP][2 * NP];
#pragma unroll
    for (int j = 0; j < LP; ++j)
#pragma unroll
        for (int c = 0; c < 2 * NP; ++c) {
            incr[j][c] = make_float2(0.0f, 0.0f);
            cre[j][c] = make_float2(0.0f, 0.0f);
            cim[j][c] = make_float2(0.0f, 0.0f);
        }

    for (int m = tid; m < S::kTw; m += kThreads) tw2[m] = p.tw[m];
    for (int m = tid; m < p.n_ant; m += kThreads) Ds[m] = p.D[m];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&tbar[0], 1);
        mbar_init(&tbar[1], 1);
        if constexpr (kPair) {
            mbar_init(&ctl.xfull, 1);
            mbar_init(&ctl.xempty, 1);
        }
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    // Paired CTAs trade channel halves each input: the partner's 4-frame halves of the channels
    // this CTA writes arrive by st.async, completing bytes on xfull; before writing into the
    // partner's buffer a CTA waits on xempty, which the partner's arrive completes once it has
    // read that buffer.  All waits are bounded; one cluster barrier at exit keeps both CTAs
    // resident while the other may still write into them.
    // partner's re + im halves of our channels: 4 frames of fp16 (16 bytes), or of int8 (8 bytes)
    constexpr uint32_t kXBytes = (M / 2) * (MODE == OUT_I8B ? 8 : 16);
    uint32_t peer_xfull = 0, peer_xempty = 0;
    if constexpr (kPair) {
        cluster_sync();                                  // both CTAs and their barriers exist
        peer_xfull = cluster_map(&ctl.xfull, rank ^ 1u);
        peer_xempty = cluster_map(&ctl.xempty, rank ^ 1u);
        if (tid == 0) {
            mbar_arrive_expect_tx(&ctl.xfull, kXBytes);  // input 0's exchange
            mbar_arrive_remote(peer_xempty);             // the partner may write into our buffer
        }
    }

    const int n_iter = p.n_in;  // polarisation-major order: it = pol * n_ant + a
    // Called by all of warp 0: lane 0 issues the bulk copy of the F frames of input `it`
    // (offset by its integer delay); bytes past the last 16-byte boundary are copied by the
    // lanes only when rounding the copy up would read past the row's readable samples.
    auto issue = [&](int it) {
        const int pol = it / p.n_ant, a = it % p.n_ant;
        const int i = a * p.n_pol + pol;
        unsigned char* dst = stage0 + (it & 1) * P::STAGE;
        const int64_t s0 = static_cast<int64_t>(t0) * N + Ds[a];
        const int64_t aligned = s0 & ~static_cast<int64_t>(15);
        const int64_t end = s0 + static_cast<int64_t>(n_fr) * N;
        const int64_t up = (end + 15) & ~static_cast<int64_t>(15);
        const int64_t bulk_end = up <= p.n_avail ? up : (end & ~static_cast<int64_t>(15));
        const uint32_t bulk = static_cast<uint32_t>(bulk_end - aligned);
        const int8_t* row = p.x + static_cast<int64_t>(i) * p.ld;
        const int lane = tid & 31;
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[it & 1], bulk);
            bulk_g2s(dst, row + aligned, bulk, &bar[it & 1]);
        }
        const int64_t q = bulk_end + lane;
        if (q < end) dst[q - aligned] = static_cast<unsigned char>(row[q]);
    };
    // phasor, beam-weight and fringe rows of the antenna of input `it` (n_fr fringe phasors:
    // n_fr * 8 bytes is a multiple of 16 since n_fr is F or a multiple of 16)
    auto issue_tab = [&](int it) {
        const int a = it % p.n_ant;
        float2* dst = tab + (it & 1) * S::kTab;
        uint64_t* tb = &tbar[it & 1];
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(tb, (2 * M + n_fr) * sizeof(float2));
        bulk_g2s(dst, p.pf + static_cast<int64_t>(a) * M, M * sizeof(float2), tb);
        bulk_g2s(dst + M, p.wcoh + static_cast<int64_t>(a) * M, M * sizeof(float2), tb);
        bulk_g2s(dst + 2 * M, p.ff + static_cast<int64_t>(a) * p.n_int + t0, n_fr * sizeof(float2), tb);
    };
    __syncthreads();                 // Ds visible to warp 0
    if (tid < 32) issue(0);
    if (tid == 0) issue_tab(0);

    int it = 0;
    for (; it < n_iter; ++it) {
        const int pol = it / p.n_ant, a = it % p.n_ant;
        const int i = a * p.n_pol + pol;
        if (tid < 32 && it + 1 < n_iter) issue(it + 1);
        const float g2 = p.ginc[a];
        float scv[2 * NP];           // requantisation scales of this thread's channels
        if constexpr (MODE != OUT_FP32) {
#pragma unroll
            for (int c = 0; c < 2 * NP; ++c) scv[c] = p.scale[static_cast<int64_t>(i) * M + chs[c]];
        }
        if (!mbar_wait(&bar[it & 1], (it >> 1) & 1, p.err, ERR_WAIT_STAGE)) abort_flag = 1;
        const int64_t s0 = static_cast<int64_t>(t0) * N + Ds[a];
        const unsigned char* st = stage0 + (it & 1) * P::STAGE + (s0 & 15) + f * N;
        float2* Xf = X + f * P::PADM;

        // ---- pass 1: radix-16 straight from the int8 staging buffer (z[n] = x[2n] + i x[2n+1])
        float2 v[kE];
        {
            constexpr int NB = M / P::R1;
            if ((s0 & 1) == 0) {                       // pairs are 2-byte aligned: one load each
                const uint16_t* st16 = reinterpret_cast<const uint16_t*>(st);
#pragma unroll
                for (int r = 0; r < kE; ++r) {
                    v[r] = pair_u16(st16[t + r * NB]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < kE; ++r) {
                    const int n = t + r * NB;
                    v[r] = pair_u16(st[2 * n] | (static_cast<uint32_t>(st[2 * n + 1]) << 8));
                }
            }
            Dft<16>::template run<1>(v);
        }
        __syncthreads();  // the previous iteration's split has finished reading X and its antenna tables
        if (abort_flag) break;
        if (kPair && tid == 0 && it > 0) {               // every thread has read the last exchange
            mbar_arrive_expect_tx(&ctl.xfull, kXBytes);
            mbar_arrive_remote(peer_xempty);
        }
        if (tid == 0 && it + 1 < n_iter) issue_tab(it + 1);   // into the buffer that split just released
        pass_store<M, P::R1, 1>(Xf, t, v);
        group_sync<T>(f);
        // ---- pass 2
        pass_load<M, P::R2, P::R1>(Xf, tw2, t, v);
        group_sync<T>(f);
        pass_store<M, P::R2, P::R1>(Xf, t, v);
        // ---- pass 3
        if constexpr (P::R3 > 1) {
            group_sync<T>(f);
            pass_load<M, P::R3, Ns3>(Xf, tw3, t, v);
            group_sync<T>(f);
            pass_store<M, P::R3, Ns3>(Xf, t, v);
        }
        __syncthreads();  // every frame's FFT is in X: the split reads the frames of its group

        // ---- real split, Eq. 2 phasor (fractional delay x fringe), beams, K-block stores
        if (!mbar_wait(&tbar[it & 1], (it >> 1) & 1, p.err, ERR_WAIT_STAGE)) abort_flag = 1;
        const float2* pfa = tab + (it & 1) * S::kTab;
        const float2* wa = pfa + M;
        const float2* fra = pfa + 2 * M;   // fringe phasors of the CTA's frames
        if constexpr (kPair) {   // the partner has read its exchange buffer: this input's halves may go in
            if (!mbar_wait_cluster(&ctl.xempty, it & 1, p.err, ERR_WAIT_STAGE)) abort_flag = 1;
        }
        if (live) {
        // component l of a frame-paired value: frame l (0 .. L - 1)
        auto comp = [](const float2 (&v)[LP], int l) { return (l & 1) ? v[l >> 1].y : v[l >> 1].x; };
        // beams and the K-block store of channel c from its L frames (yr, yi: frame pairs)
        auto emit = [&](int c, const float2 (&yr)[LP], const float2 (&yi)[LP]) {
            const float2 w = wa[chs[c]];
            const float2 wx = make_float2(w.x, w.x), wy = make_float2(w.y, w.y), nwy = make_float2(-w.y, -w.y);
            const float2 g22 = make_float2(g2, g2);
#pragma unroll
            for (int j = 0; j < LP; ++j) {
                incr[j][c] = __ffma2_rn(g22, __ffma2_rn(yr[j], yr[j], __fmul2_rn(yi[j], yi[j])), incr[j][c]);
                if (a == 0) {
                    cre[j][c] = make_float2(0.0f, 0.0f);
                    cim[j][c] = make_float2(0.0f, 0.0f);
                }
                cre[j][c] = __ffma2_rn(nwy, yi[j], __ffma2_rn(wx, yr[j], cre[j][c]));
                cim[j][c] = __ffma2_rn(wy, yr[j], __ffma2_rn(wx, yi[j], cim[j][c]));
                if (a == p.n_ant - 1) {  // this polarisation's coherent sum is complete: detect
                    const float2 pw = __ffma2_rn(cim[j][c], cim[j][c], __fmul2_rn(cre[j][c], cre[j][c]));
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        float* bc = p.beams + (static_cast<int64_t>(p.n_int) + t0 + fg * L + 2 * j + h) * M + chs[c];
                        const float v = h ? pw.y : pw.x;
                        *bc = (pol == 0) ? v : *bc + v;
                    }
                }
            }
            const int64_t blk = (static_cast<int64_t>(chs[c]) * ntb + kb_run) * blk_elems;
            if constexpr (MODE == OUT_FP32) {
                // 4-frame K-blocks: one 32-byte piece per (channel, input), rows 2i and 2i + 1 as
                // neighbouring granules, in the order the XOR placement of row group G gives them
                const int G = (2 * i) >> 3;
                const int pos = ((2 * i) & 7) ^ (G & 7);
                const bool flip = pos & 1;
                uint32_t u[8];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const uint32_t re = __float_as_uint(comp(yr, l)), im = __float_as_uint(comp(yi, l));
                    u[l] = flip ? im : re;
                    u[4 + l] = flip ? re : im;
                }
                st_global_v8(static_cast<float*>(p.spec) + blk + G * 32 + (pos & ~1) * 4, u);
            } else if constexpr (MODE == OUT_I8B) {
                // int8 bytes (the channel-quad piece i8q_piece: 8 re then 8 im bytes): this CTA's
                // 4 frames go, as one 8-byte word (re 4 | im 4), to slot `rank` of the exchange
                // buffer of the pair's CTA that writes channel ch (rank 0: channels < M/2)
                uint32_t wv[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // h = 0 re, 1 im
                    int qv[4];
#pragma unroll
                    for (int l = 0; l < 4; ++l) qv[l] = max(-127, min(127, __float2int_rn((h ? comp(yi, l) : comp(yr, l)) * scv[c])));
                    wv[h] = __byte_perm(__byte_perm(qv[0], qv[1], 0x0040), __byte_perm(qv[2], qv[3], 0x0040), 0x5410);
                }
                const int ch = chs[c];
                const uint32_t owner = ch < M / 2 ? 0u : 1u;
                unsigned char* d = xch + (static_cast<size_t>(rank) * (M / 2) + ch % (M / 2)) * 8;
                if (owner == rank)
                    *reinterpret_cast<uint2*>(d) = make_uint2(wv[0], wv[1]);
                else
                    st_async_v2(cluster_map(d, owner), wv[0], wv[1], peer_xfull);
            } else {
                // fp16: the 4-frame halves of the 8-frame run go into the exchange buffer of the CTA
                // of the pair that writes this channel (rank 0: channels < M/2): slot 2c + rank
                // (c = 0 re, 1 im), word ch % (M/2)
                __half hr[4], hi[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    hr[l] = __float2half_rn(comp(yr, l) * scv[c]);
                    hi[l] = __float2half_rn(comp(yi, l) * scv[c]);
                }
                const int ch = chs[c];
                const uint32_t owner = ch < M / 2 ? 0u : 1u;
                unsigned char* dre = xch + (static_cast<size_t>(rank) * (M / 2) + ch % (M / 2)) * 8;
                unsigned char* dim = dre + static_cast<size_t>(M) * 8;
                const uint2 vr = make_uint2(pack_half2(hr[0], hr[1]), pack_half2(hr[2], hr[3]));
                const uint2 vi = make_uint2(pack_half2(hi[0], hi[1]), pack_half2(hi[2], hi[3]));
                if (owner == rank) {
                    *reinterpret_cast<uint2*>(dre) = vr;
                    *reinterpret_cast<uint2*>(dim) = vi;
                } else {
                    st_async_v2(cluster_map(dre, owner), vr.x, vr.y, peer_xfull);
                    st_async_v2(cluster_map(dim, owner), vi.x, vi.y, peer_xfull);
                }
            }
        };
        // ---- real split and Eq. 2 phasor.  With zk = Z[k], zm = Z[M - k]:
        //   2 X[k] = E + Q, 2 X[M - k] = conj(E - Q), E = zk + conj(zm), Q = (-i W_N^k)(zk - conj(zm));
        //   Y = X pf fr = ((2 X) (pf / 2)) fr.  Pair 0: 2 X[0] = 2 (Re + Im of Z[0]), 2 X[M/2] = 2 conj(Z[M/2]).
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int k = chs[2 * q], kc = chs[2 * q + 1];
            const float2 w = twN[k];
            const float2 wnx = make_float2(w.y, w.y), wny = make_float2(-w.x, -w.x), nwny = make_float2(w.x, w.x);
            const float2 hk = pfa[k], hm = pfa[kc];
            const float2 pkx = make_float2(0.5f * hk.x, 0.5f * hk.x), pky = make_float2(0.5f * hk.y, 0.5f * hk.y);
            const float2 npky = make_float2(-0.5f * hk.y, -0.5f * hk.y);
            const float2 pmx = make_float2(0.5f * hm.x, 0.5f * hm.x), pmy = make_float2(0.5f * hm.y, 0.5f * hm.y);
            const float2 npmy = make_float2(-0.5f * hm.y, -0.5f * hm.y);
            float2 ykr[LP], yki[LP], ymr[LP], ymi[LP];
#pragma unroll
            for (int j = 0; j < LP; ++j) {
                const int f0 = fg * L + 2 * j;
                const float2* X0 = X + f0 * P::PADM;
                const float2* X1 = X0 + P::PADM;
                const float2 a0 = X0[pad16(k)], a1 = X1[pad16(k)], b0 = X0[pad16(kc)], b1 = X1[pad16(kc)];
                const float2 zkr = make_float2(a0.x, a1.x), zki = make_float2(a0.y, a1.y);
                const float2 zmr = make_float2(b0.x, b1.x), zmi = make_float2(b0.y, b1.y);
                float2 xkr, xki, xmr, xmi;     // 2 X[k], 2 X[M - k]
                if (k == 0) {
                    xkr = __fmul2_rn(make_float2(2.0f, 2.0f), __fadd2_rn(zkr, zki));     // DC
                    xki = make_float2(0.0f, 0.0f);
                    xmr = __fmul2_rn(make_float2(2.0f, 2.0f), zmr);                     // channel M/2
                    xmi = __fmul2_rn(make_float2(-2.0f, -2.0f), zmi);
                } else {
                    const float2 er = __fadd2_rn(zkr, zmr), ei = psub(zki, zmi);
                    const float2 dr = psub(zkr, zmr), di = __fadd2_rn(zki, zmi);
                    const float2 qr = __ffma2_rn(nwny, di, __fmul2_rn(wnx, dr));
                    const float2 qi = __ffma2_rn(wny, dr, __fmul2_rn(wnx, di));
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
                const float2 r0 = fra[f0], r1 = fra[f0 + 1];
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
        }  // live
        if constexpr (kPair) {
            // our halves are in (local stores, barrier) and the partner's have landed (xfull): write
            // this CTA's half of the channels as whole 8-frame pieces (rows 2i, 2i+1: 32 bytes)
            __syncthreads();
            if (!mbar_wait_cluster(&ctl.xfull, it & 1, p.err, ERR_WAIT_STAGE)) abort_flag = 1;
            const int64_t kb8 = (t0 - 4 * static_cast<int>(rank)) / TB;
            const uint2* xw = reinterpret_cast<const uint2*>(xch);   // [slot][M/2]
            if constexpr (MODE == OUT_I8B) {
                // slots 0, 1: (re 4 | im 4) of frames 0-3 and 4-7; one 16-byte piece per channel,
                // consecutive channels' pieces contiguous within a channel quad
                int8_t* spec = static_cast<int8_t*>(p.spec);
                for (int j = tid; j < M / 2; j += kThreads) {
                    const int ch = static_cast<int>(rank) * (M / 2) + j;
                    const uint2 b0 = xw[j], b1 = xw[M / 2 + j];
                    *reinterpret_cast<uint4*>(spec + i8q_piece(ch, kb8, i, ntb, p.n_in)) = make_uint4(b0.x, b1.x, b0.y, b1.y);
                }
            } else {
                __half* spec = static_cast<__half*>(p.spec);
                for (int j = tid; j < M / 2; j += kThreads) {
                    const int ch = static_cast<int>(rank) * (M / 2) + j;
                    const uint2 r0 = xw[j], r1 = xw[M / 2 + j], i0 = xw[M + j], i1 = xw[3 * (M / 2) + j];
                    const uint32_t u[8] = {r0.x, r0.y, r1.x, r1.y, i0.x, i0.y, i1.x, i1.y};
                    st_global_v8(spec + (static_cast<int64_t>(ch) * ntb + kb8) * blk_elems + 2 * i * TB, u);
                }
            }
        }
    }

    // incoherent beam of this thread's points
    __syncthreads();
    if (!abort_flag) {
        if (live) {
#pragma unroll
            for (int l = 0; l < L; ++l)
#pragma unroll
                for (int c = 0; c < 2 * NP; ++c)
                    p.beams[static_cast<int64_t>(t0 + fg * L + l) * M + chs[c]] = (l & 1) ? incr[l >> 1][c].y : incr[l >> 1][c].x;
        }
    } else if (tid == 0) {
        // copies issued ahead of an aborted iteration must land before the CTA exits: the
        // stages of iterations it and it + 1, and the antenna tables of iterations it - 1 and it
        mbar_wait(&bar[it & 1], (it >> 1) & 1, nullptr, 0);
        if (it + 1 < n_iter) mbar_wait(&bar[(it + 1) & 1], ((it + 1) >> 1) & 1, nullptr, 0);
        if (it > 0) mbar_wait(&tbar[(it - 1) & 1], ((it - 1) >> 1) & 1, nullptr, 0);
        mbar_wait(&tbar[it & 1], (it >> 1) & 1, nullptr, 0);
    }
    if constexpr (kPair) cluster_sync();   // neither CTA leaves while the other may still write into it
}

template <int M, int MODE>
__global__ void __launch_bounds__(kThreads, 1) fengine_kernel(const FeParams p) {
    __shared__ __align__(8) FeCtl ctl;
    fengine_cta<M, MODE>(p, blockIdx.x, ctl);
}

template <int M, int MODE>
cudaError_t launch_t(const FeParams& p, cudaStream_t s) {
    using P = Plan<M>;
    const size_t smem = Smem<M>::total;
    cudaError_t e = cudaFuncSetAttribute(fengine_kernel<M, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int grid = (p.n_int + P::F - 1) / P::F;
    if constexpr (Epi<M, MODE>::kPair) {
        // clusters of two consecutive frame blocks (grid is even: n_int is a multiple of 16)
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
        e = cudaLaunchKernelEx(&cfg, fengine_kernel<M, MODE>, p);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    fengine_kernel<M, MODE><<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace
}  // namespace gbx
