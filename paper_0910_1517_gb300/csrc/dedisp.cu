// dedisp.cu -- coherent dedispersion of the phased-array voltage beam (Sec. 5): the beam's
// voltage spectra (n_chan channels per frame, two polarisations) are turned back into the
// complex baseband series by an inverse FFT per frame, the series is multiplied in the Fourier
// domain by the inverse ISM chirp over overlapping blocks of M = F n_chan samples
// (overlap-save, the first S = (F - O) n_chan samples of each block kept), and both
// polarisations are detected, added and averaged over `avg` samples.
//
// The per-frame inverse FFT and the M-point FFTs share one four-step factorisation, M = F x
// n_chan (sample n = n_chan l + m of a block: frame l, sample m of the frame; frequency
// j = k1 + F k2), so that a block costs three passes over HBM:
//   A  per channel k: F-point DFT over the block's frames l         -> W[k1][k]
//   B  per row k1:    inverse n_chan-point DFT over k (the frames' inverse FFTs, all at once),
//                     twiddle W_M^{m k1}, n_chan-point DFT over m   -> spectrum X[k1 + F k2];
//                     times the chirp; inverse DFT over k2, twiddle W_M^{-n k1} -> W[k1][n]
//   C  per column n:  inverse F-point DFT over k1 -> y[n_chan l + n] for the kept frames l,
//                     |y_X|^2 + |y_Y|^2 summed over the CTA's columns -> P[col group][l]
//   D  per frame:     the column-group sums of each `avg`-sample window, scaled to a mean.
// A and C keep two channels (four sequences: 2 x polarisation) per CTA, B one row per
// polarisation group; every FFT runs in padded shared memory (smem_fft).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/corr.h"
#include "common.cuh"
#include "fft_smem.cuh"
#include "handle.cuh"

namespace gbx {

std::vector<float2> smem_fft_twiddles(int L) {
    const int R2 = (L / 16 >= 16) ? 16 : L / 16, R3 = L / (16 * R2), Ns3 = 16 * R2;
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<float2> tw;
    auto w = [&](double num, double den) {
        return make_float2(static_cast<float>(std::cos(two_pi * num / den)),
                           static_cast<float>(-std::sin(two_pi * num / den)));
    };
    for (int r = 0; r < R2; ++r)
        for (int j = 0; j < 16; ++j) tw.push_back(w(static_cast<double>(j) * r, 16.0 * R2));
    if (R3 > 1)
        for (int r = 0; r < R3; ++r)
            for (int j = 0; j < Ns3; ++j) tw.push_back(w(static_cast<double>(j) * r, static_cast<double>(L)));
    return tw;
}

namespace {

constexpr double kDispConst = 4.148808e3;   // s MHz^2 pc^-1 cm^3: delay = D DM / nu^2
// channels (A) / columns (C) per CTA: two, so that each frame's read or write is one whole
// 32-byte sector (one channel per CTA measured slower at 4096 frames, despite two CTAs per SM)
__host__ __device__ constexpr int col_g(int) { return 2; }

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }


// W_M^{p} = exp(-2 pi i p / M) for 0 <= p < M (M a power of two: 2p / M is exact)
__device__ __forceinline__ float2 twiddle_m(int p, float inv_half_m) {
    float s, c;
    sincospif(static_cast<float>(p) * inv_half_m, &s, &c);
    return make_float2(c, -s);
}

struct DdBlocks {
    const float4* ring;     // [cap][n_chan] voltage spectra (X re, X im, Y re, Y im)
    int64_t cap;            // frames in the ring
    int64_t start0;         // ring frame of block 0's first frame
    int step;               // frames between blocks (F - O)
    float2* work;           // [n_blocks][F][n_chan] float4 as pairs: pol X then pol Y per element
    float* part;            // [n_blocks][n_chan / col_g(F)][keep] detected column-group sums
    int keep;               // frames kept per block (F - O)
};

// A: per channel, the F-point DFT over the block's frames.  Groups g = 2 kk + pol.
template <int F>
__global__ void __launch_bounds__(2 * col_g(F) * SmemFft<F>::T, (2 * col_g(F) * SmemFft<F>::T <= 512) ? 2 : 1)
dd_pass_a(DdBlocks d, int n_chan, const float2* __restrict__ tw) {
    using P = SmemFft<F>;
    constexpr int kColG = col_g(F);
    extern __shared__ float2 sm[];
    const int g = threadIdx.x / P::T, t = threadIdx.x % P::T;
    const int k0 = blockIdx.x * kColG, blk = blockIdx.y;
    int64_t f0 = d.start0 + static_cast<int64_t>(blk) * d.step;
    if (f0 >= d.cap) f0 -= d.cap;
    for (int i = threadIdx.x; i < F * kColG; i += blockDim.x) {
        const int l = i / kColG, kk = i % kColG;
        int64_t f = f0 + l;
        if (f >= d.cap) f -= d.cap;
        const float4 v = __ldg(d.ring + f * n_chan + k0 + kk);
        sm[(2 * kk) * P::PAD + pad16(l)] = make_float2(v.x, v.y);
        sm[(2 * kk + 1) * P::PAD + pad16(l)] = make_float2(v.z, v.w);
    }
    __syncthreads();
    smem_fft<F>(sm + g * P::PAD, tw, t, g, [](int, float2 x) { return x; });
    __syncthreads();
    float4* out = reinterpret_cast<float4*>(d.work) + static_cast<int64_t>(blk) * F * n_chan;
    for (int i = threadIdx.x; i < F * kColG; i += blockDim.x) {
        const int k1 = i / kColG, kk = i % kColG;
        const float2 x = sm[(2 * kk) * P::PAD + pad16(k1)], y = sm[(2 * kk + 1) * P::PAD + pad16(k1)];
        out[static_cast<int64_t>(k1) * n_chan + k0 + kk] = make_float4(x.x, x.y, y.x, y.y);
    }
}

// B: per row k1, the frames' inverse FFTs, the twiddle, the spectrum, the chirp and the first
// half of the inverse transform, in place.  Inverse DFTs run as conj(DFT(conj(.))), the
// conjugations folded into the element-wise steps.  RB rows per CTA, groups g = 2 row + pol.
template <int NC, int RB>
__global__ void __launch_bounds__(2 * RB * SmemFft<NC>::T, (2 * RB * SmemFft<NC>::T <= 256) ? 2 : 1)
dd_pass_b(float2* __restrict__ work, int F, const float2* __restrict__ chirp, const float2* __restrict__ tw,
          float inv_half_m) {
    using P = SmemFft<NC>;
    extern __shared__ float2 sm[];
    float2* trow = sm + 2 * RB * P::PAD;             // [RB][NC] W_M^{m k1} of the CTA's rows
    float2* crows = trow + RB * NC;                  // [RB][NC] the rows' chirp
    const int g = threadIdx.x / P::T, t = threadIdx.x % P::T;
    const int row0 = blockIdx.x * RB, blk = blockIdx.y;
    float4* rows = reinterpret_cast<float4*>(work) + (static_cast<int64_t>(blk) * F + row0) * NC;
    for (int i = threadIdx.x; i < RB * NC; i += blockDim.x) {
        const int r = i / NC, k = i % NC;
        const float4 v = rows[static_cast<int64_t>(r) * NC + k];
        sm[(2 * r) * P::PAD + pad16(k)] = make_float2(v.x, -v.y);           // conj: inverse DFT
        sm[(2 * r + 1) * P::PAD + pad16(k)] = make_float2(v.z, -v.w);
        trow[i] = twiddle_m(k * (row0 + r), inv_half_m);
        crows[i] = __ldg(chirp + static_cast<int64_t>(row0) * NC + i);
    }
    __syncthreads();
    float2* buf = sm + g * P::PAD;
    const float2* tr = trow + (g / 2) * NC;
    const float2* crow = crows + (g / 2) * NC;
    // a = DFT(conj V) = conj(n_chan x~); next input n_chan x~ W^{m k1} = conj(a) W^{m k1}
    smem_fft<NC>(buf, tw, t, g, [=](int m, float2 a) { return cmul(conjf2(a), tr[m]); });
    // X at k2; next input conj(X C)
    smem_fft<NC>(buf, tw, t, g, [=](int k2, float2 x) { return conjf2(cmul(x, crow[k2])); });
    // c = DFT(conj Y) = conj(inverse DFT of Y); keep conj(c) W^{-n k1} = conj(c W^{n k1})
    smem_fft<NC>(buf, tw, t, g, [=](int n, float2 c) { return conjf2(cmul(c, tr[n])); });
    __syncthreads();
    for (int i = threadIdx.x; i < RB * NC; i += blockDim.x) {
        const int r = i / NC, n = i % NC;
        const float2 x = sm[(2 * r) * P::PAD + pad16(n)], y = sm[(2 * r + 1) * P::PAD + pad16(n)];
        rows[static_cast<int64_t>(r) * NC + n] = make_float4(x.x, x.y, y.x, y.y);
    }
}

// C: per column n, the inverse F-point DFT over k1 (conj(DFT(conj))), then the detected power
// of the kept frames summed over the CTA's columns and both polarisations.
template <int F>
__global__ void __launch_bounds__(2 * col_g(F) * SmemFft<F>::T, (2 * col_g(F) * SmemFft<F>::T <= 512) ? 2 : 1)
dd_pass_c(DdBlocks d, int n_chan, const float2* __restrict__ tw, float scale) {
    using P = SmemFft<F>;
    constexpr int kColG = col_g(F);
    extern __shared__ float2 sm[];
    const int g = threadIdx.x / P::T, t = threadIdx.x % P::T;
    const int n0 = blockIdx.x * kColG, blk = blockIdx.y;
    const float4* in = reinterpret_cast<const float4*>(d.work) + static_cast<int64_t>(blk) * F * n_chan;
    for (int i = threadIdx.x; i < F * kColG; i += blockDim.x) {
        const int k1 = i / kColG, kk = i % kColG;
        const float4 v = in[static_cast<int64_t>(k1) * n_chan + n0 + kk];
        sm[(2 * kk) * P::PAD + pad16(k1)] = make_float2(v.x, -v.y);
        sm[(2 * kk + 1) * P::PAD + pad16(k1)] = make_float2(v.z, -v.w);
    }
    __syncthreads();
    smem_fft<F>(sm + g * P::PAD, tw, t, g, [](int, float2 x) { return x; });
    __syncthreads();
    float* part = d.part + (static_cast<int64_t>(blk) * (n_chan / kColG) + blockIdx.x) * d.keep;
    for (int l = threadIdx.x; l < d.keep; l += blockDim.x) {
        float p = 0.0f;
#pragma unroll
        for (int q = 0; q < 2 * kColG; ++q) {
            const float2 y = sm[q * P::PAD + pad16(l)];
            const float a = y.x * scale, b = y.y * scale;
            p = fmaf(a, a, fmaf(b, b, p));
        }
        part[l] = p;
    }
}

// D: window means from the column-group sums part[blk][c][l] (G columns per group).
// Windows inside a frame (avg < n_chan): one thread per (block, window, frame), consecutive
// threads on consecutive frames (coalesced reads).  Whole-frame windows: a CTA takes 32 frames
// (lanes) and its 8 warps split the column groups; the warps' partial sums are added in order
// in shared memory, then over the avg / n_chan frames of a window by shuffles.
__global__ void dd_pass_d_in_frame(const float* __restrict__ part, int n_blocks, int keep, int n_chan, int G,
                                   int avg, float* __restrict__ out) {
    const int n_cg = n_chan / G, nw = n_chan / avg, per = avg / G;
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<int64_t>(n_blocks) * nw * keep) return;
    const int l = static_cast<int>(i % keep);
    const int w = static_cast<int>((i / keep) % nw);
    const int blk = static_cast<int>(i / (static_cast<int64_t>(keep) * nw));
    const float* pp = part + (static_cast<int64_t>(blk) * n_cg + static_cast<int64_t>(w) * per) * keep + l;
    float s = 0.0f;
    for (int c = 0; c < per; ++c) s += pp[static_cast<int64_t>(c) * keep];
    out[(static_cast<int64_t>(blk) * keep + l) * nw + w] = s * (1.0f / static_cast<float>(avg));
}

__global__ void __launch_bounds__(256) dd_pass_d_frames(const float* __restrict__ part, int keep, int n_chan, int G,
                                                        int avg, float* __restrict__ out) {
    __shared__ float red[8][32];
    const int n_cg = n_chan / G, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int blk = blockIdx.y, l = blockIdx.x * 32 + lane;
    const int c0 = w * (n_cg / 8), c1 = c0 + n_cg / 8;
    float s = 0.0f;
    if (l < keep) {
        const float* pp = part + static_cast<int64_t>(blk) * n_cg * keep + l;
        for (int c = c0; c < c1; ++c) s += pp[static_cast<int64_t>(c) * keep];
    }
    red[w][lane] = s;
    __syncthreads();
    if (w != 0) return;
    s = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += red[q][lane];
    const int fr = avg / n_chan;             // frames per window: a power of two <= 32, divides keep
    for (int o = fr / 2; o > 0; o /= 2) s += __shfl_down_sync(0xffffffffu, s, o, fr);
    if (l < keep && (l % fr) == 0)
        out[(static_cast<int64_t>(blk) * keep + l) / fr] = s * (1.0f / static_cast<float>(avg));
}

template <int F>
cudaError_t launch_ac(bool c_pass, const DdBlocks& d, int n_chan, int n_blocks, const float2* tw, float scale,
                      cudaStream_t s) {
    using P = SmemFft<F>;
    constexpr int kColG = col_g(F);
    const size_t smem = static_cast<size_t>(2 * kColG) * P::PAD * sizeof(float2);
    const dim3 grid(n_chan / kColG, n_blocks), block(2 * kColG * P::T);
    if (!c_pass) {
        cudaError_t e = cudaFuncSetAttribute(dd_pass_a<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        dd_pass_a<F><<<grid, block, smem, s>>>(d, n_chan, tw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(dd_pass_c<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        dd_pass_c<F><<<grid, block, smem, s>>>(d, n_chan, tw, scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_ac_any(int F, bool c_pass, const DdBlocks& d, int n_chan, int n_blocks, const float2* tw,
                          float scale, cudaStream_t s) {
    switch (F) {
        case 256: return launch_ac<256>(c_pass, d, n_chan, n_blocks, tw, scale, s);
        case 512: return launch_ac<512>(c_pass, d, n_chan, n_blocks, tw, scale, s);
        case 1024: return launch_ac<1024>(c_pass, d, n_chan, n_blocks, tw, scale, s);
        case 2048: return launch_ac<2048>(c_pass, d, n_chan, n_blocks, tw, scale, s);
        case 4096: return launch_ac<4096>(c_pass, d, n_chan, n_blocks, tw, scale, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int NC>
cudaError_t launch_b(float2* work, int F, int n_blocks, const float2* chirp, const float2* tw, float inv_half_m,
                     cudaStream_t s) {
    using P = SmemFft<NC>;
    constexpr int RB = (2 * P::T >= 256) ? 1 : 256 / (2 * P::T);   // at least 256 threads a CTA
    const size_t smem = (static_cast<size_t>(2 * RB) * P::PAD + static_cast<size_t>(2 * RB) * NC) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(dd_pass_b<NC, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const dim3 grid(F / RB, n_blocks), block(2 * RB * P::T);
    dd_pass_b<NC, RB><<<grid, block, smem, s>>>(work, F, chirp, tw, inv_half_m);
    return cudaGetLastError();
}

cudaError_t launch_b_any(int NC, float2* work, int F, int n_blocks, const float2* chirp, const float2* tw,
                         float inv_half_m, cudaStream_t s) {
    switch (NC) {
        case 64: return launch_b<64>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 128: return launch_b<128>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 256: return launch_b<256>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 512: return launch_b<512>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 1024: return launch_b<1024>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 2048: return launch_b<2048>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        case 4096: return launch_b<4096>(work, F, n_blocks, chirp, tw, inv_half_m, s);
        default: return cudaErrorInvalidValue;
    }
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace gbx

using namespace gbx;

struct corr_dd {
    int dev = 0;
    int n_chan = 0, F = 0, O = 0, max_push = 0, avg = 0;
    double dm = 0, f_lo = 0, bw = 0;
    int64_t cap = 0, wpos = 0, have = 0;    // ring: frames stored, next write frame, frames unconsumed
    int max_blocks = 0;
    float4* ring = nullptr;
    float2* work = nullptr;
    float* part = nullptr;
    float2* chirp = nullptr;                // [F][n_chan]: C[k1 + F k2] at [k1][k2]
    float2* tw_f = nullptr;                 // smem_fft twiddles for F and n_chan points
    float2* tw_c = nullptr;
    // stage timing (corr_dd_set_timing): events around the ring copy and passes A-D of a push
    bool timing = false;
    cudaEvent_t ev[6] = {};
    double stage_ms[5] = {};
    int timed = 0;
};

namespace {
int ddfail(int code, const char* msg) { return fail_code(code, msg); }
#define DDCU(call)                                                           \
    do {                                                                     \
        if ((call) != cudaSuccess) return ddfail(CORR_E_CUDA, #call);        \
    } while (0)

void dd_free(corr_dd* d) {
    void* bufs[] = {d->ring, d->work, d->part, d->chirp, d->tw_f, d->tw_c};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t e : d->ev)
        if (e) cudaEventDestroy(e);
    delete d;
}
}  // namespace

extern "C" {

double corr_dd_smear_samples(double dm, double f_lo, double bw) {
    if (!(f_lo > 0) || !(bw > 0)) return -1.0;
    return kDispConst * dm * (1.0 / (f_lo * f_lo) - 1.0 / ((f_lo + bw) * (f_lo + bw))) * bw * 1e6;
}

int corr_dd_create(corr_dd_t** out, int n_chan, int fft_frames, int overlap_frames, int max_push_frames, double dm,
                   double f_lo, double bw, int avg) {
    if (!out) return ddfail(CORR_E_INVAL, "null output pointer");
    *out = nullptr;
    if (!pow2_in(n_chan, 64, 4096)) return ddfail(CORR_E_INVAL, "n_chan must be a power of two in [64, 4096]");
    if (!pow2_in(fft_frames, 256, 4096)) return ddfail(CORR_E_INVAL, "fft_frames must be a power of two in [256, 4096]");
    if (static_cast<int64_t>(fft_frames) * n_chan > (int64_t(1) << 24))
        return ddfail(CORR_E_INVAL, "fft_frames * n_chan must be <= 2^24");
    if (overlap_frames < 0 || overlap_frames >= fft_frames)
        return ddfail(CORR_E_INVAL, "overlap_frames must be in [0, fft_frames)");
    if (max_push_frames < 1) return ddfail(CORR_E_INVAL, "max_push_frames must be >= 1");
    if (!(f_lo > 0) || !(bw > 0) || !(dm >= 0) || !std::isfinite(dm))
        return ddfail(CORR_E_INVAL, "need f_lo > 0, bw > 0 (an upper-sideband band) and dm >= 0");
    const int keep = fft_frames - overlap_frames;
    const int64_t S = static_cast<int64_t>(keep) * n_chan;
    if (avg < 2 || (avg & (avg - 1)) || avg > 32 * n_chan || S % avg)
        return ddfail(CORR_E_INVAL, "avg must be a power of two in [2, 32 n_chan] dividing (fft_frames - overlap) n_chan");
    if (corr_dd_smear_samples(dm, f_lo, bw) > static_cast<double>(overlap_frames) * n_chan)
        return ddfail(CORR_E_RANGE, "overlap_frames * n_chan is below the dispersion smear across the band");
    corr_dd* d = new corr_dd();
    cudaGetDevice(&d->dev);
    d->n_chan = n_chan;
    d->F = fft_frames;
    d->O = overlap_frames;
    d->max_push = max_push_frames;
    d->avg = avg;
    d->dm = dm;
    d->f_lo = f_lo;
    d->bw = bw;
    d->cap = static_cast<int64_t>(fft_frames) + max_push_frames;
    d->max_blocks = max_push_frames / keep + 1;
    const int64_t M = static_cast<int64_t>(fft_frames) * n_chan;
    auto bad = [&](const char* what) {
        dd_free(d);
        return ddfail(CORR_E_CUDA, what);
    };
    if (cudaMalloc(&d->ring, d->cap * n_chan * sizeof(float4)) != cudaSuccess) return bad("cudaMalloc(ring)");
    if (cudaMalloc(&d->work, static_cast<size_t>(d->max_blocks) * M * sizeof(float4)) != cudaSuccess)
        return bad("cudaMalloc(work)");
    if (cudaMalloc(&d->part, static_cast<size_t>(d->max_blocks) * (n_chan / col_g(fft_frames)) * keep * sizeof(float)) !=
        cudaSuccess)
        return bad("cudaMalloc(part)");
    // the chirp, FP64 phase reduced to [0, 1) cycles before rounding, stored [k1][k2]
    std::vector<float2> ch(static_cast<size_t>(M));
    const double nu_ref = f_lo + bw, two_pi = 6.283185307179586476925286766559;
    for (int64_t j = 0; j < M; ++j) {
        const double nu = f_lo + static_cast<double>(j) * (bw / static_cast<double>(M));
        const double df = nu - nu_ref;
        const double cyc = 1e6 * kDispConst * dm * df * df / (nu_ref * nu_ref * nu);
        const double ph = -two_pi * (cyc - std::floor(cyc));
        const int64_t k1 = j % fft_frames, k2 = j / fft_frames;
        ch[static_cast<size_t>(k1 * n_chan + k2)] = make_float2(static_cast<float>(std::cos(ph)), static_cast<float>(std::sin(ph)));
    }
    if (cudaMalloc(&d->chirp, ch.size() * sizeof(float2)) != cudaSuccess) return bad("cudaMalloc(chirp)");
    if (cudaMemcpy(d->chirp, ch.data(), ch.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return bad("cudaMemcpy(chirp)");
    const std::vector<float2> twf = smem_fft_twiddles(fft_frames), twc = smem_fft_twiddles(n_chan);
    if (cudaMalloc(&d->tw_f, twf.size() * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&d->tw_c, twc.size() * sizeof(float2)) != cudaSuccess)
        return bad("cudaMalloc(twiddles)");
    if (cudaMemcpy(d->tw_f, twf.data(), twf.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d->tw_c, twc.data(), twc.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return bad("cudaMemcpy(twiddles)");
    *out = d;
    return CORR_OK;
}

int corr_dd_push_device(corr_dd_t* d, const float* spec, int64_t n_frames, float* out, int64_t out_cap,
                        int64_t* n_out, void* stream) {
    if (!d) return ddfail(CORR_E_INVAL, "null dedisperser");
    if (n_out) *n_out = 0;
    if (n_frames < 0 || n_frames > d->max_push) return ddfail(CORR_E_INVAL, "n_frames must be in [0, max_push_frames]");
    if (n_frames > 0 && !spec) return ddfail(CORR_E_INVAL, "null spectra");
    if (reinterpret_cast<uintptr_t>(spec) & 15) return ddfail(CORR_E_INVAL, "spec must be 16-byte aligned");
    const int keep = d->F - d->O;
    const int64_t have = d->have + n_frames;
    const int n_blocks = have >= d->F ? static_cast<int>((have - d->F) / keep + 1) : 0;
    const int64_t per_block = static_cast<int64_t>(keep) * d->n_chan / d->avg;
    if (static_cast<int64_t>(n_blocks) * per_block > out_cap || (n_blocks > 0 && !out))
        return ddfail(CORR_E_INVAL, "out_cap is below the outputs this push completes");
    cudaSetDevice(d->dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t fb = static_cast<size_t>(d->n_chan) * sizeof(float4);
    const bool tm = d->timing && n_blocks > 0;
    if (tm) DDCU(cudaEventRecord(d->ev[0], s));
    // append to the ring (two pieces at the wrap)
    int64_t done = 0;
    while (done < n_frames) {
        const int64_t take = std::min(n_frames - done, d->cap - d->wpos);
        DDCU(cudaMemcpyAsync(d->ring + d->wpos * d->n_chan, spec + done * d->n_chan * 4, take * fb,
                             cudaMemcpyDeviceToDevice, s));
        d->wpos = (d->wpos + take) % d->cap;
        done += take;
    }
    if (n_blocks > 0) {
        int64_t start0 = d->wpos - have;        // ring frame of the oldest unconsumed frame
        start0 = ((start0 % d->cap) + d->cap) % d->cap;
        DdBlocks b{d->ring, d->cap, start0, keep, d->work, d->part, keep};
        const int64_t M = static_cast<int64_t>(d->F) * d->n_chan;
        const float inv_half_m = 2.0f / static_cast<float>(M);
        const float scale = static_cast<float>(1.0 / (static_cast<double>(d->n_chan) * static_cast<double>(M)));
        if (tm) DDCU(cudaEventRecord(d->ev[1], s));
        DDCU(launch_ac_any(d->F, false, b, d->n_chan, n_blocks, d->tw_f, scale, s));
        if (tm) DDCU(cudaEventRecord(d->ev[2], s));
        DDCU(launch_b_any(d->n_chan, d->work, d->F, n_blocks, d->chirp, d->tw_c, inv_half_m, s));
        if (tm) DDCU(cudaEventRecord(d->ev[3], s));
        DDCU(launch_ac_any(d->F, true, b, d->n_chan, n_blocks, d->tw_f, scale, s));
        if (tm) DDCU(cudaEventRecord(d->ev[4], s));
        const int G = col_g(d->F);
        if (d->avg < d->n_chan) {
            const int64_t threads = static_cast<int64_t>(n_blocks) * (d->n_chan / d->avg) * keep;
            dd_pass_d_in_frame<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(d->part, n_blocks, keep,
                                                                                           d->n_chan, G, d->avg, out);
        } else {
            dd_pass_d_frames<<<dim3((keep + 31) / 32, n_blocks), 256, 0, s>>>(d->part, keep, d->n_chan, G, d->avg, out);
        }
        DDCU(cudaGetLastError());
        if (tm) {   // timing mode waits for the push and adds up its stages
            DDCU(cudaEventRecord(d->ev[5], s));
            DDCU(cudaEventSynchronize(d->ev[5]));
            for (int q = 0; q < 5; ++q) {
                float ms = 0.0f;
                DDCU(cudaEventElapsedTime(&ms, d->ev[q], d->ev[q + 1]));
                d->stage_ms[q] += ms;
            }
            d->timed += 1;
        }
    }
    d->have = have - static_cast<int64_t>(n_blocks) * keep;
    if (n_out) *n_out = static_cast<int64_t>(n_blocks) * per_block;
    return CORR_OK;
}

int corr_dd_set_timing(corr_dd_t* d, int on) {
    if (!d) return ddfail(CORR_E_INVAL, "null dedisperser");
    cudaSetDevice(d->dev);
    for (cudaEvent_t& e : d->ev)
        if (!e) DDCU(cudaEventCreate(&e));
    d->timing = on != 0;
    std::memset(d->stage_ms, 0, sizeof d->stage_ms);
    d->timed = 0;
    return CORR_OK;
}

int corr_dd_stage_times(corr_dd_t* d, float* ms5, int* n_timed) {
    if (!d || !ms5) return ddfail(CORR_E_INVAL, "null argument");
    for (int q = 0; q < 5; ++q) ms5[q] = static_cast<float>(d->stage_ms[q]);
    if (n_timed) *n_timed = d->timed;
    return CORR_OK;
}

int corr_dd_reset(corr_dd_t* d) {
    if (!d) return ddfail(CORR_E_INVAL, "null dedisperser");
    d->have = 0;
    d->wpos = 0;
    return CORR_OK;
}

int corr_dd_destroy(corr_dd_t* d) {
    if (!d) return CORR_OK;
    cudaSetDevice(d->dev);
    cudaDeviceSynchronize();
    dd_free(d);
    return CORR_OK;
}

}  // extern "C"
