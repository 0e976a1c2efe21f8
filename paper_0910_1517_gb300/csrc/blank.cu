// blank.cu -- statistics of the time-domain voltage blanker (Sec. 5, Eq. 3-4) on sm_103a.
//
// For every (input, block) of raw int8 samples: the median, the MAD (median of |x - med|)
// and the flag threshold of Eq. 4, |x - med| > M MAD / 0.6745.  int8 data make both medians
// exact: a 256-bin histogram of x gives the two middle values (their sum is 2 med), a 511-bin
// histogram of d2 = |2x - 2med| gives the two middle deviations (their sum is 4 MAD), and the
// threshold becomes the integer T2 = floor(2 M MAD / 0.6745) (computed in FP64), so that a
// sample is replaced iff d2 > T2 -- the same decision as the FP64 comparison -- by
// rint(sigma g) clamped to +-127, sigma = MAD / 0.6745 rounded to FP32 and g the input's
// table noise at the sample's position.  The same CTA then writes the block's blanked samples
// (testing four samples at a time against integer bounds), which the F-engine reads instead of
// the raw rows.  (Fusing the replacement into the F-engine's sample conversion was measured
// first: +1.75 ms on the GMRT-scale F-engine, more than this separate pass.)
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

constexpr int kBlankThreads = 256;
constexpr int kBlankWarps = kBlankThreads / 32;

// Called by one whole warp: the rank-th smallest (0-based) of the values counted in hist[0..NB).
// Each lane sums NB/32 consecutive bins, a shuffle scan finds the lane holding the rank, and
// that lane walks its bins.
template <int NB>
__device__ __forceinline__ int warp_select(const int* hist, int rank, int lane) {
    constexpr int per = NB / 32;
    int local = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) local += hist[lane * per + q];
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const int before = incl - local;
    const unsigned hit = __ballot_sync(0xffffffffu, rank >= before && rank < incl);
    const int src = __ffs(hit) - 1;
    int bin = 0;
    if (lane == src) {
        int c = before;
        for (int q = 0; q < per; ++q) {
            c += hist[lane * per + q];
            if (rank < c) {
                bin = lane * per + q;
                break;
            }
        }
    }
    return __shfl_sync(0xffffffffu, bin, src);
}

// int4 pieces of the block a thread keeps in registers between the histogram and the copy;
// the copy reads the others again (from L1 / L2).  One: at 48 registers (four pieces) the SM
// holds 5 CTAs instead of 8, and the GMRT-scale pass ran 10 % slower.
constexpr int kBlankCache = 1;

__global__ void __launch_bounds__(kBlankThreads) blank_kernel(const int8_t* __restrict__ x, int64_t ld, int64_t n,
                                                               int block, double M, const float* __restrict__ noise,
                                                               int noise_mask, int32_t* __restrict__ stats,
                                                               int8_t* __restrict__ y, int64_t ldy) {
    __shared__ int hw[kBlankWarps][256];   // per-warp histograms of x + 128
    __shared__ int hd[512];                // histogram of d2 = |2x - 2med|
    __shared__ int med2_s, t2_s;
    __shared__ float sig_s;
    const int i = blockIdx.y, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t b = blockIdx.x, p0 = b * block;
    const int len = static_cast<int>(p0 + block <= n ? block : n - p0);
    const int8_t* row = x + static_cast<int64_t>(i) * ld + p0;
    for (int q = threadIdx.x; q < kBlankWarps * 256; q += kBlankThreads) (&hw[0][0])[q] = 0;
    for (int q = threadIdx.x; q < 512; q += kBlankThreads) hd[q] = 0;
    __syncthreads();
    // pass 1: histogram of x (16-byte loads: rows and blocks start on 16-byte boundaries).  The
    // first kBlankCache pieces of each thread are loaded together and kept for pass 3; a byte
    // b of w ^ 0x80808080 is x + 128.
    const int n16 = len / 16;
    int* h = hw[warp];
    auto count = [&](const int4& w) {
        const uint32_t u[4] = {static_cast<uint32_t>(w.x) ^ 0x80808080u, static_cast<uint32_t>(w.y) ^ 0x80808080u,
                               static_cast<uint32_t>(w.z) ^ 0x80808080u, static_cast<uint32_t>(w.w) ^ 0x80808080u};
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(&h[(u[e >> 2] >> (8 * (e & 3))) & 0xff], 1);
    };
    int4 keep[kBlankCache];
#pragma unroll
    for (int k = 0; k < kBlankCache; ++k) {
        const int q = threadIdx.x + k * kBlankThreads;
        keep[k] = q < n16 ? __ldg(reinterpret_cast<const int4*>(row) + q) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < kBlankCache; ++k)
        if (threadIdx.x + k * kBlankThreads < n16) count(keep[k]);
    for (int q = threadIdx.x + kBlankCache * kBlankThreads; q < n16; q += kBlankThreads)
        count(__ldg(reinterpret_cast<const int4*>(row) + q));
    for (int q = 16 * n16 + threadIdx.x; q < len; q += kBlankThreads) atomicAdd(&h[row[q] + 128], 1);
    __syncthreads();
    {   // merge the warp histograms into hw[0]
        int c = 0;
#pragma unroll
        for (int w = 0; w < kBlankWarps; ++w) c += hw[w][threadIdx.x];
        __syncthreads();
        hw[0][threadIdx.x] = c;
    }
    __syncthreads();
    const int lo = (len - 1) / 2, hi = len / 2;       // the two middle ranks (equal for odd len)
    if (warp == 0) {
        const int m2 = warp_select<256>(hw[0], lo, lane) + warp_select<256>(hw[0], hi, lane) - 256;
        if (lane == 0) med2_s = m2;
    }
    __syncthreads();
    const int med2 = med2_s;
    {   // pass 2: d2 histogram straight from the value histogram
        const int c = hw[0][threadIdx.x];
        if (c) atomicAdd(&hd[abs(2 * (static_cast<int>(threadIdx.x) - 128) - med2)], c);
    }
    __syncthreads();
    if (warp == 0) {
        const int mad4 = warp_select<512>(hd, lo, lane) + warp_select<512>(hd, hi, lane);
        const double mad = mad4 / 4.0;
        double t2 = floor(2.0 * (M * mad / 0.6745));
        if (t2 > 1024.0) t2 = 1024.0;
        const int T2 = static_cast<int>(t2);
        int count = 0;
        for (int d = lane; d < 511; d += 32) count += d > T2 ? hd[d] : 0;
#pragma unroll
        for (int off = 16; off; off >>= 1) count += __shfl_xor_sync(0xffffffffu, count, off);
        if (lane == 0) {
            const int64_t q = static_cast<int64_t>(i) * gridDim.x + b;
            int32_t* st = stats + 4 * q;
            st[0] = med2;
            st[1] = mad4;
            st[2] = T2;
            st[3] = count;
            t2_s = T2;
            sig_s = static_cast<float>(mad / 0.6745);
        }
    }
    __syncthreads();
    // pass 3: the blanked block.  |2x - med2| > T2 holds exactly for x > hi_x or x < lo_x,
    // hi_x = floor((med2 + T2) / 2), lo_x = ceil((med2 - T2) / 2) (integer x); clamped to the
    // int8 range they compare four samples at a time, and only a word holding a flagged sample
    // takes the per-byte replacement.
    const int T2 = t2_s;
    const float sg = sig_s;
    const int hi_x = min(127, (med2 + T2) >> 1), lo_x = max(-128, (med2 - T2 + 1) >> 1);
    const uint32_t hi4 = static_cast<uint32_t>(hi_x & 0xff) * 0x01010101u;
    const uint32_t lo4 = static_cast<uint32_t>(lo_x & 0xff) * 0x01010101u;
    const float* g = noise + static_cast<int64_t>(i) * (noise_mask + 1);
    int8_t* out = y + static_cast<int64_t>(i) * ldy + p0;
    auto repl = [&](int64_t pos) {
        const float r = rintf(__fmul_rn(sg, __ldg(g + (pos & noise_mask))));
        return static_cast<int>(fminf(127.0f, fmaxf(-127.0f, r)));
    };
    auto fix_word = [&](uint32_t w, int64_t pos) {   // 4 samples starting at block position pos
        const uint32_t flag = __vcmpgts4(w, hi4) | __vcmplts4(w, lo4);
        if (flag == 0u) return w;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((flag >> (8 * e)) & 0xffu)
                w = (w & ~(0xffu << (8 * e))) | ((static_cast<uint32_t>(repl(pos + e)) & 0xffu) << (8 * e));
        return w;
    };
    auto fix = [&](const int4& v, int q) {
        const int64_t pos = p0 + 16 * static_cast<int64_t>(q);
        reinterpret_cast<int4*>(out)[q] = make_int4(static_cast<int>(fix_word(static_cast<uint32_t>(v.x), pos)),
                                                    static_cast<int>(fix_word(static_cast<uint32_t>(v.y), pos + 4)),
                                                    static_cast<int>(fix_word(static_cast<uint32_t>(v.z), pos + 8)),
                                                    static_cast<int>(fix_word(static_cast<uint32_t>(v.w), pos + 12)));
    };
#pragma unroll
    for (int k = 0; k < kBlankCache; ++k) {
        const int q = threadIdx.x + k * kBlankThreads;
        if (q < n16) fix(keep[k], q);
    }
    for (int q = threadIdx.x + kBlankCache * kBlankThreads; q < n16; q += kBlankThreads)
        fix(__ldg(reinterpret_cast<const int4*>(row) + q), q);
    for (int q = 16 * n16 + threadIdx.x; q < len; q += kBlankThreads) {
        const int v = row[q];
        out[q] = static_cast<int8_t>(v > hi_x || v < lo_x ? repl(p0 + q) : v);
    }
}

}  // namespace

cudaError_t launch_blank(const int8_t* x, int64_t ld, int n_in, int64_t n, int block, double M,
                         const float* noise, int noise_mask, int32_t* stats, int8_t* y, int64_t ldy,
                         cudaStream_t s) {
    if (n < 1 || block < 16 || (block & 15) || (ld & 15) || (ldy & 15)) return cudaErrorInvalidValue;
    const int64_t nb = (n + block - 1) / block;
    if (nb > 2147483647LL || n_in > 65535) return cudaErrorInvalidValue;
    blank_kernel<<<dim3(static_cast<unsigned>(nb), n_in), kBlankThreads, 0, s>>>(x, ld, n, block, M, noise,
                                                                                   noise_mask, stats, y, ldy);
    return cudaGetLastError();
}

}  // namespace gbx
