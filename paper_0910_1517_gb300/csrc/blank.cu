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
// (a second read of the block, from L1), which the F-engine reads instead of the raw rows.
// (Fusing the replacement into the F-engine's sample conversion was measured first: +1.75 ms
// on the GMRT-scale F-engine against +0.3 ms for this separate pass.)
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
    // pass 1: histogram of x (16-byte loads: rows and blocks start on 16-byte boundaries)
    const int n16 = len / 16;
    int* h = hw[warp];
    for (int q = threadIdx.x; q < n16; q += kBlankThreads) {
        const int4 w = __ldg(reinterpret_cast<const int4*>(row) + q);
        const uint32_t u[4] = {static_cast<uint32_t>(w.x), static_cast<uint32_t>(w.y), static_cast<uint32_t>(w.z),
                               static_cast<uint32_t>(w.w)};
#pragma unroll
        for (int e = 0; e < 16; ++e)
            atomicAdd(&h[static_cast<int>(static_cast<int8_t>((u[e >> 2] >> (8 * (e & 3))) & 0xff)) + 128], 1);
    }
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
    // pass 3: the blanked block
    const int T2 = t2_s;
    const float sg = sig_s;
    const float* g = noise + static_cast<int64_t>(i) * (noise_mask + 1);
    int8_t* out = y + static_cast<int64_t>(i) * ldy + p0;
    auto fix = [&](int v, int64_t pos) {
        if (abs(2 * v - med2) <= T2) return v;
        const float r = rintf(__fmul_rn(sg, __ldg(g + (pos & noise_mask))));
        return static_cast<int>(fminf(127.0f, fmaxf(-127.0f, r)));
    };
    for (int q = threadIdx.x; q < n16; q += kBlankThreads) {
        const int4 w = __ldg(reinterpret_cast<const int4*>(row) + q);
        uint32_t u[4] = {static_cast<uint32_t>(w.x), static_cast<uint32_t>(w.y), static_cast<uint32_t>(w.z),
                         static_cast<uint32_t>(w.w)};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int v = static_cast<int>(static_cast<int8_t>((u[e >> 2] >> (8 * (e & 3))) & 0xff));
            const int nv = fix(v, p0 + 16 * q + e);
            if (nv != v)
                u[e >> 2] = (u[e >> 2] & ~(0xffu << (8 * (e & 3)))) |
                            ((static_cast<uint32_t>(nv) & 0xffu) << (8 * (e & 3)));
        }
        reinterpret_cast<int4*>(out)[q] = make_int4(static_cast<int>(u[0]), static_cast<int>(u[1]),
                                                    static_cast<int>(u[2]), static_cast<int>(u[3]));
    }
    for (int q = 16 * n16 + threadIdx.x; q < len; q += kBlankThreads)
        out[q] = static_cast<int8_t>(fix(row[q], p0 + q));
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
