// blank.cu -- statistics of the time-domain voltage blanker (Sec. 5, Eq. 3-4) on sm_103a.
//
// For every (input, block) of raw int8 samples: the median, the MAD (median of |x - med|)
// and the flag threshold of Eq. 4, |x - med| > M MAD / 0.6745.  int8 data make both medians
// exact: a 256-bin histogram of x gives the two middle values (their sum is 2 med), a 511-bin
// histogram of d2 = |2x - 2med| gives the two middle deviations (their sum is 4 MAD), and the
// threshold becomes the integer T2 = floor(2 M MAD / 0.6745) (computed in FP64), so that a
// sample is replaced iff d2 > T2 -- the same decision as the FP64 comparison.  The F-engine
// applies the replacement while it converts the samples (fengine.cu).
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

constexpr int kBlankThreads = 256;

// the rank-th smallest (0-based) of the values counted in hist[0..nb), by a block-wide scan:
// thread j sums bins [j * per, (j + 1) * per)
template <int NB>
__device__ int hist_select(const int* hist, int rank, int* scan) {
    constexpr int per = (NB + kBlankThreads - 1) / kBlankThreads;
    const int j = threadIdx.x;
    int local = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int b = j * per + q;
        if (b < NB) local += hist[b];
    }
    scan[j] = local;
    __syncthreads();
    // inclusive scan over the 256 partial sums (Hillis-Steele, in place, two buffers)
    for (int off = 1; off < kBlankThreads; off <<= 1) {
        const int v = (j >= off) ? scan[j - off] : 0;
        __syncthreads();
        scan[j] += v;
        __syncthreads();
    }
    const int before = j ? scan[j - 1] : 0;
    __shared__ int found;
    if (j == 0) found = -1;
    __syncthreads();
    if (rank >= before && rank < scan[j]) {
        int c = before;
        for (int q = 0; q < per; ++q) {
            const int b = j * per + q;
            if (b >= NB) break;
            c += hist[b];
            if (rank < c) {
                found = b;
                break;
            }
        }
    }
    __syncthreads();
    const int r = found;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBlankThreads) blank_stats_kernel(const int8_t* __restrict__ x, int64_t ld,
                                                                     int64_t n, int block, double M,
                                                                     int32_t* __restrict__ stats) {
    __shared__ int hx[256];
    __shared__ int hd[512];
    __shared__ int scan[kBlankThreads];
    const int i = blockIdx.y;
    const int64_t b = blockIdx.x, p0 = b * block;
    const int len = static_cast<int>(p0 + block <= n ? block : n - p0);
    const int8_t* row = x + static_cast<int64_t>(i) * ld + p0;
    for (int q = threadIdx.x; q < 512; q += kBlankThreads) {
        hd[q] = 0;
        if (q < 256) hx[q] = 0;
    }
    __syncthreads();
    // pass 1: histogram of x (16-byte loads: rows and blocks start on 16-byte boundaries)
    const int n16 = len / 16;
    for (int q = threadIdx.x; q < n16; q += kBlankThreads) {
        const int4 w = reinterpret_cast<const int4*>(row)[q];
        const uint32_t u[4] = {static_cast<uint32_t>(w.x), static_cast<uint32_t>(w.y), static_cast<uint32_t>(w.z),
                               static_cast<uint32_t>(w.w)};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int v = static_cast<int>(static_cast<int8_t>((u[e >> 2] >> (8 * (e & 3))) & 0xff));
            atomicAdd(&hx[v + 128], 1);
        }
    }
    for (int q = 16 * n16 + threadIdx.x; q < len; q += kBlankThreads) atomicAdd(&hx[row[q] + 128], 1);
    __syncthreads();
    const int lo = (len - 1) / 2, hi = len / 2;       // the two middle ranks (equal for odd len)
    const int med2 = hist_select<256>(hx, lo, scan) + hist_select<256>(hx, hi, scan) - 256;
    // pass 2: histogram of d2 = |2 x - 2 med| in [0, 510]
    for (int v = threadIdx.x; v < 256; v += kBlankThreads) {
        const int c = hx[v];
        if (c) atomicAdd(&hd[abs(2 * (v - 128) - med2)], c);
    }
    __syncthreads();
    const int mad4 = hist_select<512>(hd, lo, scan) + hist_select<512>(hd, hi, scan);
    if (threadIdx.x == 0) {
        const double mad = mad4 / 4.0;
        double t2 = floor(2.0 * (M * mad / 0.6745));
        if (t2 > 1024.0) t2 = 1024.0;
        const int T2 = static_cast<int>(t2);
        int count = 0;
        for (int d = T2 + 1; d < 511; ++d) count += (d >= 0) ? hd[d] : 0;
        int32_t* st = stats + 4 * (static_cast<int64_t>(i) * gridDim.x + b);
        st[0] = med2;
        st[1] = mad4;
        st[2] = T2;
        st[3] = count;
    }
}

}  // namespace

cudaError_t launch_blank_stats(const int8_t* x, int64_t ld, int n_in, int64_t n, int block, double M,
                               int32_t* stats, cudaStream_t s) {
    if (n < 1 || block < 16 || (block & 15)) return cudaErrorInvalidValue;
    const int64_t nb = (n + block - 1) / block;
    if (nb > 2147483647LL || n_in > 65535) return cudaErrorInvalidValue;
    blank_stats_kernel<<<dim3(static_cast<unsigned>(nb), n_in), kBlankThreads, 0, s>>>(x, ld, n, block, M, stats);
    return cudaGetLastError();
}

}  // namespace gbx
