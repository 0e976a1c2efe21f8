// fft_smem.cuh -- building blocks of the shared-memory FFTs (F-engine, coherent dedispersion):
// padded indexing, constant twiddles, in-register radix-R DFTs, group barriers, and a generic
// Stockham FFT of L points by L/16 threads with a hook on its output.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace gbx {

// one pad element per 16: every Stockham exchange of 8-byte points is free of bank conflicts
__host__ __device__ constexpr int pad16(int i) { return i + (i >> 4); }

// Packed FP32x2 arithmetic (sm_100 family): both components of a complex sum or difference in
// one instruction, each rounded exactly as the scalar operation (a - b as fma(b, -1, a)).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// cos(2 pi m / 32), m = 0..16
__device__ __forceinline__ constexpr float c32(int m) {
    return m == 0 ? 1.0f : m == 1 ? 0.98078528040323044913f : m == 2 ? 0.92387953251128675613f
         : m == 3 ? 0.83146961230254523708f : m == 4 ? 0.70710678118654752440f
         : m == 5 ? 0.55557023301960222474f : m == 6 ? 0.38268343236508977173f
         : m == 7 ? 0.19509032201612826785f : m == 8 ? 0.0f : -c32(16 - m);
}

// o * exp(-2 pi i K / R) (R <= 32) with the trivial cases spelled out
template <int R, int K>
__device__ __forceinline__ float2 twiddle_const(float2 o) {
    static_assert(R <= 32 && K < R / 2, "constant twiddles of radix <= 32");
    constexpr int m = K * (32 / R);              // position on the 32-point circle, 0..15
    if constexpr (m == 0) {
        return o;
    } else if constexpr (m == 8) {               // -i
        return make_float2(o.y, -o.x);
    } else if constexpr (m == 4) {               // (1 - i) / sqrt2
        constexpr float h = 0.70710678118654752f;
        return make_float2(h * (o.x + o.y), h * (o.y - o.x));
    } else if constexpr (m == 12) {              // (-1 - i) / sqrt2
        constexpr float h = 0.70710678118654752f;
        return make_float2(h * (o.y - o.x), -h * (o.x + o.y));
    } else {
        constexpr float c = c32(m);
        constexpr float s = (m <= 8) ? c32(8 - m) : c32(m - 8);  // sin(2 pi m / 32), m = 1..15
        // w = c - i s
        return make_float2(c * o.x + s * o.y, c * o.y - s * o.x);
    }
}

// In-register forward DFT of R points, natural order in and out: radix-2 decimation in time,
// written stage by stage (inputs in bit-reversed order, then log2 R stages of R/2 butterflies),
// so that every stage offers R/2 independent butterflies to the instruction scheduler.  Stage H
// joins the H-point DFTs of the even- and odd-indexed points into 2H-point ones:
// out[j] = E[j] + W_2H^j O[j], out[j + H] = E[j] - W_2H^j O[j].
template <int R>
struct Dft {
    static constexpr int brev(int i) {
        int r = 0;
        for (int b = 1; b < R; b <<= 1) {
            r = (r << 1) | (i & 1);
            i >>= 1;
        }
        return r;
    }
    template <int S>
    __device__ __forceinline__ static void run(float2* v) {
        // v[0], v[S], v[2S], ... hold the R inputs; transform in place
        float2 u[R];
#pragma unroll
        for (int i = 0; i < R; ++i) u[i] = v[S * brev(i)];
        stage<1>(u);
#pragma unroll
        for (int k = 0; k < R; ++k) v[S * k] = u[k];
    }
    template <int H>
    __device__ __forceinline__ static void stage(float2* u) {
        if constexpr (H < R) {
            bfly<H, 0>(u);
            stage<2 * H>(u);
        }
    }
    template <int H, int J>
    __device__ __forceinline__ static void bfly(float2* u) {
        if constexpr (J < H) {
#pragma unroll
            for (int blk = 0; blk < R; blk += 2 * H) {
                const float2 e = u[blk + J];
                const float2 t = twiddle_const<2 * H, J>(u[blk + J + H]);
                u[blk + J] = padd(e, t);
                u[blk + J + H] = psub(e, t);
            }
            bfly<H, J + 1>(u);
        }
    }
};

// barrier among the T threads of one FFT group (group g); a warp when T <= 32
template <int T>
__device__ __forceinline__ void group_sync(int g) {
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(T) : "memory");
    }
}

// ---- generic FFT of L = 2^n points (64 <= L <= 4096) in padded shared memory ----------------
// Stockham passes of radix 16, R2 and R3 (16 points per thread in registers, shared memory
// between passes); natural order in and out.  Pass p of radix R over span Ns reads
// X[b + r L/R], multiplies by W_{Ns R}^{(b mod Ns) r}, takes the R-point DFT and writes
// X[(b / Ns) Ns R + b mod Ns + r Ns].  Twiddles: table tw = [R2][16] (pass 2) then [R3][16 R2]
// (pass 3), from smem_fft_twiddles().
template <int L>
struct SmemFft {
    static constexpr int T = L / 16;                          // threads per FFT
    static constexpr int R2 = (L / 16 >= 16) ? 16 : L / 16;
    static constexpr int R3 = L / (16 * R2);
    static constexpr int PAD = L + L / 16;                    // padded length (float2)
    static_assert(L >= 64 && L <= 4096 && (L & (L - 1)) == 0, "64 <= L <= 4096, a power of two");
};

template <int L, int R, int Ns>
__device__ __forceinline__ void gfft_load(const float2* __restrict__ buf, const float2* __restrict__ tw, int t,
                                          float2 (&v)[16]) {
    constexpr int T = L / 16, NB = L / R, PER = 16 / R;
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int b = t + m * T;
#pragma unroll
        for (int r = 0; r < R; ++r) v[m * R + r] = buf[pad16(b + r * NB)];
        if constexpr (Ns > 1) {
            const int j = b % Ns;
#pragma unroll
            for (int r = 1; r < R; ++r) v[m * R + r] = cmul(__ldg(tw + r * Ns + j), v[m * R + r]);
        }
        Dft<R>::template run<1>(v + m * R);
    }
}

template <int L, int R, int Ns, typename Post>
__device__ __forceinline__ void gfft_store(float2* __restrict__ buf, int t, const float2 (&v)[16], Post&& post) {
    constexpr int T = L / 16, PER = 16 / R;
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int b = t + m * T;
        const int base = (b / Ns) * Ns * R + (b % Ns);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + r * Ns)] = post(base + r * Ns, v[m * R + r]);
    }
}

// Forward FFT in place of buf[pad16(0 .. L-1)] by threads t = 0 .. T-1 of group g; every output
// X[i] is stored as post(i, X[i]).  Ends with the group synchronised.
template <int L, typename Post>
__device__ __forceinline__ void smem_fft(float2* buf, const float2* __restrict__ tw, int t, int g, Post&& post) {
    using P = SmemFft<L>;
    constexpr int T = P::T, R2 = P::R2, R3 = P::R3;
    auto keep = [](int, float2 x) { return x; };
    float2 v[16];
    gfft_load<L, 16, 1>(buf, tw, t, v);
    group_sync<T>(g);
    gfft_store<L, 16, 1>(buf, t, v, keep);
    group_sync<T>(g);
    gfft_load<L, R2, 16>(buf, tw, t, v);
    group_sync<T>(g);
    if constexpr (R3 == 1) {
        gfft_store<L, R2, 16>(buf, t, v, post);
    } else {
        gfft_store<L, R2, 16>(buf, t, v, keep);
        group_sync<T>(g);
        gfft_load<L, R3, 16 * R2>(buf, tw + 16 * R2, t, v);
        group_sync<T>(g);
        gfft_store<L, R3, 16 * R2>(buf, t, v, post);
    }
    group_sync<T>(g);
}

// the twiddle table of smem_fft<L>, from FP64 and rounded once
std::vector<float2> smem_fft_twiddles(int L);

}  // namespace gbx
