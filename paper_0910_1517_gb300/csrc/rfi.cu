// rfi.cu -- RFI-flagging stage for sm_103a: per-patch median / MAD statistics and
// flags (Sec. 5, Eq. 3-4), and a small convolutional flagger trained and run by
// hand-written kernels (direct 3x3 convolutions over 16x16 output tiles, FP16
// weights and activations, FP32 accumulation, FP32 gradients, Adam on FP32
// master weights).  Every network kernel is templated on the type TA its weights
// and activations are kept in: __half for the flagger, float for the FP32 build
// (rfi_create_fp32) that checks the kernels' arithmetic against the FP64 oracle.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/corr.h"
#include "../../include/rfi.h"
#include "common.cuh"

namespace gbx {
void set_last_error(const char* msg);
}

namespace {

__device__ __forceinline__ float ldf(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ void stf(__half* p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }

constexpr int PH = 64, PW = 64, PHW = PH * PW;   // patch: 64 dumps x 64 channels
constexpr int T = 16, TH = T + 2;                 // output tile and tile with halo
constexpr int kTiles = (PH / T) * (PW / T);       // 16 tiles per patch
constexpr int NPAR = 9441;
constexpr int OW1 = 0, OB1 = 144, OW2 = 160, OB2 = 4768, OW3 = 4800, OB3 = 9408, OW4 = 9424, OB4 = 9440;

// ---------------------------------------------------------------- convolution
// One CTA computes a 16x16 output tile of one patch for all CO output channels.
// MODE 0 (forward):       out[o] = relu(b[o] + sum_c sum_tap w[c][tap][o] in[c][pixel + tap])   (fp16 -> fp16)
// MODE 1 (backward data): the same correlation without bias / ReLU on dZ = dA * (act > 0)        (fp32 -> fp32)
// w is laid out [CI][9][CO] so that one (c, tap) reads CO consecutive weights (a broadcast).
// TIN: type of the forward input (the FP16 patches for layer 1, TA after it); TA: weights and activations.
template <int CI, int CO, int MODE, typename TIN, typename TA>
__global__ void __launch_bounds__(256) conv3x3_kernel(const void* __restrict__ in, const TA* __restrict__ act,
                                                      const TA* __restrict__ w, const TA* __restrict__ bias,
                                                      void* __restrict__ out) {
    extern __shared__ __align__(16) float sm[];
    float* wsm = sm;                                   // CI * 9 * CO
    float* tile = sm + CI * 9 * CO;                    // CI * TH * TH
    const int b = blockIdx.x / kTiles, tl = blockIdx.x % kTiles;
    const int ty0 = (tl / (PW / T)) * T, tx0 = (tl % (PW / T)) * T;
    const int tid = threadIdx.x, py = tid / T, px = tid % T;
    for (int q = tid; q < CI * 9 * CO; q += 256) wsm[q] = ldf(w + q);
    for (int q = tid; q < CI * TH * TH; q += 256) {
        const int c = q / (TH * TH), r = q % (TH * TH), yy = r / TH, xx = r % TH;
        const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
        float v = 0.0f;
        if (gy >= 0 && gy < PH && gx >= 0 && gx < PW) {
            const size_t gi = (static_cast<size_t>(b) * CI + c) * PHW + gy * PW + gx;
            if constexpr (MODE == 0) {
                v = ldf(static_cast<const TIN*>(in) + gi);
            } else {
                v = static_cast<const float*>(in)[gi];
                if (!(ldf(act + gi) > 0.0f)) v = 0.0f;             // ReLU gradient
            }
        }
        tile[q] = v;
    }
    __syncthreads();
    float acc[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o] = (MODE == 0) ? ldf(bias + o) : 0.0f;
    for (int c = 0; c < CI; ++c) {
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const float x = tile[(c * TH + py + tap / 3) * TH + px + tap % 3];
            const float4* w4 = reinterpret_cast<const float4*>(wsm + (c * 9 + tap) * CO);
#pragma unroll
            for (int o4 = 0; o4 < CO / 4; ++o4) {
                const float4 ww = w4[o4];
                acc[4 * o4] = fmaf(ww.x, x, acc[4 * o4]);
                acc[4 * o4 + 1] = fmaf(ww.y, x, acc[4 * o4 + 1]);
                acc[4 * o4 + 2] = fmaf(ww.z, x, acc[4 * o4 + 2]);
                acc[4 * o4 + 3] = fmaf(ww.w, x, acc[4 * o4 + 3]);
            }
        }
    }
    const size_t base = static_cast<size_t>(b) * CO * PHW + (ty0 + py) * PW + tx0 + px;
#pragma unroll
    for (int o = 0; o < CO; ++o) {
        if constexpr (MODE == 0)
            stf(static_cast<TA*>(out) + base + static_cast<size_t>(o) * PHW, fmaxf(acc[o], 0.0f));
        else
            static_cast<float*>(out)[base + static_cast<size_t>(o) * PHW] = acc[o];
    }
}

template <int CI, int CO>
size_t conv_smem() {
    return sizeof(float) * (CI * 9 * CO + CI * TH * TH);
}

// ------------------------------------------------------------- weight gradient
// dW[o][c][tap] += sum_pixels dZ[o][p] A[c][p + tap],  db[o] += sum_pixels dZ[o][p],
// dZ = dA * (act > 0).  A CTA loops over tiles; each thread owns one input channel c,
// NO output channels and a pixel subset, and adds its partial sums atomically at the end.
template <int CI, int CO, typename TIN, typename TA>
__global__ void __launch_bounds__(256) wgrad_kernel(const TIN* __restrict__ A, const float* __restrict__ dA,
                                                    const TA* __restrict__ act, float* __restrict__ dW,
                                                    float* __restrict__ db, int n_tiles) {
    constexpr int PAIRS = CI * CO;
    constexpr int G = PAIRS >= 256 ? 1 : 256 / PAIRS;          // pixel groups
    constexpr int NO = PAIRS >= 256 ? PAIRS / 256 : 1;          // output channels per thread
    constexpr int OSTRIDE = PAIRS >= 256 ? 256 / CI : 1;
    static_assert(PAIRS % 256 == 0 || 256 % PAIRS == 0, "pair split");
    extern __shared__ __align__(16) float sm[];
    float* at = sm;                         // CI * TH * TH
    float* dz = sm + CI * TH * TH;          // CO * T * T
    const int tid = threadIdx.x;
    int c, o0, g;
    if constexpr (PAIRS >= 256) {
        c = tid % CI;
        o0 = tid / CI;
        g = 0;
    } else {
        const int pr = tid % PAIRS;
        c = pr % CI;
        o0 = pr / CI;
        g = tid / PAIRS;
    }
    float acc[NO][9], accb[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) {
        accb[j] = 0.0f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) acc[j][tap] = 0.0f;
    }
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int b = tile / kTiles, tl = tile % kTiles;
        const int ty0 = (tl / (PW / T)) * T, tx0 = (tl % (PW / T)) * T;
        __syncthreads();   // previous tile's readers are done
        for (int q = tid; q < CI * TH * TH; q += 256) {
            const int cc = q / (TH * TH), r = q % (TH * TH), yy = r / TH, xx = r % TH;
            const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
            float v = 0.0f;
            if (gy >= 0 && gy < PH && gx >= 0 && gx < PW)
                v = ldf(A + (static_cast<size_t>(b) * CI + cc) * PHW + gy * PW + gx);
            at[q] = v;
        }
        for (int q = tid; q < CO * T * T; q += 256) {
            const int oo = q / (T * T), r = q % (T * T);
            const size_t gi = (static_cast<size_t>(b) * CO + oo) * PHW + (ty0 + r / T) * PW + tx0 + r % T;
            dz[q] = ldf(act + gi) > 0.0f ? dA[gi] : 0.0f;
        }
        __syncthreads();
        for (int p = g; p < T * T; p += G) {
            const int y = p / T, x = p % T;
            float a9[9];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) a9[tap] = at[(c * TH + y + tap / 3) * TH + x + tap % 3];
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const float z = dz[(o0 + j * OSTRIDE) * T * T + p];
                accb[j] += z;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) acc[j][tap] = fmaf(z, a9[tap], acc[j][tap]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NO; ++j) {
        const int o = o0 + j * OSTRIDE;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) atomicAdd(&dW[(o * CI + c) * 9 + tap], acc[j][tap]);
        if (c == 0) atomicAdd(&db[o], accb[j]);
    }
}

template <int CI, int CO>
size_t wgrad_smem() {
    return sizeof(float) * (CI * TH * TH + CO * T * T);
}

// ------------------------------------------------------------------- head
// logit = b4 + sum_c W4[c] A3[c][p].  Training: loss += BCE, dlogit = (sigmoid - m) / N,
// dA3[c][p] = W4[c] dlogit, dW4[c] += dlogit A3[c][p], db4 += dlogit.  Inference: prob.
template <typename TA>
__global__ void __launch_bounds__(256) head_kernel(const TA* __restrict__ A3, const uint8_t* __restrict__ mask,
                                                   const TA* __restrict__ pf16, int B, float inv_n,
                                                   float* __restrict__ dA3, float* __restrict__ grad,
                                                   float* __restrict__ loss, float* __restrict__ prob) {
    __shared__ float red[8][18];
    const int64_t q = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x;   // pixel over the batch
    float part[18];
#pragma unroll
    for (int j = 0; j < 18; ++j) part[j] = 0.0f;
    if (q < static_cast<int64_t>(B) * PHW) {
        const int64_t b = q / PHW, p = q % PHW;
        float a[16];
        float s = ldf(pf16 + OB4);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            a[c] = ldf(A3 + (b * 16 + c) * PHW + p);
            s = fmaf(ldf(pf16 + OW4 + c), a[c], s);
        }
        const float pr = 1.0f / (1.0f + expf(-s));
        if (prob) prob[q] = pr;
        if (mask) {
            const float m = mask[q] ? 1.0f : 0.0f;
            part[17] = fmaxf(s, 0.0f) - s * m + log1pf(expf(-fabsf(s)));
            const float ds = (pr - m) * inv_n;
            part[16] = ds;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                part[c] = ds * a[c];
                dA3[(b * 16 + c) * PHW + p] = ds * ldf(pf16 + OW4 + c);
            }
        }
    }
    if (!mask) return;
    // warp then block reduction of the 16 + 1 head gradients and the loss
#pragma unroll
    for (int j = 0; j < 18; ++j)
        for (int off = 16; off > 0; off >>= 1) part[j] += __shfl_xor_sync(0xffffffffu, part[j], off);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0)
        for (int j = 0; j < 18; ++j) red[warp][j] = part[j];
    __syncthreads();
    if (threadIdx.x < 18) {
        float s = 0.0f;
        for (int w8 = 0; w8 < 8; ++w8) s += red[w8][threadIdx.x];
        if (threadIdx.x < 17)
            atomicAdd(&grad[OW4 + threadIdx.x], s);      // W4[0..15] then b4 (OB4 = OW4 + 16)
        else
            atomicAdd(loss, s);
    }
}

// ------------------------------------------------------- optimiser / weights
// TA copies of every parameter (rounded once from the FP32 masters) and the transposed /
// flipped layouts the convolutions read.
template <typename TA>
struct Wts {
    TA* pf16;                   // [NPAR] flat
    TA *wf1, *wf2, *wf3;        // forward  [CI][9][CO]
    TA *wb3, *wb2;              // backward [CO_fwd][9][CI_fwd], taps flipped
};

template <typename TA>
__global__ void transform_kernel(const float* __restrict__ p, Wts<TA> w) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NPAR; q += gridDim.x * blockDim.x) {
        TA h;
        stf(&h, p[q]);
        w.pf16[q] = h;
        int o, c, tap, ci, co;
        TA* fwd = nullptr;
        TA* bwd = nullptr;
        int off;
        if (q < OB1) {
            off = q - OW1; ci = 1; co = 16; fwd = w.wf1;
        } else if (q >= OW2 && q < OB2) {
            off = q - OW2; ci = 16; co = 32; fwd = w.wf2; bwd = w.wb2;
        } else if (q >= OW3 && q < OB3) {
            off = q - OW3; ci = 32; co = 16; fwd = w.wf3; bwd = w.wb3;
        } else {
            continue;
        }
        o = off / (ci * 9);
        c = (off / 9) % ci;
        tap = off % 9;
        fwd[(c * 9 + tap) * co + o] = h;                         // [c][tap][o]
        if (bwd) bwd[(o * 9 + (8 - tap)) * ci + c] = h;          // [o][8 - tap][c]
    }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1t, float b2t) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < NPAR; q += gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.0f - b1) * gq;
        const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq / (1.0f - b1t)) / (sqrtf(vq / (1.0f - b2t)) + eps);
    }
}

// ------------------------------------------------------------ patch stats
// One CTA per patch: gather its 4096 powers, bitonic-sort a copy for the median, sort the
// absolute deviations for the MAD, then write Eq. 4 flags and the compressed network input.
__device__ void bitonic4096(float* s) {
    for (int k = 2; k <= PHW; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < PHW; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const float a = s[i], b = s[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(1024) patch_kernel(const float* __restrict__ P, int n_dump, int n_chan, float M,
                                                     __half* __restrict__ x, uint8_t* __restrict__ flags,
                                                     float* __restrict__ stats) {
    __shared__ float v[PHW];
    __shared__ float s[PHW];
    const int nkw = n_chan / PW, ndw = n_dump / PH;
    const int b = blockIdx.x;
    const int kw = b % nkw, dw = (b / nkw) % ndw, i = b / (nkw * ndw);
    for (int q = threadIdx.x; q < PHW; q += blockDim.x) {
        const int h = q / PW, w = q % PW;
        const float val = P[(static_cast<int64_t>(i) * n_dump + dw * PH + h) * n_chan + kw * PW + w];
        v[q] = val;
        s[q] = val;
    }
    __syncthreads();
    bitonic4096(s);
    const float med = 0.5f * (s[PHW / 2 - 1] + s[PHW / 2]);
    __syncthreads();
    for (int q = threadIdx.x; q < PHW; q += blockDim.x) s[q] = fabsf(v[q] - med);
    __syncthreads();
    bitonic4096(s);
    const float mad = 0.5f * (s[PHW / 2 - 1] + s[PHW / 2]);
    const float sig = mad / 0.6745f;
    for (int q = threadIdx.x; q < PHW; q += blockDim.x) {
        const float dev = v[q] - med;
        const int64_t o = static_cast<int64_t>(b) * PHW + q;
        if (flags) flags[o] = fabsf(dev) > M * sig ? 1 : 0;
        if (x) {
            const float u = sig > 0.0f ? dev / sig : 0.0f;
            x[o] = __float2half_rn(copysignf(log1pf(fabsf(u)), u));
        }
    }
    if (stats && threadIdx.x == 0) {
        stats[2 * b] = med;
        stats[2 * b + 1] = mad;
    }
}

}  // namespace

// ===================================================================== C ABI

struct rfi_net {
    int max_batch = 0;
    int step = 0;
    int fp32 = 0;                        // weights and activations in FP32 (rfi_create_fp32), else FP16
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *loss = nullptr;
    void* w[6] = {};                     // Wts<TA>: pf16, wf1, wf2, wf3, wb3, wb2
    void *A1 = nullptr, *A2 = nullptr, *A3 = nullptr;   // TA activations
    float *dA1 = nullptr, *dA2 = nullptr, *dA3 = nullptr;
    int n_sm = 0;
};

namespace {

int rfail(int code, const char* what, cudaError_t e = cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s%s%s", what, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
    gbx::set_last_error(buf);
    return code;
}

#define RCU(call)                                                     \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return rfail(CORR_E_CUDA, #call, e_);  \
    } while (0)

template <typename TA>
Wts<TA> wts(rfi_net* n) {
    Wts<TA> w;
    w.pf16 = static_cast<TA*>(n->w[0]);
    w.wf1 = static_cast<TA*>(n->w[1]);
    w.wf2 = static_cast<TA*>(n->w[2]);
    w.wf3 = static_cast<TA*>(n->w[3]);
    w.wb3 = static_cast<TA*>(n->w[4]);
    w.wb2 = static_cast<TA*>(n->w[5]);
    return w;
}

template <int CI, int CO, int MODE, typename TIN, typename TA>
cudaError_t conv(const void* in, const TA* act, const TA* w, const TA* bias, void* out, int B, cudaStream_t s) {
    const size_t smem = conv_smem<CI, CO>();
    auto kern = conv3x3_kernel<CI, CO, MODE, TIN, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<B * kTiles, 256, smem, s>>>(in, act, w, bias, out);
    return cudaGetLastError();
}

template <int CI, int CO, typename TIN, typename TA>
cudaError_t wgrad(const TIN* A, const float* dA, const TA* act, float* dW, float* db, int B, int n_sm,
                  cudaStream_t s) {
    const size_t smem = wgrad_smem<CI, CO>();
    auto kern = wgrad_kernel<CI, CO, TIN, TA>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int n_tiles = B * kTiles;
    const int grid = std::max(1, std::min(n_tiles, 4 * n_sm));
    kern<<<grid, 256, smem, s>>>(A, dA, act, dW, db, n_tiles);
    return cudaGetLastError();
}

template <typename TA>
int forward_t(rfi_net* n, const uint16_t* x, int B, cudaStream_t s) {
    const Wts<TA> w = wts<TA>(n);
    TA *A1 = static_cast<TA*>(n->A1), *A2 = static_cast<TA*>(n->A2), *A3 = static_cast<TA*>(n->A3);
    RCU((conv<1, 16, 0, __half, TA>(x, nullptr, w.wf1, w.pf16 + OB1, A1, B, s)));
    RCU((conv<16, 32, 0, TA, TA>(A1, nullptr, w.wf2, w.pf16 + OB2, A2, B, s)));
    RCU((conv<32, 16, 0, TA, TA>(A2, nullptr, w.wf3, w.pf16 + OB3, A3, B, s)));
    return CORR_OK;
}

template <typename TA>
int forward_backward_t(rfi_net* n, const uint16_t* x, const uint8_t* mask, int B, cudaStream_t s) {
    RCU(cudaMemsetAsync(n->g, 0, sizeof(float) * NPAR, s));
    RCU(cudaMemsetAsync(n->loss, 0, sizeof(float), s));
    if (int rc = forward_t<TA>(n, x, B, s)) return rc;
    const Wts<TA> w = wts<TA>(n);
    TA *A1 = static_cast<TA*>(n->A1), *A2 = static_cast<TA*>(n->A2), *A3 = static_cast<TA*>(n->A3);
    const int64_t npx = static_cast<int64_t>(B) * PHW;
    head_kernel<TA><<<static_cast<int>((npx + 255) / 256), 256, 0, s>>>(A3, mask, w.pf16, B, 1.0f / npx, n->dA3,
                                                                         n->g, n->loss, nullptr);
    RCU(cudaGetLastError());
    RCU((wgrad<32, 16, TA, TA>(A2, n->dA3, A3, n->g + OW3, n->g + OB3, B, n->n_sm, s)));
    RCU((conv<16, 32, 1, TA, TA>(n->dA3, A3, w.wb3, nullptr, n->dA2, B, s)));
    RCU((wgrad<16, 32, TA, TA>(A1, n->dA2, A2, n->g + OW2, n->g + OB2, B, n->n_sm, s)));
    RCU((conv<32, 16, 1, TA, TA>(n->dA2, A2, w.wb2, nullptr, n->dA1, B, s)));
    RCU((wgrad<1, 16, __half, TA>(reinterpret_cast<const __half*>(x), n->dA1, A1, n->g + OW1, n->g + OB1, B,
                                  n->n_sm, s)));
    return CORR_OK;
}

int forward(rfi_net* n, const uint16_t* x, int B, cudaStream_t s) {
    return n->fp32 ? forward_t<float>(n, x, B, s) : forward_t<__half>(n, x, B, s);
}

int forward_backward(rfi_net* n, const uint16_t* x, const uint8_t* mask, int B, cudaStream_t s) {
    return n->fp32 ? forward_backward_t<float>(n, x, mask, B, s) : forward_backward_t<__half>(n, x, mask, B, s);
}

int transform(rfi_net* n, cudaStream_t s) {
    if (n->fp32)
        transform_kernel<float><<<(NPAR + 255) / 256, 256, 0, s>>>(n->p, wts<float>(n));
    else
        transform_kernel<__half><<<(NPAR + 255) / 256, 256, 0, s>>>(n->p, wts<__half>(n));
    RCU(cudaGetLastError());
    return CORR_OK;
}

int head_infer(rfi_net* n, int B, float* prob, cudaStream_t s) {
    const int64_t npx = static_cast<int64_t>(B) * PHW;
    const int grid = static_cast<int>((npx + 255) / 256);
    if (n->fp32)
        head_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(n->A3), nullptr, wts<float>(n).pf16, B, 0.0f,
                                                nullptr, nullptr, nullptr, prob);
    else
        head_kernel<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(n->A3), nullptr, wts<__half>(n).pf16, B,
                                                 0.0f, nullptr, nullptr, nullptr, prob);
    RCU(cudaGetLastError());
    return CORR_OK;
}

int check_batch(rfi_net* n, const void* x, int B) {
    if (!n) return rfail(CORR_E_INVAL, "null network");
    if (!x || B < 1 || B > n->max_batch) return rfail(CORR_E_INVAL, "batch must be 1..max_batch with inputs given");
    return CORR_OK;
}

int create(rfi_net_t** out, int max_batch, int fp32) {
    if (!out || max_batch < 1) return rfail(CORR_E_INVAL, "rfi_create: bad arguments");
    *out = nullptr;
    rfi_net* n = new rfi_net();
    n->max_batch = max_batch;
    n->fp32 = fp32;
    auto bail = [&](cudaError_t e) {
        rfi_destroy(n);
        return rfail(CORR_E_NOMEM, "rfi_create: allocation", e);
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->n_sm, cudaDevAttrMultiProcessorCount, dev);
    const size_t px = static_cast<size_t>(max_batch) * PHW;
    const size_t ta = fp32 ? sizeof(float) : sizeof(__half);
    void** f32[] = {reinterpret_cast<void**>(&n->p), reinterpret_cast<void**>(&n->m), reinterpret_cast<void**>(&n->v),
                    reinterpret_cast<void**>(&n->g)};
    for (void** q : f32)
        if (e == cudaSuccess) e = cudaMalloc(q, sizeof(float) * NPAR);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->loss), sizeof(float));
    const size_t wn[6] = {NPAR, 144, 4608, 4608, 4608, 4608};
    for (int q = 0; q < 6; ++q)
        if (e == cudaSuccess) e = cudaMalloc(&n->w[q], ta * wn[q]);
    if (e == cudaSuccess) e = cudaMalloc(&n->A1, ta * px * 16);
    if (e == cudaSuccess) e = cudaMalloc(&n->A2, ta * px * 32);
    if (e == cudaSuccess) e = cudaMalloc(&n->A3, ta * px * 16);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->dA1), sizeof(float) * px * 16);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->dA2), sizeof(float) * px * 32);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->dA3), sizeof(float) * px * 16);
    if (e != cudaSuccess) return bail(e);
    for (void** q : f32)
        if ((e = cudaMemset(*q, 0, sizeof(float) * NPAR)) != cudaSuccess) return bail(e);
    if (transform(n, nullptr) != CORR_OK || cudaDeviceSynchronize() != cudaSuccess)
        return bail(cudaGetLastError());
    *out = n;
    return CORR_OK;
}

}  // namespace

extern "C" {

int rfi_n_params(void) { return NPAR; }

int rfi_create(rfi_net_t** out, int max_batch) { return create(out, max_batch, 0); }

int rfi_create_fp32(rfi_net_t** out, int max_batch) { return create(out, max_batch, 1); }

int rfi_destroy(rfi_net_t* n) {
    if (!n) return CORR_OK;
    void* bufs[] = {n->p, n->m, n->v, n->g, n->loss, n->w[0], n->w[1], n->w[2], n->w[3], n->w[4],
                    n->w[5], n->A1, n->A2, n->A3, n->dA1, n->dA2, n->dA3};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete n;
    return CORR_OK;
}

int rfi_set_params(rfi_net_t* n, const float* params) {
    if (!n || !params) return rfail(CORR_E_INVAL, "rfi_set_params: null argument");
    for (int q = 0; q < NPAR; ++q)
        if (!std::isfinite(params[q])) return rfail(CORR_E_INVAL, "rfi_set_params: non-finite parameter");
    RCU(cudaMemcpy(n->p, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
    RCU(cudaMemset(n->m, 0, sizeof(float) * NPAR));
    RCU(cudaMemset(n->v, 0, sizeof(float) * NPAR));
    n->step = 0;
    if (int rc = transform(n, nullptr)) return rc;
    RCU(cudaDeviceSynchronize());
    return CORR_OK;
}

int rfi_get_params(rfi_net_t* n, float* params) {
    if (!n || !params) return rfail(CORR_E_INVAL, "rfi_get_params: null argument");
    RCU(cudaDeviceSynchronize());
    RCU(cudaMemcpy(params, n->p, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int rfi_loss_grad(rfi_net_t* n, const uint16_t* x, const uint8_t* mask, int B, float* loss, float* grad,
                  void* stream) {
    if (int rc = check_batch(n, x, B)) return rc;
    if (!mask || !loss) return rfail(CORR_E_INVAL, "rfi_loss_grad: mask and loss are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = forward_backward(n, x, mask, B, s)) return rc;
    RCU(cudaStreamSynchronize(s));
    RCU(cudaMemcpy(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost));
    *loss /= static_cast<float>(static_cast<int64_t>(B) * PHW);
    if (grad) RCU(cudaMemcpy(grad, n->g, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
    return CORR_OK;
}

int rfi_train_step(rfi_net_t* n, const uint16_t* x, const uint8_t* mask, int B, float lr, float* loss,
                   void* stream) {
    if (int rc = check_batch(n, x, B)) return rc;
    if (!mask || !(lr > 0.0f)) return rfail(CORR_E_INVAL, "rfi_train_step: mask required and lr > 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = forward_backward(n, x, mask, B, s)) return rc;
    n->step += 1;
    const float b1t = std::pow(0.9f, static_cast<float>(n->step)), b2t = std::pow(0.999f, static_cast<float>(n->step));
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(n->p, n->m, n->v, n->g, lr, b1t, b2t);
    RCU(cudaGetLastError());
    if (int rc = transform(n, s)) return rc;
    if (loss) {
        RCU(cudaStreamSynchronize(s));
        RCU(cudaMemcpy(loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost));
        *loss /= static_cast<float>(static_cast<int64_t>(B) * PHW);
    }
    return CORR_OK;
}

int rfi_infer(rfi_net_t* n, const uint16_t* x, int B, float* prob, void* stream) {
    if (int rc = check_batch(n, x, B)) return rc;
    if (!prob) return rfail(CORR_E_INVAL, "rfi_infer: prob is null");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = forward(n, x, B, s)) return rc;
    return head_infer(n, B, prob, s);
}

int rfi_patches(const float* power, int n_in, int n_dump, int n_chan, float M, uint16_t* x, uint8_t* mad_flags,
                float* stats, void* stream) {
    if (!power || n_in < 1 || n_dump < PH || n_chan < PW || n_dump % PH || n_chan % PW || !(M > 0.0f))
        return rfail(CORR_E_INVAL, "rfi_patches: need n_dump, n_chan multiples of 64 and M > 0");
    const int B = n_in * (n_dump / PH) * (n_chan / PW);
    patch_kernel<<<B, 1024, 0, static_cast<cudaStream_t>(stream)>>>(power, n_dump, n_chan, M,
                                                                    reinterpret_cast<__half*>(x), mad_flags, stats);
    RCU(cudaGetLastError());
    return CORR_OK;
}

}  // extern "C"
