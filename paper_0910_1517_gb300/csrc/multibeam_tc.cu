// multibeam_tc.cu -- the phased beams of multibeam.cu (Sec. 2.2, 5) as a dense contraction on
// the tcgen05 tensor cores.  Per channel k, every beam voltage is
//   U_bp[t] = sum_a w[k][b][a] Y_{a,p}[t][k],
// in real form D = A B^T with A[(b, re|im)][(a, re|im)] the weights ([[wr, -wi], [wi, wr]]) and
// B[(p, t)][(a, re|im)] the spectra: M = 128 rows (up to 64 beams), K = 2 n_ant (padded to 16),
// N = n_pol x 64 frames per stage.  FP32 accuracy as in the FP32 X-engine form: both operands are
// split on chip into fp16 hi + lo (Veltkamp's split: hi exact to 11 bits, lo = v - hi exact) and
// D = Ah Bh^T + Ah Bl^T + Al Bh^T in FP32 TMEM accumulators (K is at most 128, so the tensor
// core's FP32 accumulation error stays at the level of the dropped Al Bl^T term).
//
// One CTA takes channel k and `span` frames.  Warp roles: 0 copies 64-frame FP32 stages (one
// bulk copy each, three in flight); 1 issues the MMAs into one of two 128-column accumulators;
// 8-15 convert each stage into the K-major fp16 hi/lo B tiles (two slots); 4-7 (the four TMEM
// lane quarters) drain an accumulator row per thread -- row 2b + c holds the re (c = 0) or im
// part of beam b for every (polarisation, frame) column -- and form the full-polar window
// means or the voltages, pairing with the neighbouring lane by shuffles.  Every wait is bounded.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "fengine.cuh"

namespace gbx {
namespace {

constexpr int kTcThreads = 512;
constexpr int kFrames = 64;                 // frames per stage
constexpr int kRows = 128;                  // M: 2 x beams
constexpr int kConv0 = 8, kConvW = 8;       // converter warps 8..15
constexpr int kConvT = kConvW * 32;
constexpr int kDrain0 = 4;                  // drain warps 4..7 (TMEM lane quarters 0..3)
constexpr uint32_t kTmemCols = 256;         // two accumulators of up to 128 columns
constexpr int kMaxF32Stages = 3;
constexpr size_t kSmemBudget = 220 * 1024;

struct TcShared {
    uint64_t f32full[kMaxF32Stages], f32empty[kMaxF32Stages];
    uint64_t full[2], empty[2];             // B slots: converted / read by the MMAs
    uint64_t accf[2], acce[2];              // accumulators: complete / drained
    uint64_t done;                          // every MMA of the CTA has completed
    uint32_t taddr;
    unsigned wmax;                          // bits of the channel's largest |weight component|
    int abort_flag;
    int consumed;                           // FP32 stages the converters have taken
};

struct TcGeo {
    int KC;                                 // K / 8 (16-byte K chunks)
    int N;                                  // MMA N = n_pol x 64
    int nf;                                 // FP32 stage buffers
    uint32_t a_bytes, b_bytes, f32_bytes;   // one hi (or lo) A tile, one hi B tile, one FP32 stage
};

__host__ __device__ inline TcGeo tc_geo(int n_ant, int n_pol, int n_in) {
    TcGeo g;
    const int K = ((2 * n_ant + 15) / 16) * 16;
    g.KC = K / 8;
    g.N = n_pol * kFrames;
    g.a_bytes = static_cast<uint32_t>(g.KC) * kRows * 16;
    g.b_bytes = static_cast<uint32_t>(g.KC) * g.N * 16;
    g.f32_bytes = static_cast<uint32_t>(rows_fp32(n_in)) * kFrames * 4;
    const size_t fixed = 2 * static_cast<size_t>(g.a_bytes) + 4 * static_cast<size_t>(g.b_bytes);
    g.nf = fixed >= kSmemBudget ? 0 : static_cast<int>((kSmemBudget - fixed) / g.f32_bytes);
    if (g.nf > kMaxF32Stages) g.nf = kMaxF32Stages;
    return g;
}

// Veltkamp split of 8 values into fp16 hi and lo words, on packed FP32x2 pairs (each lane rounds
// as the scalar operation: t = 8193 v, hi = t - (t - v), lo = v - hi)
__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
    uint32_t hw[4], lw[4];
    const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float2 v = make_float2(x[2 * m], x[2 * m + 1]);
        const float2 t = __fmul2_rn(v, make_float2(8193.0f, 8193.0f));
        const float2 hv = __ffma2_rn(__ffma2_rn(v, m1, t), m1, t);
        const float2 lv = __ffma2_rn(hv, m1, v);
        const __half2 hh = __floats2half2_rn(hv.x, hv.y);
        const __half2 ll = __floats2half2_rn(lv.x, lv.y);
        hw[m] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[m] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    hi = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// (v.x, v.y, v.z, v.w) rotated left by r (0..3): two stages of selects
__device__ __forceinline__ float4 rot4(float4 v, int r) {
    if (r & 1) v = make_float4(v.y, v.z, v.w, v.x);
    if (r & 2) v = make_float4(v.z, v.w, v.x, v.y);
    return v;
}

__global__ void __launch_bounds__(kTcThreads, 1)
multibeam_tc_kernel(const float* __restrict__ spec, int n_ant, int n_pol, int n_chan, int n_int,
                    const float2* __restrict__ w, int wstride, int n_beams, int products, int avg, int span,
                    float split_scale, float4* __restrict__ out, unsigned* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcShared sh;
    const int n_in = n_ant * n_pol, tb = tb_fp32(n_chan), Rp = rows_fp32(n_in);
    const TcGeo G = tc_geo(n_ant, n_pol, n_in);
    unsigned char* a_hi = smem;                                  // [KC][128][8] fp16
    unsigned char* a_lo = a_hi + G.a_bytes;
    unsigned char* b_base = a_lo + G.a_bytes;                    // slot s: hi at + 2 s b_bytes, lo after it
    unsigned char* f32_base = b_base + 4 * G.b_bytes;            // FP32 stages
    const int k = blockIdx.x, t0 = blockIdx.y * span, n_stage = span / kFrames;
    const int64_t ntb = n_int / tb;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    if (tid == 0) {
        for (int s = 0; s < G.nf; ++s) {
            mbar_init(&sh.f32full[s], 1);
            mbar_init(&sh.f32empty[s], kConvW);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.full[s], kConvW);
            mbar_init(&sh.empty[s], 1);
            mbar_init(&sh.accf[s], 1);
            mbar_init(&sh.acce[s], 128);
        }
        mbar_init(&sh.done, 1);
        fence_mbar_init();
        sh.abort_flag = 0;
        sh.consumed = 0;
        sh.wmax = 0u;
    }
    if (warp == 0) {
        tmem_alloc(&sh.taddr, kTmemCols);
        tmem_relinquish();
    }
    __syncthreads();
    // ---- the channel's weights: a power-of-two scale bringing the largest component near 2^13,
    // then the A tiles (every thread)
    const float2* wk = w + static_cast<int64_t>(k) * wstride;
    for (int i = tid; i < n_beams * n_ant; i += kTcThreads) {
        const float2 v = wk[i];
        atomicMax(&sh.wmax, __float_as_uint(fmaxf(fabsf(v.x), fabsf(v.y))));
    }
    __syncthreads();
    const float wmax = __uint_as_float(sh.wmax);
    const float wscale = wmax > 0.0f ? ldexpf(1.0f, 13 - ilogbf(wmax)) : 1.0f;
    for (int u = tid; u < G.KC * kRows; u += kTcThreads) {
        const int kc = u / kRows, m = u % kRows, b = m >> 1, cout = m & 1;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int kk = 8 * kc + j, a = kk >> 1, cin = kk & 1;
            float v = 0.0f;
            if (b < n_beams && a < n_ant) {
                const float2 q = wk[b * n_ant + a];
                v = cout == 0 ? (cin == 0 ? q.x : -q.y) : (cin == 0 ? q.y : q.x);
            }
            x[j] = v * wscale;
        }
        uint4 hi, lo;
        split8(x, hi, lo);
        *reinterpret_cast<uint4*>(a_hi + static_cast<size_t>(u) * 16) = hi;
        *reinterpret_cast<uint4*>(a_lo + static_cast<size_t>(u) * 16) = lo;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.taddr;
    volatile int* abort_flag = &sh.abort_flag;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int st = 0;
            for (; st < n_stage && !*abort_flag; ++st) {
                const int s = st % G.nf;
                if (!mbar_wait(&sh.f32empty[s], ((st / G.nf) & 1) ^ 1, err, ERR_WAIT_MMA)) {
                    *abort_flag = 1;
                    break;
                }
                const float* src = spec + (static_cast<int64_t>(k) * ntb + (t0 + st * kFrames) / tb) * Rp * tb;
                mbar_arrive_expect_tx(&sh.f32full[s], G.f32_bytes);
                bulk_g2s(f32_base + static_cast<size_t>(s) * G.f32_bytes, src, G.f32_bytes, &sh.f32full[s]);
            }
            // every issued copy lands before the CTA may exit
            for (int q = *(volatile int*)&sh.consumed; q < st; ++q)
                mbar_wait(&sh.f32full[q % G.nf], (q / G.nf) & 1, nullptr, 0);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_f16_f32(kRows, G.N);
            const uint32_t lbo_a = kRows * 16, lbo_b = static_cast<uint32_t>(G.N) * 16, sbo = 128;
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
            for (int st = 0; st < n_stage && !*abort_flag; ++st) {
                const int s = st & 1;
                if (!mbar_wait(&sh.full[s], (st >> 1) & 1, err, ERR_WAIT_STAGE) ||
                    !mbar_wait(&sh.acce[s], ((st >> 1) & 1) ^ 1, err, ERR_WAIT_EPI)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t bh = smem_u32(b_base + static_cast<size_t>(2 * s) * G.b_bytes);
                const uint32_t bl = bh + G.b_bytes;
                const uint32_t d = tmem + s * 128;
                for (int kk = 0; kk < G.KC / 2; ++kk) {
                    const uint64_t dah = smem_desc_noswizzle(ah + kk * 2 * lbo_a, lbo_a, sbo);
                    const uint64_t dal = smem_desc_noswizzle(al + kk * 2 * lbo_a, lbo_a, sbo);
                    const uint64_t dbh = smem_desc_noswizzle(bh + kk * 2 * lbo_b, lbo_b, sbo);
                    const uint64_t dbl = smem_desc_noswizzle(bl + kk * 2 * lbo_b, lbo_b, sbo);
                    umma_f16(d, dah, dbh, idesc, kk == 0 ? 0u : 1u);
                    umma_f16(d, dah, dbl, idesc, 1u);
                    umma_f16(d, dal, dbh, idesc, 1u);
                }
                umma_commit(&sh.empty[s]);      // the B slot is free once these MMAs finish
                umma_commit(&sh.accf[s]);       // the accumulator is complete
            }
            umma_commit(&sh.done);
            mbar_wait(&sh.done, 0, err, ERR_WAIT_MMA);
        }
    } else if (warp >= kConv0) {
        // ------------------------------------------------------------ converters
        const int ct = tid - kConv0 * 32;
        const int units = G.KC * n_pol * (kFrames / 4);   // at most 2 kConvT (K <= 128)
        // a thread's units are the same in every stage: their source offsets within an FP32 stage
        // (-1 for padding antennas) and their (polarisation, K chunk, frame quad), once
        constexpr int kMaxU = 2;
        int soff[kMaxU][8], uq[kMaxU];
#pragma unroll
        for (int m = 0; m < kMaxU; ++m) {
            const int u = ct + m * kConvT;
            const int tq = u % (kFrames / 4), p = (u / (kFrames / 4)) % n_pol, kc = u / ((kFrames / 4) * n_pol);
            const int f0 = 4 * tq, kb = f0 / tb, e0 = f0 % tb;
            uq[m] = u;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int kk = 8 * kc + j, a = kk >> 1;
                soff[m][j] = (u < units && a < n_ant) ? kb * Rp * tb + fp32_off(2 * (a * n_pol + p) + (kk & 1), e0, tb) : -1;
            }
        }
        for (int st = 0; st < n_stage; ++st) {
            const int fs = st % G.nf, s = st & 1;
            int ok = 1;
            if (lane == 0) {
                ok = !*abort_flag && mbar_wait(&sh.f32full[fs], (st / G.nf) & 1, err, ERR_WAIT_STAGE) &&
                     mbar_wait(&sh.empty[s], ((st >> 1) & 1) ^ 1, err, ERR_WAIT_MMA);
                if (!ok) *abort_flag = 1;
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const float* src = reinterpret_cast<const float*>(f32_base + static_cast<size_t>(fs) * G.f32_bytes);
            unsigned char* bh = b_base + static_cast<size_t>(2 * s) * G.b_bytes;
#pragma unroll
            for (int m = 0; m < kMaxU; ++m) {
                const int u = uq[m];
                if (u >= units) break;
                // unit: K chunk kc (antennas 4 kc .. 4 kc + 3, re and im), polarisation p, frames 4 tq .. 4 tq + 3
                const int tq = u % (kFrames / 4), p = (u / (kFrames / 4)) % n_pol, kc = u / ((kFrames / 4) * n_pol);
                const int f0 = 4 * tq;
                float4 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = soff[m][j] >= 0 ? *reinterpret_cast<const float4*>(src + soff[m][j]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = rot4(v[j], tq & 3);
#pragma unroll
                for (int e1 = 0; e1 < 4; ++e1) {
                    // frame f0 + e, rotated by tq so that the warp's 16-byte stores spread over
                    // the bank groups (lanes are 64 bytes apart); v[j] is already rotated, so
                    // component e1 is frame e
                    const int e = (e1 + tq) & 3;
                    float x[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        x[j] = (e1 == 0 ? v[j].x : e1 == 1 ? v[j].y : e1 == 2 ? v[j].z : v[j].w) * split_scale;
                    uint4 hi, lo;
                    split8(x, hi, lo);
                    const size_t off = (static_cast<size_t>(kc) * G.N + p * kFrames + f0 + e) * 16;
                    *reinterpret_cast<uint4*>(bh + off) = hi;
                    *reinterpret_cast<uint4*>(bh + G.b_bytes + off) = lo;
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (ct == 0) sh.consumed = st + 1;
                mbar_arrive(&sh.f32empty[fs]);
                mbar_arrive(&sh.full[s]);
            }
        }
    } else if (warp >= kDrain0) {
        // ------------------------------------------------------------ drain + products
        const int q = warp & 3, m = 32 * q + lane, b = m >> 1, c = m & 1;
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const float ds = 1.0f / (split_scale * wscale);   // D units -> voltage units (powers of two)
        const float sc = ds * ds / static_cast<float>(avg);
        const int n_out = n_int / avg;
        float s00 = 0.f, s11 = 0.f, s01 = 0.f, sx = 0.f;
        for (int st = 0; st < n_stage; ++st) {
            const int s = st & 1;
            if (!mbar_wait(&sh.accf[s], (st >> 1) & 1, err, ERR_WAIT_MMA)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            for (int h = 0; h < 2; ++h) {                      // 32 frames at a time
                uint32_t r0[32], r1[32];
                tmem_ld32(tmem + lane_off + s * 128 + h * 32, r0);
                if (n_pol == 2) tmem_ld32(tmem + lane_off + s * 128 + kFrames + h * 32, r1);
                tmem_wait_ld();
                if (h == 1) {
                    tc_fence_before();
                    mbar_arrive(&sh.acce[s]);                   // every column of this accumulator is read
                }
                const int f32 = st * kFrames + h * 32;          // first frame of these 32 in the CTA's span
                if (products == 1) {                            // voltages (avg 1)
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float u0 = __uint_as_float(r0[j]);
                        const float u1 = n_pol == 2 ? __uint_as_float(r1[j]) : 0.0f;
                        const float p0 = __shfl_xor_sync(0xffffffffu, u0, 1);
                        const float p1 = __shfl_xor_sync(0xffffffffu, u1, 1);
                        if (c == 0 && b < n_beams)
                            out[(static_cast<int64_t>(b) * n_out + t0 + f32 + j) * n_chan + k] =
                                make_float4(u0 * ds, p0 * ds, u1 * ds, p1 * ds);
                    }
                    continue;
                }
                // window complete after frame j when (j + 1) is a multiple of avg (avg <= 32: j is a
                // compile-time index, avg a power of two), or after the 32 when avg > 32
                auto flush = [&](int f_last) {                 // add the partner lane's half and write
                    const float a00 = s00 + __shfl_xor_sync(0xffffffffu, s00, 1);
                    const float a11 = s11 + __shfl_xor_sync(0xffffffffu, s11, 1);
                    const float a01 = s01 + __shfl_xor_sync(0xffffffffu, s01, 1);
                    const float ax = sx + __shfl_xor_sync(0xffffffffu, sx, 1);
                    if (c == 0 && b < n_beams)
                        out[(static_cast<int64_t>(b) * n_out + (t0 + f_last) / avg) * n_chan + k] =
                            make_float4(a00 * sc, a11 * sc, a01 * sc, ax * sc);
                    s00 = s11 = s01 = sx = 0.f;
                };
                // the 32 frames with the window length as a compile-time constant (A = 0: avg > 32,
                // at most one flush after the 32), so the flushes sit at fixed frames
                auto frames32 = [&](auto a_c) {
                    constexpr int A = decltype(a_c)::value;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float u0 = __uint_as_float(r0[j]);
                        const float u1 = n_pol == 2 ? __uint_as_float(r1[j]) : 0.0f;
                        const float p1 = __shfl_xor_sync(0xffffffffu, u1, 1);
                        s00 = fmaf(u0, u0, s00);
                        s11 = fmaf(u1, u1, s11);
                        s01 = fmaf(u0, u1, s01);
                        sx = fmaf(c == 0 ? -u0 : u0, p1, sx);      // re: -re0 im1, im: im0 re1
                        if constexpr (A > 0) {
                            if ((j + 1) % A == 0) flush(f32 + j);
                        }
                    }
                    if constexpr (A == 0) {
                        if (((f32 + 32) & (avg - 1)) == 0) flush(f32 + 31);
                    }
                };
                switch (avg) {
                    case 1: frames32(std::integral_constant<int, 1>{}); break;
                    case 2: frames32(std::integral_constant<int, 2>{}); break;
                    case 4: frames32(std::integral_constant<int, 4>{}); break;
                    case 8: frames32(std::integral_constant<int, 8>{}); break;
                    case 16: frames32(std::integral_constant<int, 16>{}); break;
                    case 32: frames32(std::integral_constant<int, 32>{}); break;
                    default: frames32(std::integral_constant<int, 0>{}); break;
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

bool multibeam_tc_supported(int n_ant, int n_pol, int n_chan, int n_int) {
    if (n_pol < 1 || n_pol > 2 || n_ant < 1 || 2 * n_ant > 128 || n_int % kFrames) return false;
    (void)n_chan;
    return tc_geo(n_ant, n_pol, n_ant * n_pol).nf >= 2;
}

cudaError_t launch_multibeam_tc(const float* spec, int n_ant, int n_pol, int n_chan, int n_int, const float2* w,
                                int wstride, int n_beams, int products, int avg, float split_scale, float4* out,
                                unsigned* err, cudaStream_t s) {
    if (!multibeam_tc_supported(n_ant, n_pol, n_chan, n_int) || n_beams < 1 || 2 * n_beams > kRows || avg < 1 ||
        (avg & (avg - 1)) || (products == 1 && avg != 1) || n_int % (avg > kFrames ? avg : kFrames))
        return cudaErrorInvalidValue;
    // frames per CTA: a multiple of 64 and of avg dividing n_int, up to 2048
    int span = avg > kFrames ? avg : kFrames;
    while (span < 2048 && n_int % (2 * span) == 0) span *= 2;
    const TcGeo G = tc_geo(n_ant, n_pol, n_ant * n_pol);
    const size_t smem = 2 * static_cast<size_t>(G.a_bytes) + 4 * static_cast<size_t>(G.b_bytes) +
                        static_cast<size_t>(G.nf) * G.f32_bytes;
    cudaError_t e = cudaFuncSetAttribute(multibeam_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const dim3 grid(n_chan, n_int / span);
    multibeam_tc_kernel<<<grid, kTcThreads, smem, s>>>(spec, n_ant, n_pol, n_chan, n_int, w, wstride, n_beams,
                                                        products, avg, span, split_scale, out, err);
    return cudaGetLastError();
}

}  // namespace gbx
