// xengine_fp32.cu -- the plain FP32 X-engine on CUDA cores (Sec. 2.1 MAC).
//
// A persistent CTA takes one work unit at a time: a channel, or one of P equal
// frame ranges of a channel (P = 2 or 4 when that spreads the units evenly over
// the resident CTAs; a second kernel then adds the P partial visibility sets in
// a fixed order).  Its threads tile the upper triangle of the n_in x n_in complex
// visibility matrix into 4x4 input blocks (I <= J); each thread keeps its 16
// complex sums in registers and walks over the frames.  Frames stream into shared
// memory as the F-engine's FP32 K-blocks (TB frames x Rp rows in 16-byte granules)
// by TMA-engine bulk copies into a ring of stages.  Sums are kept per 256-frame
// chunk and added into running sums in shared memory, which bounds the rounding
// error of long integrations.  In the self-polar (total-intensity) mode with two
// polarisations the tiles are 4x4 antenna blocks of one polarisation (products RR*
// or LL* only): half the tiles, half the multiply-adds (Sec. 2.1 sizes the MAC so).
#include "common.cuh"
#include "fengine.cuh"
#include "xengine.cuh"

namespace gbx {
namespace {

constexpr int kStageFrames = 32;            // frames per stage
constexpr int kStages = 3;
constexpr int kChunkSlices = 64;            // 256 frames (64 slices of 4) per FP32 partial sum

__device__ __forceinline__ void decode_tri(int idx, int nb, int& I, int& J) {
    I = 0;
    int rem = idx;
    while (rem >= nb - I) {
        rem -= nb - I;
        ++I;
    }
    J = I + rem;
}

// TB: frames per K-block of the FP32 layout (4 or 8); a K-block is TB/4 slices of 4 frames,
// each slice one 16-byte granule per row
// SELF: self-polar mode with n_pol = 2 (tiles of one polarisation's antennas)
template <int MAXT, int TB, bool SELF>
__global__ void __launch_bounds__(MAXT) xengine_fp32_kernel(const XParams p, int n_split) {
    constexpr int TQ = TB / 4, KBS = kStageFrames / TB;   // slices per K-block, K-blocks per stage
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ __align__(8) uint64_t empty[kStages];
    const int R = rows_fp32(p.n_in);             // rows per K-block, a multiple of 8
    const int stage_bytes = kStageFrames * R * 4;
    float* part = reinterpret_cast<float*>(smem + kStages * stage_bytes);   // [32][blockDim] chunk sums
    // full: 4x4 blocks of inputs; self: 4x4 blocks of antennas of polarisation pol
    const int nb = SELF ? (p.n_ant + 3) / 4 : (p.n_in + 3) / 4;
    const int n_tri = nb * (nb + 1) / 2;
    const int n_work = SELF ? 2 * n_tri : n_tri;
    const int tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
    const bool active = tid < n_work;
    int I = 0, J = 0;
    const int pol = SELF && tid >= n_tri ? 1 : 0;
    if (active) decode_tri(tid - pol * n_tri, nb, I, J);
    // self: antenna 4I + ii of polarisation pol is input 8I + 2 ii + pol: row group 2I + (ii >> 1),
    // position 2 (ii & 1) + pol in it; groups past the last row (antennas beyond n_ant, never
    // written out) read group 0 instead of running off the K-block
    const int n_grp = R / 8;
    const int gi0 = SELF ? min(2 * I, n_grp - 1) : I, gi1 = SELF ? min(2 * I + 1, n_grp - 1) : I;
    const int gj0 = SELF ? min(2 * J, n_grp - 1) : J, gj1 = SELF ? min(2 * J + 1, n_grp - 1) : J;
    const int ntb = p.n_int / TB;
    const int nkb_u = ntb / n_split;                                 // K-blocks per work unit
    const int n_stage_ch = (nkb_u + KBS - 1) / KBS;                  // stages per unit
    const int n_units = p.n_chan * n_split;
    const int n_ch_mine = (n_units - static_cast<int>(blockIdx.x) + gridDim.x - 1) / gridDim.x;
    const int total = n_ch_mine * n_stage_ch;
    const float* spec = static_cast<const float*>(p.spec);

    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], nthr / 32);
        }
        fence_mbar_init();
    }
    for (int e = 0; e < 32; ++e) part[e * nthr + tid] = 0.0f;
    __syncthreads();
    auto issue = [&](int w) {
        const int slot = w % kStages;
        const int u = blockIdx.x + (w / n_stage_ch) * gridDim.x;     // unit: channel u / n_split
        const int kb0 = (w % n_stage_ch) * KBS;                      // within the unit's frames
        const int nkb = min(KBS, nkb_u - kb0);
        const uint32_t bytes = static_cast<uint32_t>(nkb) * R * TB * 4;
        const float* src =
            spec + (static_cast<int64_t>(u / n_split) * ntb + (u % n_split) * nkb_u + kb0) * R * TB;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[slot], bytes);
        bulk_g2s(smem + slot * stage_bytes, src, bytes, &full[slot]);
    };
    int issued = 0;                              // stages issued so far (thread 0)
    if (tid == 0)
        for (; issued < min(kStages - 1, total); ++issued) issue(issued);

    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    int kb_in_chunk = 0;
    bool ok = true;

    int w = 0;
    for (; w < total && ok; ++w) {
        const int slot = w % kStages;
        if (tid == 0 && w + kStages - 1 < total) {
            const int ws = w + kStages - 1;
            // the slot's previous stage (ws - kStages) must be released by every warp
            if (ws >= kStages &&
                !mbar_wait(&empty[ws % kStages], ((ws / kStages) - 1) & 1, p.err, ERR_WAIT_STAGE)) {
                ok = false;
            } else {
                issue(ws);
                issued = ws + 1;
            }
        }
        if (!mbar_wait(&full[slot], (w / kStages) & 1, p.err, ERR_WAIT_STAGE)) ok = false;
        const int kb0 = (w % n_stage_ch) * KBS;
        const int nkb = min(KBS, nkb_u - kb0);
        const float4* st = reinterpret_cast<const float4*>(smem + slot * stage_bytes);
        if (active && ok) {
            for (int sl = 0; sl < nkb * TQ; ++sl) {
                // rows 8I..8I+7 (and 8J..8J+7) are row group I (J): 8 TQ granules, granule g of group
                // G at position g ^ (G & 7), so a warp's loads of one granule spread over the banks
                const int h = sl % TQ;
                const float4* blk = st + (sl / TQ) * R * TQ;
                float4 ar[4], ai[4];
                if constexpr (!SELF) {
                    const float4* li = blk + 8 * TQ * I;
                    const int si = I & 7;
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        ar[ii] = li[(2 * ii * TQ + h) ^ si];
                        ai[ii] = li[((2 * ii + 1) * TQ + h) ^ si];
                    }
                } else {
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        const int G = (ii >> 1) ? gi1 : gi0, pos = 2 * (ii & 1) + pol;
                        const float4* li = blk + 8 * TQ * G;
                        ar[ii] = li[(2 * pos * TQ + h) ^ (G & 7)];
                        ai[ii] = li[((2 * pos + 1) * TQ + h) ^ (G & 7)];
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float4 br, bi;
                    if constexpr (!SELF) {
                        const float4* lj = blk + 8 * TQ * J;
                        br = lj[(2 * jj * TQ + h) ^ (J & 7)];
                        bi = lj[((2 * jj + 1) * TQ + h) ^ (J & 7)];
                    } else {
                        const int G = (jj >> 1) ? gj1 : gj0, pos = 2 * (jj & 1) + pol;
                        const float4* lj = blk + 8 * TQ * G;
                        br = lj[(2 * pos * TQ + h) ^ (G & 7)];
                        bi = lj[((2 * pos + 1) * TQ + h) ^ (G & 7)];
                    }
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        float2 c = acc[ii][jj];
                        // Y_i conj(Y_j) = (ar + i ai)(br - i bi)
                        c.x = fmaf(ar[ii].x, br.x, c.x); c.x = fmaf(ai[ii].x, bi.x, c.x);
                        c.y = fmaf(ai[ii].x, br.x, c.y); c.y = fmaf(-ar[ii].x, bi.x, c.y);
                        c.x = fmaf(ar[ii].y, br.y, c.x); c.x = fmaf(ai[ii].y, bi.y, c.x);
                        c.y = fmaf(ai[ii].y, br.y, c.y); c.y = fmaf(-ar[ii].y, bi.y, c.y);
                        c.x = fmaf(ar[ii].z, br.z, c.x); c.x = fmaf(ai[ii].z, bi.z, c.x);
                        c.y = fmaf(ai[ii].z, br.z, c.y); c.y = fmaf(-ar[ii].z, bi.z, c.y);
                        c.x = fmaf(ar[ii].w, br.w, c.x); c.x = fmaf(ai[ii].w, bi.w, c.x);
                        c.y = fmaf(ai[ii].w, br.w, c.y); c.y = fmaf(-ar[ii].w, bi.w, c.y);
                        acc[ii][jj] = c;
                    }
                }
                if (++kb_in_chunk == kChunkSlices) {   // fold this chunk's FP32 sums into the running ones
                    kb_in_chunk = 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            part[(8 * a + 2 * b) * nthr + tid] += acc[a][b].x;
                            part[(8 * a + 2 * b + 1) * nthr + tid] += acc[a][b].y;
                            acc[a][b] = make_float2(0.f, 0.f);
                        }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);  // this warp is done with the stage
        const bool ch_done = (w % n_stage_ch) == n_stage_ch - 1;
        if (ch_done && active && ok) {
            const int u = blockIdx.x + (w / n_stage_ch) * gridDim.x;
            const int k = u / n_split;
            const int n_bl = p.n_ant * (p.n_ant + 1) / 2, npp = p.self ? p.n_pol : p.n_pol * p.n_pol;
            float2* out = n_split == 1 ? p.vis
                                       : p.vis_part + static_cast<int64_t>(u % n_split) * p.n_chan * n_bl * npp;
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int i = 4 * I + ii, j = 4 * J + jj;
                    float* pr = &part[(8 * ii + 2 * jj) * nthr + tid];
                    float* pi = &part[(8 * ii + 2 * jj + 1) * nthr + tid];
                    const float2 v = make_float2(*pr + acc[ii][jj].x, *pi + acc[ii][jj].y);
                    *pr = 0.0f;
                    *pi = 0.0f;
                    acc[ii][jj] = make_float2(0.f, 0.f);
                    int a, pp, a2, qq;
                    if constexpr (SELF) {
                        a = 4 * I + ii;
                        a2 = 4 * J + jj;
                        pp = qq = pol;
                        if (a >= p.n_ant || a2 >= p.n_ant) continue;
                    } else {
                        if (i >= p.n_in || j >= p.n_in) continue;
                        a = i / p.n_pol, pp = i % p.n_pol, a2 = j / p.n_pol, qq = j % p.n_pol;
                        if (a > a2 || (p.self && pp != qq)) continue;
                    }
                    if (a > a2) continue;
                    const int bl = a * p.n_ant - a * (a - 1) / 2 + (a2 - a);
                    out[(static_cast<int64_t>(k) * n_bl + bl) * npp + vis_prod(p.self, p.n_pol, pp, qq)] = v;
                }
            kb_in_chunk = 0;
        }
        if (ch_done) kb_in_chunk = 0;
    }
    if (tid == 0) {
        // stages issued but never consumed (only after a failed wait) must land before exit
        for (int q = w; q < issued; ++q) mbar_wait(&full[q % kStages], (q / kStages) & 1, nullptr, 0);
    }
}

// vis = sum over s of part[s], s = 0 .. n_split - 1 in order
__global__ void vis_split_sum_kernel(const float2* __restrict__ part, float2* __restrict__ vis, int64_t n,
                                     int n_split) {
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < n;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float2 v = part[q];
        for (int s = 1; s < n_split; ++s) {
            const float2 x = part[static_cast<int64_t>(s) * n + q];
            v.x += x.x;
            v.y += x.y;
        }
        vis[q] = v;
    }
}

}  // namespace

cudaError_t launch_xengine_fp32(const XParams& p, int n_sm, cudaStream_t s) {
    const bool self2 = p.self && p.n_pol == 2;   // self-polar with one polarisation is the full mode
    const int nb = self2 ? (p.n_ant + 3) / 4 : (p.n_in + 3) / 4;
    const int n_work = (self2 ? 2 : 1) * nb * (nb + 1) / 2;
    const int threads = ((n_work + 31) / 32) * 32;
    if (threads > 544) return cudaErrorInvalidValue;
    const int tb = tb_fp32(p.n_chan);
    const size_t smem = kStages * (static_cast<size_t>(kStageFrames) * rows_fp32(p.n_in) * 4) +
                        32 * sizeof(float) * threads;
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        int per_sm = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        const int slots = n_sm * std::max(per_sm, 1);
        // frame split: the fewest of 1, 2, 4 parts that keep the last round of units at least
        // 90% full (each part a whole number of stages)
        int n_split = 1;
        if (p.vis_part) {
            double best = 0.0;
            for (int P = 1; P <= std::min(4, p.max_split); P *= 2) {
                if (P > 1 && (p.n_int / tb) % (P * (kStageFrames / tb))) break;
                const long units = static_cast<long>(p.n_chan) * P;
                const long rounds = (units + slots - 1) / slots;
                const double eff = static_cast<double>(units) / (static_cast<double>(rounds) * slots);
                if (eff > best + 1e-9) {
                    best = eff;
                    n_split = P;
                }
                if (eff >= 0.9) break;
            }
        }
        const int grid = static_cast<int>(std::max(1L, std::min(static_cast<long>(p.n_chan) * n_split,
                                                                 static_cast<long>(slots))));
        kern<<<grid, threads, smem, s>>>(p, n_split);
        e = cudaGetLastError();
        if (e != cudaSuccess || n_split == 1) return e;
        const int64_t n = static_cast<int64_t>(p.n_chan) * (p.n_ant * (p.n_ant + 1) / 2) * (p.self ? p.n_pol : p.n_pol * p.n_pol);
        const int sgrid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 4 * n_sm));
        vis_split_sum_kernel<<<sgrid, 256, 0, s>>>(p.vis_part, p.vis, n, n_split);
        return cudaGetLastError();
    };
    if (self2) {
        if (tb == 8) return threads <= 256 ? go(xengine_fp32_kernel<256, 8, true>) : go(xengine_fp32_kernel<544, 8, true>);
        return threads <= 256 ? go(xengine_fp32_kernel<256, 4, true>) : go(xengine_fp32_kernel<544, 4, true>);
    }
    if (tb == 8) return threads <= 256 ? go(xengine_fp32_kernel<256, 8, false>) : go(xengine_fp32_kernel<544, 8, false>);
    return threads <= 256 ? go(xengine_fp32_kernel<256, 4, false>) : go(xengine_fp32_kernel<544, 4, false>);
}

}  // namespace gbx
