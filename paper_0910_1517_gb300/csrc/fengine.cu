// fengine.cu -- F-engine of the FX correlator for sm_103a: launches of the kernels in
// fengine_wfft.cuh and fengine_impl.cuh for single integrations, the per-integration phasor
// set-up, the RFI stage's power dumps and the beam averaging.
#include <cmath>
#include <vector>

#include "fengine_wfft.cuh"

namespace gbx {
namespace {
__global__ void phasor_setup_kernel(int n_ant, int n_chan, int n_fft, int n_int, int64_t g0_val,
                                    const int64_t* __restrict__ g0_ptr,
                                    const double* __restrict__ tau, const double* __restrict__ phi0,
                                    const double* __restrict__ rate, float2* __restrict__ pf,
                                    float2* __restrict__ ff, int* __restrict__ D) {
    const int64_t g0 = g0_ptr ? *g0_ptr : g0_val;
    const int64_t n1 = static_cast<int64_t>(n_ant) * n_chan, n2 = static_cast<int64_t>(n_ant) * n_int;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < n1 + n2 + n_ant;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (q < n1) {
            const int a = static_cast<int>(q / n_chan), k = static_cast<int>(q % n_chan);
            pf[q] = model_fstc_phasor(tau[a], k, n_fft);
        } else if (q < n1 + n2) {
            const int64_t r = q - n1;
            const int a = static_cast<int>(r / n_int), t = static_cast<int>(r % n_int);
            ff[r] = model_fringe_phasor(phi0[a], rate[a], g0 + t);
        } else {
            const int a = static_cast<int>(q - n1 - n2);
            D[a] = model_int_delay(tau[a]);
        }
    }
}

__global__ void twiddle_kernel(int n_fft, int count, float2* __restrict__ tw) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        double num, den, sn, cs;
        fengine_tw_angle(n_fft, e, num, den);
        sincospi(2.0 * num / den, &sn, &cs);
        tw[e] = make_float2(static_cast<float>(cs), static_cast<float>(-sn));
    }
}

// grid.x: dumps, grid.y: 32-channel groups; lane = channel, warp rows step over inputs
__global__ void power_dump_kernel(const float* __restrict__ spec, int n_in, int n_chan, int n_int, int dump,
                                  float* __restrict__ P, bool quad) {
    const int d = blockIdx.x, k = blockIdx.y * 32 + threadIdx.x;
    if (k >= n_chan) return;
    const int tb = tb_fp32(n_chan);
    const int Rp = rows_fp32(n_in), ntb = n_int / tb, n_dump = n_int / dump;
    const int kb0 = d * dump / tb, nkb = dump / tb;
    for (int i = threadIdx.y; i < n_in; i += blockDim.y) {
        float acc = 0.0f;
        for (int kb = kb0; kb < kb0 + nkb; ++kb) {
            if (quad) {   // one 64-byte piece: 8 re then 8 im values, summed in the order of the other layout
                const float4* pc = reinterpret_cast<const float4*>(spec + f32q_piece(k, kb, i, ntb, n_in));
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float4 v = pc[(m >> 1) + 2 * (m & 1)];   // re 0-3, im 0-3, re 4-7, im 4-7
                    acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
                }
                continue;
            }
            const float* blk = spec + (static_cast<int64_t>(k) * ntb + kb) * Rp * tb;
            for (int e = 0; e < tb; e += 4) {            // one 4-frame granule of each row at a time
                const float4 re = *reinterpret_cast<const float4*>(blk + fp32_off(2 * i, e, tb));
                const float4 im = *reinterpret_cast<const float4*>(blk + fp32_off(2 * i + 1, e, tb));
                acc += re.x * re.x + re.y * re.y + re.z * re.z + re.w * re.w;
                acc += im.x * im.x + im.y * im.y + im.z * im.z + im.w * im.w;
            }
        }
        P[(static_cast<int64_t>(i) * n_dump + d) * n_chan + k] = acc;
    }
}

__global__ void beam_average_kernel(const float* __restrict__ raw, float* __restrict__ out, int n_int, int n_chan,
                                    int beam_avg) {
    const int n_out = n_int / beam_avg;
    const int64_t total = 2LL * n_out * n_chan;
    const float inv = 1.0f / beam_avg;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(q % n_chan);
        const int64_t bt = q / n_chan;
        const int b = static_cast<int>(bt / n_out), to = static_cast<int>(bt % n_out);
        const float* src = raw + (static_cast<int64_t>(b) * n_int + static_cast<int64_t>(to) * beam_avg) * n_chan + k;
        float acc = 0.0f;
        for (int j = 0; j < beam_avg; ++j) acc += src[static_cast<int64_t>(j) * n_chan];
        out[q] = acc * inv;
    }
}

}  // namespace

cudaError_t launch_fengine_twiddles(int n_fft, float2* tw, cudaStream_t s) {
    const int count = fengine_tw_count(n_fft);
    twiddle_kernel<<<(count + 255) / 256, 256, 0, s>>>(n_fft, count, tw);
    return cudaGetLastError();
}

cudaError_t launch_fengine(const FeParams& p, int mode, cudaStream_t s) {
    if (p.n_chan * 2 != p.n_fft) return cudaErrorInvalidValue;
    switch (mode) {
        case OUT_FP32: return launch_w_mode<OUT_FP32>(p, s);
        case OUT_F16: return launch_w_mode<OUT_F16>(p, s);
        case OUT_F32Q: return launch_w_mode<OUT_F32Q>(p, s);
        case OUT_I8B: return launch_w_mode<OUT_I8B>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

bool fengine_clustered(int n_chan, int mode) {
    return n_chan == 2048 && (mode == OUT_F16 || mode == OUT_I8B);
}

cudaError_t launch_phasor_setup(int n_ant, int n_chan, int n_fft, int n_int, int64_t g0, const double* tau,
                                const double* phi0, const double* rate, float2* pf, float2* ff, int* D,
                                cudaStream_t s, const int64_t* g0_dev) {
    const int64_t total = static_cast<int64_t>(n_ant) * (n_chan + n_int) + n_ant;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4096));
    phasor_setup_kernel<<<grid, 256, 0, s>>>(n_ant, n_chan, n_fft, n_int, g0, g0_dev, tau, phi0, rate, pf, ff, D);
    return cudaGetLastError();
}

cudaError_t launch_power_dumps(const float* spec, int n_in, int n_chan, int n_int, int dump, float* P,
                               cudaStream_t s, bool quad) {
    const int tb = tb_fp32(n_chan);
    if (dump < tb || dump % tb || n_int % dump) return cudaErrorInvalidValue;
    const dim3 grid(n_int / dump, (n_chan + 31) / 32), block(32, 8);
    power_dump_kernel<<<grid, block, 0, s>>>(spec, n_in, n_chan, n_int, dump, P, quad);
    return cudaGetLastError();
}

cudaError_t launch_beam_average(const float* raw, float* out, int n_int, int n_chan, int beam_avg,
                                cudaStream_t s) {
    const int64_t total = 2LL * (n_int / beam_avg) * n_chan;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 8192));
    beam_average_kernel<<<grid, 256, 0, s>>>(raw, out, n_int, n_chan, beam_avg);
    return cudaGetLastError();
}

}  // namespace gbx
