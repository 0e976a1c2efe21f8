// fengine.cuh -- launch interface of the F-engine (integer delay, real FFT,
// Eq. 2 phasor, beams, requantisation) and of the per-integration phasor set-up.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>
#include <vector>

namespace gbx {

enum OutMode : int { OUT_FP32 = 0, OUT_F16 = 2, OUT_F32Q = 3, OUT_I8B = 4 };

// Spectra hand-off layout ("K-block layout"), shared by every X-engine:
//   S[k][kb][r][TB]   k channel, kb = t / TB, r = 2*i + c (c = 0 re, 1 im), TB = t % TB
// One (k, kb) block holds every input's rows for TB consecutive frames.
// fp16 (tensor-core X-engine): TB = 8, R = 2 n_in unswizzled rows of 16 bytes -- exactly
// the no-swizzle K-major canonical layout of a tcgen05 operand tile (OUT_F16).  OUT_I8B writes
// the int8 requantised values as bytes in the channel-quad arrangement (i8q_piece) that the
// X-engine gathers by TMA into [kb][r][8 bytes] and widens to fp16 on chip.
// FP32 (CUDA-core X-engine): TB = tb_fp32(n_chan) = 8 frames (4 when an F-engine CTA covers
// only 4 frames, n_chan = 2048), rows padded to Rp = round_up(2 n_in, 8).  The block is cut
// into 16-byte granules of 4 frames of one row, 8 rows (one input group of 4) per row group
// G, and granule g = (r % 8) * TB/4 + (frame % TB) / 4 of group G sits at position
// g ^ (G & 7): the CUDA-core X-engine's threads, which read the same granule of different
// row groups at once, then hit distinct banks, while the re and im rows of one input over
// the TB frames stay one contiguous, aligned 8 * TB-byte piece (the F-engine writes each
// piece in one store instruction).  Padding rows only meet padding inputs, whose products
// are never kept.
constexpr int kTbHalf = 8;

__host__ __device__ constexpr int tb_fp32(int n_chan) { return n_chan >= 2048 ? 4 : 8; }
__host__ __device__ constexpr int rows_fp32(int n_in) { return ((2 * n_in + 7) / 8) * 8; }
// float offset of row r, frame e (0 <= e < tb) inside one FP32 K-block
__host__ __device__ constexpr int fp32_off(int r, int e, int tb) {
    const int G = r >> 3, g = (r & 7) * (tb >> 2) + (e >> 2);
    return G * 8 * tb + ((g ^ (G & 7)) << 2) + (e & 3);
}

// FP32 spectra in the channel-quad layout (OUT_F32Q, the F-to-X hand-off of CORR_FP32TC for
// n_chan <= 1024): the piece of channel k, 8-frame K-block kb and input i -- 8 re then 8 im FP32
// values, 64 bytes -- at float offset
//   (((k / 4) * ntb + kb) * n_in + i) * 64 + (k % 4) * 16
// i.e. [k / 4][kb][i][k % 4][16]: the F-engine, which holds one input of 8 frames for every
// channel, writes 256 contiguous bytes per channel quad (instead of 64-byte pieces 4 MB apart,
// which leave its stores at a third of the HBM bandwidth), and a channel's stage is a strided
// gather that one 5-D TMA tensor copy performs ([kb][i][16] = [kb][row 2i + c][8 frames]).
__host__ __device__ constexpr int64_t f32q_piece(int k, int64_t kb, int i, int64_t ntb, int n_in) {
    return (((static_cast<int64_t>(k) >> 2) * ntb + kb) * n_in + i) * 64 + (k & 3) * 16;
}
// The same channel-quad arrangement for the int8 bytes of OUT_I8B: the piece of (k, kb, i) -- 8 re
// then 8 im bytes, 16 bytes -- at byte offset (((k / 4) * ntb + kb) * n_in + i) * 64 + (k % 4) * 16,
// so that four consecutive channels' pieces make whole 64-byte runs.
__host__ __device__ constexpr int64_t i8q_piece(int k, int64_t kb, int i, int64_t ntb, int n_in) {
    return f32q_piece(k, kb, i, ntb, n_in);
}

struct FeParams {
    const int8_t* x;       // input rows, row i at x + i*ld
    int64_t ld;            // row stride in bytes (multiple of 16)
    int64_t n_avail;       // readable samples per row
    int n_ant, n_pol, n_in, n_fft, n_chan, n_int;
    const int* D;          // [n_ant] integer delays
    const float2* pf;      // [n_ant][n_chan] fractional-delay phasor exp(+2 pi i k tau_f / N)
    const float2* ff;      // [n_ant][n_int] fringe phasor exp(-i phi_a(g0 + t))
    const float2* wcoh;    // [n_ant][n_chan] coherent-beam weight g_a exp(i theta_ak), 0 if unselected
    const float* ginc;     // [n_ant] incoherent weight g_a^2, 0 if unselected
    const float* scale;    // [n_in][n_chan] requantisation scales (I8 / F16)
    void* spec;            // spectra in the K-block layout
    float* beams;          // [2][n_int][n_chan] raw-resolution beams (0 inc, 1 coh)
    const float2* tw;      // FFT twiddles laid out as fengine_tw_angle() describes
    unsigned* err;
};

// Sub-arrays of one batch (corr_batch_*).
constexpr int kMaxSub = 8;

// Twiddle table of the F-engines for n_fft (M = n_fft / 2); entry e holds exp(-2 pi i num / den)
// (fengine_tw_angle), evaluated in FP64 on the device and rounded once (launch_fengine_twiddles).
//   part A, read by the kernel of fengine_impl.cuh (n_fft = 4096): [R2][16]
//     pass-2 twiddles W_{16 R2}^(j r), [R3][16 R2] pass-3 twiddles W_M^(j r) when R3 > 1, then
//     [M/2 + 1] real-split twiddles W_N^k;
//   part B (M <= 1024), read by the warp-FFT kernel of fengine_wfft.cuh: [P/2][32][2] inter-pass
//     twiddles W_M^(l k1) (k1 = 2 j + b at [j][l][b]; P = M/32; at P = 1 its 32 entries are
//     unused), then [M/2 + 1] W_N^k.
__host__ __device__ constexpr int fengine_tw_r2(int M) { return (M / 16 >= 16) ? 16 : M / 16; }
__host__ __device__ constexpr int fengine_tw_r3(int M) { return M / (16 * fengine_tw_r2(M)); }
__host__ __device__ constexpr int fengine_tw_a_count(int n_fft) {
    return fengine_tw_r2(n_fft / 2) * 16 +
           (fengine_tw_r3(n_fft / 2) > 1 ? fengine_tw_r3(n_fft / 2) * 16 * fengine_tw_r2(n_fft / 2) : 0) + n_fft / 4 + 1;
}
__host__ __device__ constexpr int fengine_tw_wfft_offset(int n_fft) { return fengine_tw_a_count(n_fft); }
__host__ __device__ constexpr int fengine_tw_count(int n_fft) {
    return fengine_tw_a_count(n_fft) + (n_fft / 2 <= 1024 ? (n_fft / 64) * 32 + n_fft / 4 + 1 : 0);
}
__host__ __device__ inline void fengine_tw_angle(int n_fft, int e, double& num, double& den) {
    const int M = n_fft / 2, R2 = fengine_tw_r2(M), R3 = fengine_tw_r3(M), Ns3 = 16 * R2;
    const int A = fengine_tw_a_count(n_fft);
    if (e < A) {
        if (e < R2 * 16) {                                   // pass 2: W_{16 R2}^(j r), [r][j]
            num = static_cast<double>(e % 16) * (e / 16);
            den = 16.0 * R2;
            return;
        }
        e -= R2 * 16;
        if (R3 > 1 && e < R3 * Ns3) {                        // pass 3: W_M^(j r), [r][j]
            num = static_cast<double>(e % Ns3) * (e / Ns3);
            den = M;
            return;
        }
        e -= (R3 > 1 ? R3 * Ns3 : 0);                        // real split: W_N^k
        num = e;
        den = n_fft;
        return;
    }
    e -= A;
    if (e < (M / 32) * 32) {                                 // inter-pass: W_M^(l k1), [k1 / 2][l][k1 % 2]
        const int l = (e >> 1) & 31, k1 = ((e >> 6) << 1) + (e & 1);
        num = static_cast<double>(l) * k1;
        den = M;
        return;
    }
    num = e - (M / 32) * 32;                                 // real split: W_N^k
    den = n_fft;
}
cudaError_t launch_fengine_twiddles(int n_fft, float2* tw, cudaStream_t s);

// int8 pair (x[2n], x[2n+1]) as the complex sample z[n], without the conversion unit: each byte
// b, offset to b + 128 (sign bit flipped), becomes the low byte of the float 2^23 + b + 128
// (exponent byte 0x4B), and one packed subtraction of 2^23 + 128 leaves b exactly
__device__ __forceinline__ float2 pair_u16(uint32_t w) {
    const uint32_t x = w ^ 0x8080u;
    const uint32_t lo = __byte_perm(x, 0x4B000000u, 0x7440), hi = __byte_perm(x, 0x4B000000u, 0x7441);
    return __fadd2_rn(make_float2(__uint_as_float(lo), __uint_as_float(hi)), make_float2(-8388736.0f, -8388736.0f));
}

// The per-antenna delay model (Sec. 2.1, Eq. 2), shared by every table set-up:
// integer delay D = floor(tau + 1/2), fractional-delay (FSTC) phasor exp(+2 pi i k tau_f / N)
// with tau_f = tau - D, fringe phasor exp(-i phi) with phi = phi0 + rate g over the global frame
// count g, reduced mod 2 pi in FP64.
__host__ __device__ inline int model_int_delay(double tau) { return static_cast<int>(floor(tau + 0.5)); }
__device__ inline float2 model_fstc_phasor(double tau, int k, int n_fft) {
    const double tf = tau - floor(tau + 0.5);
    double sn, cs;
    sincospi(2.0 * k * tf / n_fft, &sn, &cs);
    return make_float2(static_cast<float>(cs), static_cast<float>(sn));
}
__device__ inline float2 model_fringe_phasor(double phi0, double rate, int64_t g) {
    const double twopi = 6.283185307179586476925286766559;
    double ph = phi0 + rate * static_cast<double>(g);
    ph -= twopi * rint(ph / twopi);
    double sn, cs;
    sincos(ph, &sn, &cs);
    return make_float2(static_cast<float>(cs), static_cast<float>(-sn));
}

cudaError_t launch_fengine(const FeParams& p, int mode, cudaStream_t s);
// true where launch_fengine launches 2-CTA clusters (n_chan 2048, fp16 layouts and int8 bytes)
bool fengine_clustered(int n_chan, int mode);

// pf, ff and D for one integration from the FP64 delay / fringe model.
// g0_dev, when given, is read on the device instead of g0 (graph-captured launches).
cudaError_t launch_phasor_setup(int n_ant, int n_chan, int n_fft, int n_int, int64_t g0, const double* tau,
                                const double* phi0, const double* rate, float2* pf, float2* ff, int* D,
                                cudaStream_t s, const int64_t* g0_dev = nullptr);

// Auto-power dumps from the FP32 K-block spectra (quad: the channel-quad layout): P[i][d][k] = sum
// of |Y_i[t][k]|^2 over the `dump` frames of dump d (dump a multiple of tb_fp32(n_chan) dividing n_int).
cudaError_t launch_power_dumps(const float* spec, int n_in, int n_chan, int n_int, int dump, float* P,
                               cudaStream_t s, bool quad = false);

// Time-domain voltage blanker (blank.cu, Sec. 5, Eq. 3-4) on rows x[i][0..n) cut into blocks of
// `block` samples (a multiple of 16): per block, stats [n_in][ceil(n / block)][4] = 2 med, 4 MAD,
// T2 = floor(2 M MAD / 0.6745) and the number of samples with |2x - 2 med| > T2, and the blanked
// rows y[i][0..n) (stride ldy): flagged samples replaced by rint(sigma g[i][pos & noise_mask])
// clamped to +-127, sigma = MAD / 0.6745 rounded to FP32; the rest copied.
cudaError_t launch_blank(const int8_t* x, int64_t ld, int n_in, int64_t n, int block, double M,
                         const float* noise, int noise_mask, int32_t* stats, int8_t* y, int64_t ldy,
                         cudaStream_t s);

// Phased beams with full-polar products or voltages (multibeam.cu) from the FP32 spectra:
// w [n_chan][wstride] float2, entry b * n_ant + a the weight of antenna a in beam b for the channel
// (wstride = multibeam_wstride(): n_beams * n_ant rounded up to even); out [n_beams][n_int/avg][n_chan]
// float4.  avg a power of two, max(64, avg) dividing n_int; products 1 (voltages) needs avg = 1.
int multibeam_max_beams();
int multibeam_wstride(int n_beams, int n_ant);
cudaError_t launch_multibeam(const float* spec, int n_ant, int n_pol, int n_chan, int n_int, const float2* w,
                             int n_beams, int products, int avg, float4* out, unsigned* err, cudaStream_t s);

// The same phased beams on the tcgen05 tensor cores (multibeam_tc.cu): FP32 accuracy from an
// on-chip fp16 hi/lo split of weights and spectra; n_ant <= 64, n_beams <= 64, n_int % 64 == 0.
// launch_multibeam takes this form for more than 24 beams where it applies.  split_scale: power of two bringing the
// spectra below the fp16 range (2^-(log2 n_fft - 8)).
bool multibeam_tc_supported(int n_ant, int n_pol, int n_chan, int n_int);
cudaError_t launch_multibeam_tc(const float* spec, int n_ant, int n_pol, int n_chan, int n_int, const float2* w,
                                int wstride, int n_beams, int products, int avg, float split_scale, float4* out,
                                unsigned* err, cudaStream_t s);

// ADC-format 4-bit ingest (ingest4.cu): card rows packed[c][0..2n) (stride ld, even) -> int8 rows
// rows[4c + j][0..n) (stride ldr), the 4 interleaved inputs of each card demultiplexed and sign-extended.
cudaError_t launch_unpack4(const uint8_t* packed, int64_t ld, int n_cards, int64_t n, int8_t* rows, int64_t ldr,
                           int n_sm, cudaStream_t s);

// beams_out[b][to][k] = mean over beam_avg frames of beams_raw[b][to*beam_avg + j][k]
cudaError_t launch_beam_average(const float* raw, float* out, int n_int, int n_chan, int beam_avg,
                                cudaStream_t s);

}  // namespace gbx
