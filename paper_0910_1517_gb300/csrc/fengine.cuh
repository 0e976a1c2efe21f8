// fengine.cuh -- launch interface of the F-engine (integer delay, real FFT,
// Eq. 2 phasor, beams, requantisation) and of the per-integration phasor set-up.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace gbx {

enum OutMode : int { OUT_FP32 = 0, OUT_I8 = 1, OUT_F16 = 2 };

// Spectra hand-off layout ("K-block layout"), shared by every X-engine:
//   S[k][kb][r][TB]   k channel, kb = t / TB, r = 2*i + c (c = 0 re, 1 im), TB = t % TB
// One (k, kb) block holds every input's rows for TB consecutive frames.
// fp16 (tensor-core X-engine): TB = 8, R = 2 n_in unswizzled rows of 16 bytes -- exactly
// the no-swizzle K-major canonical layout of a tcgen05 operand tile.
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
    const float2* tw;      // FFT twiddles laid out by fengine_twiddles()
    unsigned* err;
};

// Several integrations in one launch (sub-arrays of uneven sizes).
constexpr int kMaxSub = 8;
struct FeBatch {
    int n_sub;
    int first[kMaxSub + 1];    // first CTA of each sub-array; first[n_sub] = total CTAs
    FeParams p[kMaxSub];
    int64_t g0[kMaxSub];       // global frame index of each sub-array's first frame
};
int fengine_blocks(int n_fft, int n_int);
cudaError_t launch_fengine_batched(const FeBatch* dtab, int total_blocks, size_t smem, int mode, cudaStream_t s);

// Dynamic shared memory needed by the F-engine for a given FFT size.
size_t fengine_smem_bytes(int n_fft);
int fengine_frames_per_cta(int n_fft);
// Twiddle tables of the F-engine's FFT plan for n_fft, computed in FP64 and rounded once.
std::vector<float2> fengine_twiddles(int n_fft);
cudaError_t launch_fengine(const FeParams& p, int mode, cudaStream_t s);

// pf, ff and D for one integration from the FP64 delay / fringe model.
// g0_dev, when given, is read on the device instead of g0 (graph-captured launches).
cudaError_t launch_phasor_setup(int n_ant, int n_chan, int n_fft, int n_int, int64_t g0, const double* tau,
                                const double* phi0, const double* rate, float2* pf, float2* ff, int* D,
                                cudaStream_t s, const int64_t* g0_dev = nullptr);

// Auto-power dumps from the FP32 K-block spectra: P[i][d][k] = sum of |Y_i[t][k]|^2 over the
// `dump` frames of dump d (dump a multiple of tb_fp32(n_chan) dividing n_int).
cudaError_t launch_power_dumps(const float* spec, int n_in, int n_chan, int n_int, int dump, float* P,
                               cudaStream_t s);

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
