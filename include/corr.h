/*
 * corr.h -- C ABI of a GB300-native FX correlator and beamformer.
 *
 * The operation is the real-time FX correlator + array beamformer of Roy et
 * al., "A real-time software backend for the GMRT" (arXiv:0910.1517):
 *   F-engine (Sec. 2.1, 2.3.2): per input (antenna a, polarisation p) the real
 *     8-bit stream is read with an integer-sample delay offset, channelised by
 *     an N-point real FFT (N/2 channels, DC kept, Nyquist dropped), and each
 *     channel is multiplied by the post-FFT phasor of Eq. 2:
 *       Y[k] = X[k] * exp(i (2 pi k tau_f / N - phi_a(g))),
 *       phi_a(g) = phi0_a + omega_a * g,  g = global frame index since create.
 *   Beams (Sec. 2.2): incoherent B_inc = sum_{a in inc} g_a^2 sum_p |Y_ap|^2 and
 *     coherent B_coh = sum_p |sum_{a in coh} g_a exp(i theta_ak) Y_ap|^2 at the raw
 *     FFT time resolution (optionally averaged over beam_avg frames).
 *   X-engine (Sec. 2.1): for every channel k, baseline a <= a' (N(N+1)/2 of them,
 *     autocorrelations included) and product pq in RR*, RL*, LR*, LL*:
 *       V[k][b][p*n_pol+q] = sum_t Y_{a,p}[t][k] conj(Y_{a',q}[t][k]) over n_int frames.
 *
 * Indexing: input i = a * n_pol + p (p = 0 is R); baselines b row-major over
 * a <= a': (0,0),(0,1)..(0,n_ant-1),(1,1),...; channels k = 0..n_fft/2-1.
 *
 * Precision modes (corr_set_mode): CORR_FP32 computes everything in FP32 on
 * CUDA cores.  CORR_I8 requantises the FP32 spectra to int8 with per-(input,
 * channel) scales, q = clamp(rint(Y*s), +-127), and accumulates q_i conj(q_j)
 * exactly (integer result, bit-exact), then divides by s_i s_j.  CORR_F16
 * rounds Y*s to FP16 and accumulates in FP32.  Both run the X-engine on the
 * tcgen05 tensor cores.  CORR_FP32TC is the FP32 X-engine of CORR_FP32 moved
 * to the tensor cores without losing FP32 accuracy: each FP32 value v = Y * 2^-e
 * (e = log2(n_fft) - 8, so |v| < 2^15 for any int8 input) is stored as fp16
 * hi = rn(v), lo = rn(v - hi), which holds v to 2^-22 |v|; the Gram is
 * H H^T + H L^T + L H^T with exact fp16 products, accumulated in FP32 over
 * 128-frame chunks that are added in FP32, then multiplied by 2^2e.  No scales
 * are needed.  Beams are always formed from the FP32 spectra.
 *
 * Ownership: the library allocates and owns every device buffer and one CUDA
 * stream per handle; callers own every host buffer and any device buffer they
 * pass in.  All entry points return CORR_OK (0) or a negative CORR_E_* code;
 * corr_last_error() then describes the failure (per calling thread).  A
 * handle is not thread-safe: one thread at a time may use it.
 */
#ifndef GB300_CORR_H
#define GB300_CORR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct corr corr_t;

enum {
    CORR_OK = 0,
    CORR_E_INVAL = -1,     /* bad argument (size, null pointer, alignment) */
    CORR_E_RANGE = -2,     /* delay outside [0, max_delay] or buffer too short */
    CORR_E_AGAIN = -3,     /* non-blocking read: no completed integration yet */
    CORR_E_DATALOSS = -4,  /* sequence gap in pushed samples; integration dropped */
    CORR_E_CUDA = -5,      /* CUDA runtime error */
    CORR_E_NOMEM = -6,     /* device or pinned allocation failed */
    CORR_E_STATE = -7,     /* call not valid in the current state */
    CORR_E_TIMEOUT = -8    /* a kernel's bounded wait ran out; results invalid */
};

enum { CORR_FP32 = 0, CORR_I8 = 1, CORR_F16 = 2, CORR_FP32TC = 3 };  /* X-engine precision */
enum { CORR_POL_FULL = 0, CORR_POL_SELF = 1 };                         /* polarisation products */

/* Create a correlator for n_ant antennas x n_pol (1 or 2) polarisations
 * (n_in = n_ant * n_pol <= 128), an n_fft-point real FFT (power of two,
 * 64..4096) and n_int frames per integration (multiple of 16).  Defaults:
 * CORR_FP32, beam_avg 1, max_delay 2048 samples, zero delays and fringes,
 * unit gains, all antennas in both beams, no scales.  *out receives the handle.
 * CORR_I8 needs n_int <= 66571 so that 2 * 127^2 * n_int fits in int32. */
int corr_create(corr_t** out, int n_ant, int n_pol, int n_fft, int n_int);
int corr_destroy(corr_t* h);

/* Message for the most recent failing call on this thread ("" if none). */
const char* corr_last_error(void);

/* Precision mode, polarisation products and beam time averaging.
 * xmode: CORR_FP32 | CORR_I8 | CORR_F16 | CORR_FP32TC (the last three need
 * n_in <= 128; CORR_FP32TC is not available in batches).
 * polmode (Sec. 2.3.2: self-polar and full-polar correlation): CORR_POL_FULL (0) produces
 * all n_pol^2 products per baseline, RR*, RL*, LR*, LL*; CORR_POL_SELF (1) only the n_pol
 * products RR*, LL* (total intensity; Sec. 2.1 sizes the MAC for these two), so the
 * visibilities become [n_fft/2][n_bl][n_pol] -- half the multiply-adds on the CUDA-core
 * X-engine (CORR_FP32); the tensor-core forms, bound by their operand read, compute the
 * same Gram and write only the pp products.  Neither polmode nor beam_avg may change while
 * an output ring is set (they size it).  beam_avg >= 1 must divide n_int. */
int corr_set_mode(corr_t* h, int xmode, int polmode, int beam_avg);

/* Largest integer delay (samples) the streaming ring supports; only before the
 * first push.  Sec. 2.3.2 keeps an overlap of this many samples between time
 * slices so the delay correction is seamless. */
int corr_set_max_delay(corr_t* h, int max_delay);

/* Per-antenna total delay tau_a in samples (Sec. 2.1; 0 <= tau_a, and
 * floor(tau_a + 1/2) <= max_delay), fringe phase phi0_a (rad) at global frame
 * 0 and fringe rate omega_a (rad/frame), all host arrays of n_ant doubles.
 * The integer part D_a = floor(tau_a + 1/2) offsets the read pointer; tau_f =
 * tau_a - D_a enters the Eq. 2 phasor.  Takes effect at the next integration. */
int corr_set_delays(corr_t* h, const double* delay, const double* phi0, const double* rate);

/* Beam weights (Sec. 2.2, 4.3): gain g_a [n_ant] (NULL = 1), phase
 * calibration theta [n_ant][n_fft/2] radians (NULL = 0), and antenna masks
 * inc_mask, coh_mask [n_ant] (nonzero = in the beam; NULL = all). */
int corr_set_beam_weights(corr_t* h, const float* gain, const float* theta,
                          const uint8_t* inc_mask, const uint8_t* coh_mask);

/* Frames per operand stage of the tensor-core X-engine (a tile-shape choice, normally
 * made by corr_batch_tune): 0 = the largest that fits, else a power of two in
 * [16, 512] with (ks / 8) * 2 n_in * 16 <= 32768 bytes.  CORR_FP32TC stages carry
 * two planes: there the stage used is min(ks, largest two-plane stage, 256). */
int corr_set_xengine_stage(corr_t* h, int ks);

/* Requantisation scales s [n_in][n_fft/2] for CORR_I8 / CORR_F16.  NULL
 * derives them from the last completed integration's autocorrelations as
 * s = 127 / (4 sigma), sigma^2 = V_ii[k] / (2 n_int) -- one component's share of
 * the power -- except at DC, sigma^2 = V_ii[0] / n_int: the DC bin of a real
 * stream is real before the Eq. 2 rotation, so one component can carry it all. */
int corr_set_scales(corr_t* h, const float* scale);

/* Streaming ingest of host samples x [n_in][n] (planar int8, row i holds n
 * samples of input i).  seq is the stream index of the first sample; it must
 * continue the previous push, else the partial integration is dropped, the
 * stream restarts at seq and CORR_E_DATALOSS is returned.  Whenever
 * n_int * n_fft + max_delay samples are buffered an integration is launched
 * asynchronously on the handle's stream.  x is copied before return (on the
 * handle's copy stream, into one of two sample rings), so the copy of the next
 * integration's samples overlaps the correlation of this one; results come from
 * corr_read_* (last launched integration) or from an output ring. */
int corr_push_samples(corr_t* h, const int8_t* x, int64_t n, int64_t seq);

/* Ring of host output slots for the streaming ingest: after each integration a
 * push launches, its visibilities (and, if beams != NULL, its beams) are copied
 * into slot j % n_slots, j = 0, 1, ... counting those integrations, in stream
 * order -- the results of integration j no longer block the push of j + 1.
 * vis: n_slots x [n_fft/2][n_bl][n_pol^2] complex64 (re, im float pairs);
 * beams: n_slots x [2][n_int/beam_avg][n_fft/2] float32; host memory, pinned
 * (cudaHostAlloc) for the copies to run asynchronously.  A slot is rewritten
 * n_slots integrations later; the caller reads it before then.  While a ring
 * is set the device outputs are double-buffered (integration j writes buffer
 * j % 2, copied back on a separate stream while j + 1 runs) and beam_avg is
 * fixed.  vis = NULL removes the ring.  Waits for queued work first.
 * CORR_E_INVAL for n_slots outside [1, 4096]; CORR_E_STATE for a batch member. */
int corr_set_output_ring(corr_t* h, float* vis, float* beams, int n_slots);

/* Block until the results of streaming integration `index` are in their slot;
 * *slot (may be NULL) receives the slot number.  CORR_E_AGAIN: not launched
 * yet (push more samples); CORR_E_STATE: no ring, or the slot was reused since;
 * CORR_E_TIMEOUT: a kernel's bounded wait ran out, results invalid. */
int corr_wait_output(corr_t* h, int64_t index, int* slot);

/* As corr_push_samples with x in device memory (row stride n); the copies are
 * ordered after work already on `stream` (a cudaStream_t; NULL and
 * cudaStreamLegacy both name the legacy default stream here). */
int corr_push_samples_device(corr_t* h, const int8_t* x, int64_t n, int64_t seq, void* stream);

/* One whole integration straight from device memory, no copy of the input:
 * row i of input starts at x + i*ld (x and ld 16-byte aligned), holds n_avail
 * readable samples, and n_avail >= n_int*n_fft + max_a D_a.  Frames are global
 * frames g0 .. g0+n_int-1 (fringe phase index).  Runs on `stream`, a
 * cudaStream_t: NULL selects the handle's own stream, cudaStreamLegacy the
 * legacy default stream.  Returns once the work is queued. */
int corr_integrate_device(corr_t* h, const int8_t* x, int64_t ld, int64_t n_avail,
                          int64_t g0, void* stream);

/* Results of the last completed integration, copied to host memory.
 * Visibilities: out [n_fft/2][n_bl][n_pol^2] complex64 as (re, im) float pairs.
 * Beams: out [2][n_int/beam_avg][n_fft/2] float32 (0 = incoherent, 1 = coherent).
 * blocking = 1 waits for an integration in flight; 0 returns CORR_E_AGAIN if
 * none has completed since create. */
int corr_read_visibilities(corr_t* h, float* out, int blocking);
int corr_read_beams(corr_t* h, float* out, int blocking);

/* Exact integer visibilities of the last CORR_I8 integration,
 * out [n_fft/2][n_bl][n_pol^2][2] int32 (re, im) = sum_t q_i conj(q_j). */
int corr_read_vis_int(corr_t* h, int32_t* out, int blocking);

/* Requantised spectra of the last CORR_I8 integration for channels k0..k0+nk-1,
 * q [n_in][n_int][nk][2] int8, and the scales used, scale [n_in][n_fft/2]
 * (either may be NULL). */
int corr_read_requant(corr_t* h, int k0, int nk, int8_t* q, float* scale);

/* FP32 spectra Y of the last CORR_FP32 integration for channels k0..k0+nk-1,
 * out [n_in][n_int][nk] complex64 (re, im pairs).  After a CORR_FP32TC
 * integration: (hi + lo) * 2^e, the values its X-engine multiplied. */
int corr_read_spectra(corr_t* h, int k0, int nk, float* out);

/* Device pointers of the result buffers of handle h (valid until destroy):
 * visibilities (float2), beams (float), and the stream results are written on. */
int corr_device_outputs(corr_t* h, void** vis, void** beams, void** stream);

/* Sizes: n_in, n_bl, n_chan, n_prod, beam frames per integration, and the
 * number of completed integrations. */
int corr_info(corr_t* h, int64_t* out6);

/* Auto-power dumps for the RFI stage (include/rfi.h): with dump > 0 every CORR_FP32
 * integration also produces P [n_in][n_int/dump][n_fft/2] float32,
 * P[i][d][k] = sum over the dump's frames of |Y_i[t][k]|^2 (the paper studies
 * RFI on such 1 ms total-intensity samples, Sec. 5).  dump: 0 (off) or a
 * multiple of 8 (of 4 when n_fft = 4096) dividing n_int.  corr_read_power copies the last integration's
 * dumps to host memory `out` (may be NULL) and/or returns their device address. */
int corr_set_power_dump(corr_t* h, int dump);
int corr_read_power(corr_t* h, float* out, void** device_ptr);

/* ADC-format ingest of the 33 MHz, 4-bit mode (Sec. 2.3.1, 2.3.2): each ADC card interleaves 4
 * inputs sample by sample, 4 bits (two's complement) each -- byte 2s of card c holds inputs 4c
 * (bits 0-3) and 4c+1 (bits 4-7) of sample s, byte 2s+1 inputs 4c+2 and 4c+3; card c carries
 * inputs 4c .. 4c+3 (n_in a multiple of 4).  The library demultiplexes and sign-extends to the
 * int8 rows the F-engine reads.  corr_push_samples_4bit: host packed [n_in/4][ld] (ld even,
 * >= 2 n), streaming as corr_push_samples (half the host-to-device bytes).
 * corr_integrate_4bit_device: one integration from device packed rows (2-byte aligned, ld even,
 * >= 2 n_avail), as corr_integrate_device. */
int corr_push_samples_4bit(corr_t* h, const uint8_t* packed, int64_t ld, int64_t n, int64_t seq);
int corr_integrate_4bit_device(corr_t* h, const uint8_t* packed, int64_t ld, int64_t n_avail, int64_t g0,
                               void* stream);

/* Multiple phased-array beams (Sec. 2.2: the coherent beamformer's voltage cross products
 * for the Stokes parameters; Sec. 5: several phased beams covering different directions),
 * formed after every later CORR_FP32 / CORR_FP32TC integration from its FP32 spectra:
 * U_bp[t][k] = sum_a w[b][a][k] Y_{a,p}[t][k], weights [n_beams][n_ant][n_fft/2] complex
 * (re, im pairs, host, copied).  CORR_BEAM_FULLPOL: per beam, window of avg frames and channel,
 * the window means of |U_b0|^2, |U_b1|^2, Re U_b0 conj U_b1, Im U_b0 conj U_b1 (polarisation-1
 * entries 0 when n_pol = 1); CORR_BEAM_VOLTAGE (avg = 1): Re U_b0, Im U_b0, Re U_b1, Im U_b1.
 * n_beams in [0, 64] (0: off); avg a power of two with max(64, avg) dividing n_int.  The
 * integration fails with CORR_E_STATE in the int8 / FP16 modes (no FP32 spectra). */
enum { CORR_BEAM_FULLPOL = 0, CORR_BEAM_VOLTAGE = 1 };
int corr_set_multibeam(corr_t* h, int n_beams, const float* weights, int products, int avg);
/* The last integration's beams, out [n_beams][n_int/avg][n_fft/2][4] float32; blocking as in
 * corr_read_visibilities. */
int corr_read_multibeam(corr_t* h, float* out, int blocking);

/* Time-domain voltage blanker (Sec. 5, Eq. 3-4) on the raw samples of every later
 * integration, before the FFT: each input row is cut into blocks of `block` samples (a
 * power of two in [4096, 32768], counted from the integration's first sample); in each
 * block the median med and MAD = median |x - med| are found, and samples with
 * |x - med| > M MAD / 0.6745 are replaced by rint(sigma g[i][pos mod L]) clamped to +-127,
 * sigma = MAD / 0.6745 rounded to FP32, g the caller's table `noise` [n_in][L] of
 * standard-normal values (L a power of two <= 2^24; pos = sample position in the row), so
 * the noise is independent between inputs.  M = 0 turns the blanker off (block, noise
 * ignored); the paper uses M = 2.5-3.  The blanked copy of the samples lives in a device
 * buffer of the handle (n_in x (n_int n_fft + max_delay) bytes).  Not available to batch members. */
int corr_set_blanker(corr_t* h, double M, int block, const float* noise, int L);
/* The blanker's statistics of the last integration: out [n_in][*n_blocks][4] int32 =
 * 2 med, 4 MAD, T2 = floor(2 M MAD / 0.6745) (a sample is replaced iff |2x - 2 med| > T2)
 * and the number of samples replaced; *n_samples = samples of each row covered.  Any
 * pointer may be NULL.  CORR_E_STATE when the blanker is off or has not run yet. */
int corr_read_blank_stats(corr_t* h, int32_t* out, int64_t* n_blocks, int64_t* n_samples);

/* Per-stage CUDA-event timing, for measurement.  While enabled (enable = 1),
 * every integration records events around its kernels on the stream it runs
 * on.  corr_stage_times waits for them and sums, over the integrations
 * recorded since its previous call (at most 4096), the milliseconds spent in
 * ms4[0] phasor set-up, ms4[1] F-engine, ms4[2] X-engine, ms4[3] beam
 * averaging; *n receives the number of integrations summed. */
int corr_set_timing(corr_t* h, int enable);
int corr_stage_times(corr_t* h, float* ms4, int* n);

/* ---- Several sub-arrays in one launch ----------------------------------------
 * A batch runs one integration of each of up to 8 handles (sub-arrays of uneven
 * antenna counts and FFT sizes, all in the same precision mode) as a single CUDA
 * graph launch: one branch per sub-array -- its phasor set-up, the F-engine
 * kernel a single handle of that size runs, and its X-engine (the persistent
 * tensor-core kernel over its (channel, row block) items, or the CUDA-core
 * kernel in CORR_FP32) -- with the branches running concurrently, so that one
 * sub-array's X-engine overlaps another's F-engine.  The paper runs its
 * functional pipeline over several time slices concurrently (Sec. 2.3.2); here
 * the concurrency is across independent observations.  Results are read per
 * handle with the functions above.  The handles stay owned by the caller and
 * must outlive the batch; a handle with an output ring (corr_set_output_ring)
 * cannot join one (CORR_E_STATE), nor can a batch member get a ring.
 * corr_batch_integrate_device takes per-sub-array
 * device sample pointers, row strides, readable samples and first global
 * frames (arrays of n_sub); the graph is captured on the first call, later
 * calls set the new pointers in its F-engine nodes (a sub-array whose F-engine
 * runs in 2-CTA clusters -- 4096-point FFTs in CORR_I8 / CORR_F16 -- captures
 * the graph again when its pointers change).
 * corr_batch_tune times every allowed X-engine stage size per sub-array on the
 * spectra of the last batch integration and keeps the fastest in the handle
 * (ks_out, ms_out per sub-array, either may be NULL); later batch integrations
 * use it (the X-engine tables are refreshed on every call). */
typedef struct corr_batch corr_batch_t;
int corr_batch_create(corr_batch_t** out, int n_sub, corr_t* const* subs);
int corr_batch_destroy(corr_batch_t* b);
int corr_batch_integrate_device(corr_batch_t* b, const int8_t* const* x, const int64_t* ld,
                                const int64_t* n_avail, const int64_t* g0, void* stream);
int corr_batch_tune(corr_batch_t* b, int* ks_out, float* ms_out);

/* One FP32 integration that allocates nothing (the paper has no counterpart:
 * this serves callers that may not allocate device memory while they run --
 * a real-time acquisition thread that cannot afford cudaMalloc's device
 * synchronisation and driver locks, or a process whose device memory budget
 * is entirely reserved by its host framework).  It runs the same F-engine and
 * FP32 X-engine as corr_integrate_device with unit beam weights over all
 * antennas; every intermediate buffer lives in one static device array of
 * 32 MiB that each GPU loading this library holds until the process exits.
 *   x, ld, n_avail, g0   as for corr_integrate_device (device samples)
 *   delay, phi0, rate    host arrays of n_ant doubles (phi0, rate may be NULL = 0),
 *                        passed to the kernels by value
 *   vis                  device out [n_fft/2][n_bl][n_pol^2] complex64
 *   beams                device out [2][n_int][n_fft/2] float32 (raw resolution)
 *   stream               cudaStream_t to run on (NULL = legacy default stream)
 *   blocking             1: wait for completion, then report kernel wait timeouts
 *                        (CORR_E_TIMEOUT); 0: return once queued.  Timeouts are
 *                        recorded in a sticky error word in the static array that
 *                        only a blocking call reads and clears, so a caller that
 *                        queues with blocking = 0 learns of a timeout in any of
 *                        those calls from its next blocking call.
 * Errors before any CUDA call: CORR_E_INVAL for n_ant outside 1..64, n_pol not 1 or
 * 2, bad n_fft / n_int, null or misaligned buffers, or a non-finite phi0 / rate;
 * CORR_E_RANGE for a delay that is negative, not finite or rounds to more than
 * 2e9 samples, for n_avail < n_int n_fft + max integer delay, and for problems
 * whose tables plus FP32 spectra exceed the 32 MiB (e.g. 4 ant x 2 pol x 512-pt
 * FFT x 64 spectra uses ~1.1 MiB).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array, so calls whose work overlaps on the GPU race with each other:
 * serialise them (one stream, or wait for the previous call). */
int corr_integrate_static(int n_ant, int n_pol, int n_fft, int n_int, const int8_t* x, int64_t ld,
                          int64_t n_avail, int64_t g0, const double* delay, const double* phi0,
                          const double* rate, float* vis, float* beams, void* stream, int blocking);

/* Coherent dedispersion of the phased-array voltage beam (Sec. 5: the coherent array's
 * pre-detected voltages per polarisation are inverse-FFT'd back to a broadband time series,
 * deconvolved from the ISM dispersion by multiplying with the inverse transfer function in the
 * Fourier domain, detected, the two polarisations added, and integrated in time).
 * Input: voltage spectra of one beam, [n_frames][n_chan] of (X re, X im, Y re, Y im) float32 --
 * the layout corr_read_multibeam gives per beam in CORR_BEAM_VOLTAGE mode; channel k of every
 * frame lies at sky frequency f_lo + k bw / n_chan MHz (an upper-sideband band, bw > 0).
 * Method (all on the GPU):
 *   z[t n_chan + m] = inverse FFT over k of frame t (complex baseband at bw MHz);
 *   blocks of M = fft_frames * n_chan samples stepping by S = (fft_frames - overlap) * n_chan
 *   (overlap-save): y = IFFT(FFT(z_block) * C), C[j] = exp(-i Phi(nu_j)),
 *   nu_j = f_lo + j bw / M, Phi(nu) = 2 pi 1e6 D DM (nu - nu_ref)^2 / (nu_ref^2 nu),
 *   nu_ref = f_lo + bw, D = 4.148808e3 s MHz^2 pc^-1 cm^3; the first S samples of each block
 *   are kept (output time = arrival time at the top of the band);
 *   out[i] = mean over samples [i avg, (i + 1) avg) of |y_X|^2 + |y_Y|^2.
 * corr_dd_create: n_chan and fft_frames powers of two in [64, 4096] and [256, 4096],
 *   fft_frames * n_chan <= 2^24; 0 <= overlap < fft_frames with overlap * n_chan at least the
 *   smear (corr_dd_smear_samples; else CORR_E_RANGE); avg a power of two in [2, 32 n_chan]
 *   dividing S; max_push_frames bounds one push.  Device memory: a ring of fft_frames +
 *   max_push_frames frames, (max_push_frames / (fft_frames - overlap) + 1) work blocks of
 *   16 M bytes, and the 8 M-byte chirp table (computed in FP64 on the host at creation).
 * corr_dd_push_device: appends n_frames frames (device pointer, 16-byte aligned) on `stream`
 *   (cudaStream_t; NULL = legacy default stream; every push of one dedisperser on one stream)
 *   and writes the outputs of every block they complete to out (device, room for out_cap
 *   floats; CORR_E_INVAL when smaller), in time order, continuing where the previous push
 *   stopped; *n_out gets their count (known at return, no synchronisation).  The first output
 *   is the window starting at the first frame ever pushed (or pushed after corr_dd_reset).
 * corr_dd_set_timing: on = 1 records CUDA events around the ring copy and the four passes of
 *   every push that completes a block (each such push then waits for itself) and clears the sums;
 *   corr_dd_stage_times: summed milliseconds per stage (ms5[5]: ring copy, A frames' DFTs,
 *   B rows + chirp, C inverse + detection, D window means) over *n_timed pushes.
 * corr_dd_reset: forget the frames pushed so far (the next push starts a new series).
 * corr_dd_smear_samples: samples by which the bottom of the band lags the top, -1 on bad input. */
typedef struct corr_dd corr_dd_t;
double corr_dd_smear_samples(double dm, double f_lo, double bw);
int corr_dd_create(corr_dd_t** out, int n_chan, int fft_frames, int overlap_frames, int max_push_frames, double dm,
                   double f_lo, double bw, int avg);
int corr_dd_push_device(corr_dd_t* d, const float* spec, int64_t n_frames, float* out, int64_t out_cap,
                        int64_t* n_out, void* stream);
int corr_dd_set_timing(corr_dd_t* d, int on);
int corr_dd_stage_times(corr_dd_t* d, float* ms5, int* n_timed);
int corr_dd_reset(corr_dd_t* d);
int corr_dd_destroy(corr_dd_t* d);

/* Failure detection, exercised without a GPU fault: one kernel waits on a barrier that nothing
 * completes; every pipeline wait of this library is bounded by the same clock budget (~2 s at the
 * maximum SM clock), after which it records an error bit in a device word and returns.
 * corr_wait_selftest returns CORR_OK when the wait gave up and reported its bit as designed
 * (*cycles_out, if given: the clock cycles it waited), CORR_E_STATE if it did not, CORR_E_CUDA on
 * a CUDA error.  Runs on the current device's legacy default stream and synchronises it. */
int corr_wait_selftest(long long* cycles_out);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif
