/*
 * fx_oracle.c -- FP64 CPU oracle for the FX correlator and beamformer of
 * Roy et al., "A real-time software backend for the GMRT" (arXiv:0910.1517).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of what the GPU path computes.  Only tests/, __graft_entry__.smoke()
 * and the cpu_baseline / reference legs of bench.py may load or call it.  It
 * shares no code, header, table or constant with the CUDA library: everything
 * below is written from the paper's definitions, in double precision, with a
 * direct DFT (no FFT, no blocking, no fusion).
 *
 * Conventions (the paper is silent on some of these; each reading is listed in
 * the design notes):
 *   input index      i = a * n_pol + p      (antenna a, polarisation p; p=0 is R)
 *   frame t reads    y[n] = x_i[t*N + D_a + n], n = 0..N-1        (Sec. 2.1, 2.3.2)
 *   integer delay    D_a = floor(tau_a + 1/2),  tau_f = tau_a - D_a in [-1/2, 1/2)
 *   channels         k = 0..N/2-1 (DC kept, Nyquist dropped)       (Sec. 2.1)
 *   DFT              X[k] = sum_n y[n] exp(-2 pi i k n / N), unnormalised
 *   phasor (Eq. 2)   Y[k] = X[k] * exp(i (2 pi k tau_f / N - phi_a(g))),
 *                    phi_a(g) = phi0_a + omega_a * g, g = global frame index
 *   visibilities     V[k][b=(a<=a')][p*n_pol+q] = sum_t Y_{a,p} conj(Y_{a',q})   (Sec. 2.1)
 *   beams (Sec. 2.2) B_inc = sum_{a in inc} g_a^2 sum_p |Y_{a,p}|^2
 *                    B_coh = sum_p | sum_{a in coh} g_a exp(i theta_{a,k}) Y_{a,p} |^2
 *   MAD (Eq. 3, 4)   flag |x - med| > M * MAD / 0.6745; the voltage blanker replaces
 *                    flagged raw samples by scaled table noise (oracle_mad_blank)
 *
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ERANGE (-2)
#define OR_ENOMEM (-3)

static const double TWO_PI = 6.283185307179586476925286766559;

/* Number of baselines including autocorrelations, N(N+1)/2 (Sec. 2.1). */
int oracle_n_baselines(int n_ant) { return n_ant * (n_ant + 1) / 2; }

/* Row-major index of baseline (a, a2), a <= a2: (0,0),(0,1)..(0,n-1),(1,1).. */
static int bl_index(int n_ant, int a, int a2) {
    return a * n_ant - a * (a - 1) / 2 + (a2 - a);
}

/* Integer part of the delay: round half up, so the residual lies in [-1/2, 1/2). */
static long long int_delay(double tau) { return (long long)floor(tau + 0.5); }

/*
 * Integer-delay correction, real DFT channelisation and the post-FFT phase
 * correction of Eq. 2 (fractional-sample time correction plus fringe stop).
 *
 * x        int8 samples, input i starts at x + i*ld, n_avail samples each
 * delay    [n_ant] total delay in samples (>= 0)
 * phi0     [n_ant] fringe phase at global frame 0, radians
 * rate     [n_ant] fringe rate, radians per frame
 * g0       global frame index of local frame 0
 * chans    channel list (n_chans entries) or NULL for all N/2 channels
 * Y        out [n_in][n_frames][n_chans][2] (re, im)
 * Returns OR_ERANGE if a frame would read outside [0, n_avail).
 */
int oracle_fengine(int n_ant, int n_pol, int n_fft, int n_frames,
                   const int8_t* x, int64_t ld, int64_t n_avail,
                   const double* delay, const double* phi0, const double* rate,
                   int64_t g0, const int* chans, int n_chans, double* Y) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_fft < 4 || (n_fft & 1) || n_frames < 0)
        return OR_EINVAL;
    const int N = n_fft, nch_all = N / 2;
    if (!chans) n_chans = nch_all;
    const int n_in = n_ant * n_pol;
    for (int a = 0; a < n_ant; ++a) {
        long long D = int_delay(delay[a]);
        if (D < 0 || (int64_t)(n_frames) * N + D > n_avail) return OR_ERANGE;
    }
    for (int c = 0; c < n_chans; ++c) {
        int k = chans ? chans[c] : c;
        if (k < 0 || k >= nch_all) return OR_EINVAL;
    }
    /* W[m] = exp(-2 pi i m / N), tabulated once; index (k*n) mod N is exact. */
    double* W = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!W) return OR_ENOMEM;
    for (int m = 0; m < N; ++m) {
        W[2 * m] = cos(TWO_PI * m / N);
        W[2 * m + 1] = -sin(TWO_PI * m / N);
    }
    const long long total = (long long)n_in * n_frames;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long it = 0; it < total; ++it) {
        const int i = (int)(it / n_frames), t = (int)(it % n_frames);
        const int a = i / n_pol;
        const long long D = int_delay(delay[a]);
        const double tf = delay[a] - (double)D;
        const int8_t* y = x + (int64_t)i * ld + (int64_t)t * N + D;
        /* fringe phase in FP64 over the global frame counter, reduced mod 2 pi */
        const double phi = fmod(phi0[a] + rate[a] * (double)(g0 + t), TWO_PI);
        for (int c = 0; c < n_chans; ++c) {
            const int k = chans ? chans[c] : c;
            double re = 0.0, im = 0.0;
            for (int n = 0; n < N; ++n) {
                const int m = (int)(((long long)k * n) % N);
                re += (double)y[n] * W[2 * m];
                im += (double)y[n] * W[2 * m + 1];
            }
            const double ph = TWO_PI * (double)k * tf / (double)N - phi;
            const double cr = cos(ph), ci = sin(ph);
            double* o = Y + (((size_t)i * n_frames + t) * n_chans + c) * 2;
            o[0] = re * cr - im * ci;
            o[1] = re * ci + im * cr;
        }
    }
    free(W);
    return OR_OK;
}

/*
 * MAC stage (Sec. 2.1): all N(N+1)/2 baselines, n_pol^2 products each,
 * accumulated over the n_frames spectra in FP64.
 * Y  [n_in][n_frames][n_chans][2];  V out [n_chans][n_bl][n_pol*n_pol][2]
 */
int oracle_xengine(int n_ant, int n_pol, int n_chans, int n_frames,
                   const double* Y, double* V) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_chans < 0 || n_frames < 0)
        return OR_EINVAL;
    const int n_bl = oracle_n_baselines(n_ant), npp = n_pol * n_pol;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chans; ++c) {
        for (int a = 0; a < n_ant; ++a)
            for (int a2 = a; a2 < n_ant; ++a2)
                for (int p = 0; p < n_pol; ++p)
                    for (int q = 0; q < n_pol; ++q) {
                        const int i = a * n_pol + p, j = a2 * n_pol + q;
                        double sr = 0.0, si = 0.0;
                        for (int t = 0; t < n_frames; ++t) {
                            const double* u = Y + (((size_t)i * n_frames + t) * n_chans + c) * 2;
                            const double* v = Y + (((size_t)j * n_frames + t) * n_chans + c) * 2;
                            /* u * conj(v) */
                            sr += u[0] * v[0] + u[1] * v[1];
                            si += u[1] * v[0] - u[0] * v[1];
                        }
                        double* o = V + (((size_t)c * n_bl + bl_index(n_ant, a, a2)) * npp + p * n_pol + q) * 2;
                        o[0] = sr;
                        o[1] = si;
                    }
    }
    return OR_OK;
}

/*
 * Self-polar (total-intensity) MAC (Sec. 2.1 sizes the MAC for these two products,
 * Sec. 2.3.2 names the self-polar mode): only the same-polarisation products
 *   V[c][b][p] = sum_t Y_{a,p}[t][c] * conj(Y_{a',p}[t][c]),  a <= a',  p = 0 (RR*), 1 (LL*).
 */
int oracle_xengine_self(int n_ant, int n_pol, int n_chans, int n_frames,
                        const double* Y, double* V) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_chans < 0 || n_frames < 0)
        return OR_EINVAL;
    const int n_bl = oracle_n_baselines(n_ant);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chans; ++c) {
        for (int a = 0; a < n_ant; ++a)
            for (int a2 = a; a2 < n_ant; ++a2)
                for (int p = 0; p < n_pol; ++p) {
                    const int i = a * n_pol + p, j = a2 * n_pol + p;
                    double sr = 0.0, si = 0.0;
                    for (int t = 0; t < n_frames; ++t) {
                        const double* u = Y + (((size_t)i * n_frames + t) * n_chans + c) * 2;
                        const double* v = Y + (((size_t)j * n_frames + t) * n_chans + c) * 2;
                        sr += u[0] * v[0] + u[1] * v[1];
                        si += u[1] * v[0] - u[0] * v[1];
                    }
                    double* o = V + (((size_t)c * n_bl + bl_index(n_ant, a, a2)) * n_pol + p) * 2;
                    o[0] = sr;
                    o[1] = si;
                }
    }
    return OR_OK;
}

/* The exact integer self-polar MAC on requantised spectra (as oracle_xint, products pp only). */
int oracle_xint_self(int n_ant, int n_pol, int n_chans, int n_frames, const int8_t* q, int64_t* Vint) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_chans < 0 || n_frames < 0)
        return OR_EINVAL;
    const int n_bl = oracle_n_baselines(n_ant);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chans; ++c)
        for (int a = 0; a < n_ant; ++a)
            for (int a2 = a; a2 < n_ant; ++a2)
                for (int p = 0; p < n_pol; ++p) {
                    const int i = a * n_pol + p, j = a2 * n_pol + p;
                    int64_t sr = 0, si = 0;
                    for (int t = 0; t < n_frames; ++t) {
                        const int8_t* u = q + (((size_t)i * n_frames + t) * n_chans + c) * 2;
                        const int8_t* v = q + (((size_t)j * n_frames + t) * n_chans + c) * 2;
                        sr += (int64_t)u[0] * v[0] + (int64_t)u[1] * v[1];
                        si += (int64_t)u[1] * v[0] - (int64_t)u[0] * v[1];
                    }
                    const size_t o = (((size_t)c * n_bl + bl_index(n_ant, a, a2)) * n_pol + p) * 2;
                    Vint[o] = sr;
                    Vint[o + 1] = si;
                }
    return OR_OK;
}

/*
 * Incoherent and coherent array beams (Sec. 2.2, 4.3), detected and summed
 * over polarisations, averaged over beam_avg consecutive frames.
 * gain   [n_ant] g_a;  theta [n_ant][n_fft/2] phase-calibration radians or NULL (=0)
 * inc_mask, coh_mask [n_ant] antenna selection (nonzero = selected)
 * chans  channel list matching Y's channel axis (NULL = all N/2)
 * B out  [2][n_frames/beam_avg][n_chans]: [0] incoherent, [1] coherent
 */
int oracle_beams(int n_ant, int n_pol, int n_fft, int n_chans, int n_frames,
                 const double* Y, const int* chans,
                 const double* gain, const double* theta,
                 const uint8_t* inc_mask, const uint8_t* coh_mask,
                 int beam_avg, double* B) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || beam_avg < 1 || n_frames % beam_avg)
        return OR_EINVAL;
    const int nch_all = n_fft / 2, n_out = n_frames / beam_avg;
    if (!chans && n_chans != nch_all) return OR_EINVAL;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n_chans; ++c) {
        const int k = chans ? chans[c] : c;
        for (int to = 0; to < n_out; ++to) {
            double binc = 0.0, bcoh = 0.0;
            for (int tt = 0; tt < beam_avg; ++tt) {
                const int t = to * beam_avg + tt;
                for (int p = 0; p < n_pol; ++p) {
                    double sr = 0.0, si = 0.0;
                    for (int a = 0; a < n_ant; ++a) {
                        const int i = a * n_pol + p;
                        const double* y = Y + (((size_t)i * n_frames + t) * n_chans + c) * 2;
                        if (inc_mask[a])
                            binc += gain[a] * gain[a] * (y[0] * y[0] + y[1] * y[1]);
                        if (coh_mask[a]) {
                            const double th = theta ? theta[(size_t)a * nch_all + k] : 0.0;
                            const double wr = gain[a] * cos(th), wi = gain[a] * sin(th);
                            sr += wr * y[0] - wi * y[1];
                            si += wr * y[1] + wi * y[0];
                        }
                    }
                    bcoh += sr * sr + si * si;
                }
            }
            B[(size_t)to * n_chans + c] = binc / beam_avg;
            B[((size_t)n_out + to) * n_chans + c] = bcoh / beam_avg;
        }
    }
    return OR_OK;
}

/*
 * Multiple phased-array beams with full-polar products (Sec. 2.2: the coherent beamformer
 * gives the voltage cross products for the Stokes parameters; Sec. 5: several phased beams
 * covering different directions).  Beam b's voltage in polarisation p is
 *   U_bp[t][k] = sum_a w[b][a][k] Y_{a,p}[t][k]   (complex weights, FP64 here),
 * and each output point carries four numbers averaged over `avg` frames:
 *   products = 0 (full polar):  |U_b0|^2, |U_b1|^2, Re(U_b0 conj U_b1), Im(U_b0 conj U_b1)
 *   products = 1 (voltages, avg = 1): Re U_b0, Im U_b0, Re U_b1, Im U_b1
 * (the entries of polarisation 1 are 0 when n_pol = 1).
 * Y [n_in][n_frames][n_chans][2]; w [n_beams][n_ant][n_chans][2] (the channels of Y);
 * out [n_beams][n_frames / avg][n_chans][4].
 */
int oracle_multibeam(int n_ant, int n_pol, int n_chans, int n_frames, const double* Y, int n_beams,
                     const double* w, int products, int avg, double* out) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_beams < 1 || avg < 1 || n_frames % avg ||
        (products != 0 && products != 1) || (products == 1 && avg != 1))
        return OR_EINVAL;
    const int n_out = n_frames / avg;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < n_beams; ++b)
        for (int c = 0; c < n_chans; ++c)
            for (int to = 0; to < n_out; ++to) {
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                for (int tt = 0; tt < avg; ++tt) {
                    const int t = to * avg + tt;
                    double ur[2] = {0.0, 0.0}, ui[2] = {0.0, 0.0};
                    for (int p = 0; p < n_pol; ++p)
                        for (int a = 0; a < n_ant; ++a) {
                            const double* y = Y + (((size_t)(a * n_pol + p) * n_frames + t) * n_chans + c) * 2;
                            const double* wa = w + (((size_t)b * n_ant + a) * n_chans + c) * 2;
                            ur[p] += wa[0] * y[0] - wa[1] * y[1];
                            ui[p] += wa[0] * y[1] + wa[1] * y[0];
                        }
                    if (products == 0) {
                        acc[0] += ur[0] * ur[0] + ui[0] * ui[0];
                        acc[1] += ur[1] * ur[1] + ui[1] * ui[1];
                        acc[2] += ur[0] * ur[1] + ui[0] * ui[1];    /* Re(U0 conj U1) */
                        acc[3] += ui[0] * ur[1] - ur[0] * ui[1];    /* Im(U0 conj U1) */
                    } else {
                        acc[0] = ur[0];
                        acc[1] = ui[0];
                        acc[2] = ur[1];
                        acc[3] = ui[1];
                    }
                }
                double* o = out + (((size_t)b * n_out + to) * n_chans + c) * 4;
                for (int q = 0; q < 4; ++q) o[q] = products == 0 ? acc[q] / avg : acc[q];
            }
    return OR_OK;
}

/*
 * Requantisation of spectra to 8-bit integers with per-(input, channel)
 * scales: q = clamp(rint(y * s), -127, 127), round half to even.  This is
 * the FP64 reading of the requantiser; the bit-exact X-engine check uses the
 * GPU's own exported q instead (rounding boundaries of an FP32 product differ).
 * Y [n_in][n_frames][n_chans][2], scale [n_in][n_chans], q out same shape as Y.
 */
int oracle_requant(int n_in, int n_frames, int n_chans, const double* Y,
                   const double* scale, int8_t* q) {
    if (n_in < 1 || n_frames < 0 || n_chans < 0) return OR_EINVAL;
    for (int i = 0; i < n_in; ++i)
        for (int t = 0; t < n_frames; ++t)
            for (int c = 0; c < n_chans; ++c)
                for (int r = 0; r < 2; ++r) {
                    const size_t e = (((size_t)i * n_frames + t) * n_chans + c) * 2 + r;
                    double v = nearbyint(Y[e] * scale[(size_t)i * n_chans + c]);
                    if (v > 127.0) v = 127.0;
                    if (v < -127.0) v = -127.0;
                    q[e] = (int8_t)v;
                }
    return OR_OK;
}

/*
 * Exact integer MAC on requantised spectra (the paper keeps integer products
 * and accumulates them without loss, Sec. 4.1): Vint = sum_t q_i conj(q_j) in
 * int64, then V = Vint / (s_i s_j) in FP64.
 * q [n_in][n_frames][n_chans][2] int8; scale [n_in][n_chans]
 * Vint out [n_chans][n_bl][npp][2] int64 (may be NULL); V out same shape, FP64 (may be NULL)
 */
int oracle_xint(int n_ant, int n_pol, int n_chans, int n_frames,
                const int8_t* q, const double* scale, int64_t* Vint, double* V) {
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || n_chans < 0 || n_frames < 0)
        return OR_EINVAL;
    const int n_bl = oracle_n_baselines(n_ant), npp = n_pol * n_pol;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < n_chans; ++c)
        for (int a = 0; a < n_ant; ++a)
            for (int a2 = a; a2 < n_ant; ++a2)
                for (int p = 0; p < n_pol; ++p)
                    for (int qq = 0; qq < n_pol; ++qq) {
                        const int i = a * n_pol + p, j = a2 * n_pol + qq;
                        int64_t sr = 0, si = 0;
                        for (int t = 0; t < n_frames; ++t) {
                            const int8_t* u = q + (((size_t)i * n_frames + t) * n_chans + c) * 2;
                            const int8_t* v = q + (((size_t)j * n_frames + t) * n_chans + c) * 2;
                            sr += (int64_t)u[0] * v[0] + (int64_t)u[1] * v[1];
                            si += (int64_t)u[1] * v[0] - (int64_t)u[0] * v[1];
                        }
                        const size_t o = (((size_t)c * n_bl + bl_index(n_ant, a, a2)) * npp + p * n_pol + qq) * 2;
                        if (Vint) { Vint[o] = sr; Vint[o + 1] = si; }
                        if (V) {
                            const double d = scale[(size_t)i * n_chans + c] * scale[(size_t)j * n_chans + c];
                            V[o] = (double)sr / d;
                            V[o + 1] = (double)si / d;
                        }
                    }
    return OR_OK;
}

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Median of n values (mean of the two middle values when n is even). */
static double median_of(double* v, int n) {
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    return (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

/*
 * Median-absolute-deviation outlier flag of Eq. 3 and Eq. 4 (Sec. 5):
 * MAD = median |x_i - median(x)|, flag x_i when |x_i - median| > M * MAD / 0.6745.
 * flags out [n] (1 = flagged); med_out, mad_out may be NULL.
 */
int oracle_mad_flag(int n, const double* x, double M, uint8_t* flags,
                    double* med_out, double* mad_out) {
    if (n < 1) return OR_EINVAL;
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    if (!w) return OR_ENOMEM;
    memcpy(w, x, sizeof(double) * (size_t)n);
    const double med = median_of(w, n);
    for (int i = 0; i < n; ++i) w[i] = fabs(x[i] - med);
    const double mad = median_of(w, n);
    const double thr = M * mad / 0.6745;
    for (int i = 0; i < n; ++i) flags[i] = fabs(x[i] - med) > thr ? 1 : 0;
    if (med_out) *med_out = med;
    if (mad_out) *mad_out = mad;
    free(w);
    return OR_OK;
}

/*
 * Time-domain voltage blanker (Sec. 5, Eq. 3-4): each input row is cut into blocks of
 * `block` samples (the last one may be shorter); within a block, samples with
 * |x - med| > M MAD / 0.6745 (oracle_mad_flag on the block) are replaced by pre-computed
 * Gaussian noise, independent per input: the standard-normal table value g[i][pos mod L]
 * (pos = sample position in the row, L a power of two) scaled by the block's robust sigma
 * MAD / 0.6745 rounded to FP32, the product rounded to FP32 and to the nearest integer
 * (ties to even), clamped to +-127.
 * x [n_in] rows of ld bytes, n samples each; out the same shape (contiguous rows of n);
 * stats [n_in][n_blocks][4] int32: 2 med, 4 MAD, floor(2 M MAD / 0.6745) (the largest
 * 2 |x - med| that is kept; clamped to [-1, 1024]) and the number of samples replaced.
 */
int oracle_mad_blank(int n_in, int64_t n, const int8_t* x, int64_t ld, int block, double M,
                     const float* noise, int L, int8_t* out, int32_t* stats) {
    if (n_in < 1 || n < 1 || block < 2 || L < 1 || (L & (L - 1))) return OR_EINVAL;
    const int64_t n_blocks = (n + block - 1) / block;
    int rc = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long q = 0; q < (long long)n_in * n_blocks; ++q) {
        const int i = (int)(q / n_blocks);
        const int64_t b = q % n_blocks, p0 = b * block;
        const int len = (int)(p0 + block <= n ? block : n - p0);
        double* v = (double*)malloc(sizeof(double) * (size_t)len);
        uint8_t* f = (uint8_t*)malloc((size_t)len);
        if (!v || !f) {
            free(v);
            free(f);
#pragma omp atomic write
            rc = OR_ENOMEM;
            continue;
        }
        for (int j = 0; j < len; ++j) v[j] = (double)x[(int64_t)i * ld + p0 + j];
        double med = 0.0, mad = 0.0;
        oracle_mad_flag(len, v, M, f, &med, &mad);
        const float sig = (float)(mad / 0.6745);
        double t2 = floor(2.0 * (M * mad / 0.6745));
        if (t2 > 1024.0) t2 = 1024.0;
        int count = 0;
        for (int j = 0; j < len; ++j) {
            int8_t y = x[(int64_t)i * ld + p0 + j];
            if (f[j]) {
                const float r = rintf(sig * noise[(size_t)i * L + (size_t)((p0 + j) & (L - 1))]);
                y = (int8_t)(r > 127.0f ? 127.0f : (r < -127.0f ? -127.0f : r));
                ++count;
            }
            out[(int64_t)i * n + p0 + j] = y;
        }
        int32_t* st = stats + 4 * q;
        st[0] = (int32_t)(2.0 * med);
        st[1] = (int32_t)(4.0 * mad);
        st[2] = (int32_t)t2;
        st[3] = count;
        free(v);
        free(f);
    }
    return rc;
}

/*
 * ADC-format ingest of the paper's 33 MHz, 4-bit mode (Sec. 2.3.1, 2.3.2): each ADC card
 * digitises 4 analog inputs and its stream interleaves them sample by sample, 4 bits each;
 * the pipeline demultiplexes the 4 streams and unpacks every sample to 8 bits.  Reading: for
 * sample s of card c, byte 2s holds input 4c (bits 0-3) and input 4c+1 (bits 4-7), byte 2s+1
 * inputs 4c+2 and 4c+3; a 4-bit sample is two's complement (-8..7), sign-extended to 8 bits.
 * packed [n_cards] rows of ld bytes (2 n used); out [4 n_cards][n] int8.
 */
int oracle_unpack4(int n_cards, int64_t n, const uint8_t* packed, int64_t ld, int8_t* out) {
    if (n_cards < 1 || n < 0 || ld < 2 * n) return OR_EINVAL;
    for (int c = 0; c < n_cards; ++c)
        for (int64_t s = 0; s < n; ++s)
            for (int j = 0; j < 4; ++j) {
                const uint8_t byte = packed[(int64_t)c * ld + 2 * s + j / 2];
                const int nib = (j % 2) ? (byte >> 4) & 0xF : byte & 0xF;
                out[(int64_t)(4 * c + j) * n + s] = (int8_t)(nib >= 8 ? nib - 16 : nib);
            }
    return OR_OK;
}

/* Threads the OpenMP runtime will use (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
