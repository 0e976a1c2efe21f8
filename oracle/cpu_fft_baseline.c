/*
 * cpu_fft_baseline.c -- a second CPU timing baseline for the bench, beside the FP64
 * direct-DFT oracle: the same F-engine steps (integer delay, real transform, Eq. 2 phasor;
 * Sec. 2.1) with the DFT replaced by a plain iterative radix-2 FFT in FP32, so that the
 * CPU number is not dominated by the O(N^2) transform.  Its spectra feed the oracle's FP64
 * X-stage unchanged.  TEST / BENCH INFRASTRUCTURE ONLY, like the rest of this directory;
 * tests/test_oracle_pins.py pins it to the oracle's F-engine.
 *
 * Transform: N-point complex FFT of the real frame (imaginary parts zero), decimation in
 * time: bit-reversed load, then log2 N stages of butterflies a' = a + w b, b' = a - w b with
 * w = exp(-2 pi i j / span) from an FP32 table rounded once from FP64.  Channels k < N/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define TWO_PI_D 6.283185307179586476925286766559

static long long fft_int_delay(double tau) { return (long long)floor(tau + 0.5); }

/* Y [n_in][n_frames][N/2][2] (double, the oracle's layout) */
int cpu_fft_fengine(int n_ant, int n_pol, int n_fft, int n_frames, const int8_t* x, int64_t ld, int64_t n_avail,
                    const double* delay, const double* phi0, const double* rate, int64_t g0, double* Y) {
    const int N = n_fft, M = N / 2, n_in = n_ant * n_pol;
    int lg = 0;
    while ((1 << lg) < N) ++lg;
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || N < 4 || (1 << lg) != N || n_frames < 0) return -1;
    for (int a = 0; a < n_ant; ++a) {
        const long long D = fft_int_delay(delay[a]);
        if (D < 0 || (int64_t)n_frames * N + D > n_avail) return -2;
    }
    float* W = (float*)malloc(sizeof(float) * (size_t)N);          /* W[j] = exp(-2 pi i j / N), j < N/2 */
    int* rev = (int*)malloc(sizeof(int) * (size_t)N);
    float* pk = (float*)malloc(sizeof(float) * 2 * (size_t)n_ant * M); /* exp(+2 pi i k tau_f / N) */
    if (!W || !rev || !pk) {
        free(W);
        free(rev);
        free(pk);
        return -3;
    }
    for (int j = 0; j < M; ++j) {
        W[2 * j] = (float)cos(TWO_PI_D * j / N);
        W[2 * j + 1] = (float)-sin(TWO_PI_D * j / N);
    }
    for (int n = 0; n < N; ++n) {
        int r = 0;
        for (int b = 0; b < lg; ++b) r |= ((n >> b) & 1) << (lg - 1 - b);
        rev[n] = r;
    }
    for (int a = 0; a < n_ant; ++a) {
        const double tf = delay[a] - (double)fft_int_delay(delay[a]);
        for (int k = 0; k < M; ++k) {
            const double ph = TWO_PI_D * k * tf / N;
            pk[2 * ((size_t)a * M + k)] = (float)cos(ph);
            pk[2 * ((size_t)a * M + k) + 1] = (float)sin(ph);
        }
    }
    const long long total = (long long)n_in * n_frames;
    int rc = 0;
#pragma omp parallel
    {
        float* buf = (float*)malloc(sizeof(float) * 2 * (size_t)N);
        if (!buf) {
#pragma omp atomic write
            rc = -3;
        }
#pragma omp for schedule(static)
        for (long long it = 0; it < total; ++it) {
            if (!buf) continue;
            const int i = (int)(it / n_frames), t = (int)(it % n_frames), a = i / n_pol;
            const int8_t* y = x + (int64_t)i * ld + (int64_t)t * N + fft_int_delay(delay[a]);
            for (int n = 0; n < N; ++n) {
                buf[2 * rev[n]] = (float)y[n];
                buf[2 * rev[n] + 1] = 0.0f;
            }
            for (int span = 2; span <= N; span <<= 1) {
                const int half = span / 2, step = N / span;
                for (int s = 0; s < N; s += span)
                    for (int j = 0; j < half; ++j) {
                        const float wr = W[2 * j * step], wi = W[2 * j * step + 1];
                        float* p = buf + 2 * (s + j);
                        float* q = buf + 2 * (s + j + half);
                        const float br = wr * q[0] - wi * q[1], bi = wr * q[1] + wi * q[0];
                        q[0] = p[0] - br;
                        q[1] = p[1] - bi;
                        p[0] += br;
                        p[1] += bi;
                    }
            }
            /* Eq. 2: fractional delay x fringe, the fringe phase in FP64 over the global frame count */
            const double phi = fmod(phi0[a] + rate[a] * (double)(g0 + t), TWO_PI_D);
            const float fr = (float)cos(phi), fi = (float)-sin(phi);
            for (int k = 0; k < M; ++k) {
                const float* w = pk + 2 * ((size_t)a * M + k);
                const float cr = w[0] * fr - w[1] * fi, ci = w[0] * fi + w[1] * fr;
                const float xr = buf[2 * k], xi = buf[2 * k + 1];
                double* o = Y + (((size_t)i * n_frames + t) * M + k) * 2;
                o[0] = xr * cr - xi * ci;
                o[1] = xr * ci + xi * cr;
            }
        }
        free(buf);
    }
    free(W);
    free(rev);
    free(pk);
    return rc;
}
