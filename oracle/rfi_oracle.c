/*
 * rfi_oracle.c -- FP64 CPU oracle for the RFI-flagging stage.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, smoke and bench baselines may call it; the
 * CUDA library never does).  Plain double-precision restatements of:
 *   - auto-power dumps: P[i][d][k] = sum over the dump's frames of |Y_i[t][k]|^2
 *     (the 1 ms total-intensity samples the paper's RFI study works on, Sec. 5);
 *   - the per-patch median / median-absolute-deviation statistics of Eq. 3 and
 *     the M * MAD / 0.6745 outlier threshold of Eq. 4, applied to a power patch;
 *   - the learned flagger: three 3x3 convolutions (1->16->32->16 channels, zero
 *     "same" padding, bias, ReLU) and a 1x1 convolution to one logit per pixel,
 *     with the mean binary cross-entropy loss against an RFI mask and its exact
 *     gradient by reverse-mode differentiation (the network the learned form
 *     stands in for the paper's thresholding with).
 * Parameter vector order: W1[16][1][3][3] b1[16] W2[32][16][3][3] b2[32]
 * W3[16][32][3][3] b3[16] W4[1][16] b4[1]  (9441 values).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NL 3
static const int CIN[NL] = {1, 16, 32};
static const int COUT[NL] = {16, 32, 16};

int oracle_rfi_n_params(void) {
    int n = 0;
    for (int l = 0; l < NL; ++l) n += COUT[l] * CIN[l] * 9 + COUT[l];
    return n + 16 + 1;
}

/* P[i][d][k] = sum_{j<dump} |Y[i][d*dump + j][k]|^2 ; Y [n_in][n_frames][n_chan][2] */
int oracle_power_dumps(int n_in, int n_frames, int n_chan, int dump, const double* Y, double* P) {
    if (dump < 1 || n_frames % dump) return -1;
    const int nd = n_frames / dump;
    for (int i = 0; i < n_in; ++i)
        for (int d = 0; d < nd; ++d)
            for (int k = 0; k < n_chan; ++k) {
                double s = 0.0;
                for (int j = 0; j < dump; ++j) {
                    const double* y = Y + (((size_t)i * n_frames + (size_t)d * dump + j) * n_chan + k) * 2;
                    s += y[0] * y[0] + y[1] * y[1];
                }
                P[((size_t)i * nd + d) * n_chan + k] = s;
            }
    return 0;
}

static int cmp_d(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double median(double* v, int n) {
    qsort(v, (size_t)n, sizeof(double), cmp_d);
    return (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

/* Per patch of n values: median, MAD (Eq. 3), flags |x - med| > M MAD / 0.6745 (Eq. 4),
 * and the network input z = sign(u) log(1 + |u|), u = (x - med) / (MAD / 0.6745). */
int oracle_patch_stats(int B, int n, const double* x, double M, double* med, double* mad,
                       uint8_t* flags, double* z) {
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    if (!w) return -3;
    for (int b = 0; b < B; ++b) {
        const double* xb = x + (size_t)b * n;
        memcpy(w, xb, sizeof(double) * (size_t)n);
        const double m = median(w, n);
        for (int i = 0; i < n; ++i) w[i] = fabs(xb[i] - m);
        const double d = median(w, n);
        const double sig = d / 0.6745;
        if (med) med[b] = m;
        if (mad) mad[b] = d;
        for (int i = 0; i < n; ++i) {
            const double u = sig > 0 ? (xb[i] - m) / sig : 0.0;
            if (flags) flags[(size_t)b * n + i] = fabs(xb[i] - m) > M * sig ? 1 : 0;
            if (z) z[(size_t)b * n + i] = (u >= 0 ? 1.0 : -1.0) * log1p(fabs(u));
        }
    }
    free(w);
    return 0;
}

/* y[o][h][w] = b[o] + sum_c sum_{dh,dw} W[o][c][dh][dw] x[c][h+dh-1][w+dw-1]   (zero outside) */
static void conv3(int ci, int co, int H, int Wd, const double* W, const double* bias, const double* x, double* y) {
    for (int o = 0; o < co; ++o)
        for (int h = 0; h < H; ++h)
            for (int w = 0; w < Wd; ++w) {
                double s = bias[o];
                for (int c = 0; c < ci; ++c)
                    for (int dh = 0; dh < 3; ++dh)
                        for (int dw = 0; dw < 3; ++dw) {
                            const int hh = h + dh - 1, ww = w + dw - 1;
                            if (hh < 0 || hh >= H || ww < 0 || ww >= Wd) continue;
                            s += W[((o * ci + c) * 3 + dh) * 3 + dw] * x[((size_t)c * H + hh) * Wd + ww];
                        }
                y[((size_t)o * H + h) * Wd + w] = s;
            }
}

struct net {
    const double *W[NL], *b[NL], *W4, *b4;
};

static void unpack(const double* p, struct net* n) {
    for (int l = 0; l < NL; ++l) {
        n->W[l] = p;
        p += COUT[l] * CIN[l] * 9;
        n->b[l] = p;
        p += COUT[l];
    }
    n->W4 = p;
    n->b4 = p + 16;
}

/* logits[b][h][w] of the network for inputs x[b][h][w] */
int oracle_rfi_forward(int B, int H, int Wd, const double* params, const double* x, double* logits) {
    struct net n;
    unpack(params, &n);
    const size_t hw = (size_t)H * Wd;
    double* a[NL + 1];
    for (int l = 0; l <= NL; ++l) a[l] = (double*)malloc(sizeof(double) * hw * 32);
    for (int b = 0; b < B; ++b) {
        memcpy(a[0], x + b * hw, sizeof(double) * hw);
        for (int l = 0; l < NL; ++l) {
            conv3(CIN[l], COUT[l], H, Wd, n.W[l], n.b[l], a[l], a[l + 1]);
            for (size_t q = 0; q < (size_t)COUT[l] * hw; ++q) a[l + 1][q] = a[l + 1][q] > 0 ? a[l + 1][q] : 0.0;
        }
        for (size_t q = 0; q < hw; ++q) {
            double s = n.b4[0];
            for (int c = 0; c < 16; ++c) s += n.W4[c] * a[NL][c * hw + q];
            logits[b * hw + q] = s;
        }
    }
    for (int l = 0; l <= NL; ++l) free(a[l]);
    return 0;
}

/* Mean binary cross-entropy of sigmoid(logit) against mask, and d loss / d params. */
int oracle_rfi_loss_grad(int B, int H, int Wd, const double* params, const double* x, const uint8_t* mask,
                         double* loss, double* grad) {
    struct net n;
    unpack(params, &n);
    const int np = oracle_rfi_n_params();
    memset(grad, 0, sizeof(double) * np);
    struct net g;
    unpack(grad, &g);
    const size_t hw = (size_t)H * Wd;
    const double inv = 1.0 / ((double)B * hw);
    double* a[NL + 1];
    double* da[NL + 1];
    for (int l = 0; l <= NL; ++l) {
        a[l] = (double*)malloc(sizeof(double) * hw * 32);
        da[l] = (double*)malloc(sizeof(double) * hw * 32);
    }
    double L = 0.0;
    for (int b = 0; b < B; ++b) {
        memcpy(a[0], x + b * hw, sizeof(double) * hw);
        for (int l = 0; l < NL; ++l) {
            conv3(CIN[l], COUT[l], H, Wd, n.W[l], n.b[l], a[l], a[l + 1]);
            for (size_t q = 0; q < (size_t)COUT[l] * hw; ++q) a[l + 1][q] = a[l + 1][q] > 0 ? a[l + 1][q] : 0.0;
        }
        /* head, loss and its gradient */
        memset(da[NL], 0, sizeof(double) * 16 * hw);
        for (size_t q = 0; q < hw; ++q) {
            double s = n.b4[0];
            for (int c = 0; c < 16; ++c) s += n.W4[c] * a[NL][c * hw + q];
            const double m = mask[b * hw + q] ? 1.0 : 0.0;
            /* -[m log p + (1-m) log(1-p)], p = 1/(1+e^-s), in a stable form */
            L += (s > 0 ? s : 0.0) - s * m + log1p(exp(-fabs(s)));
            const double p = 1.0 / (1.0 + exp(-s));
            const double ds = (p - m) * inv;
            ((double*)g.b4)[0] += ds;
            for (int c = 0; c < 16; ++c) {
                ((double*)g.W4)[c] += ds * a[NL][c * hw + q];
                da[NL][c * hw + q] += ds * n.W4[c];
            }
        }
        /* back through the three conv + ReLU layers */
        for (int l = NL - 1; l >= 0; --l) {
            const int ci = CIN[l], co = COUT[l];
            double* dW = (double*)g.W[l];
            double* db = (double*)g.b[l];
            memset(da[l], 0, sizeof(double) * (size_t)ci * hw);
            for (int o = 0; o < co; ++o)
                for (int h = 0; h < H; ++h)
                    for (int w = 0; w < Wd; ++w) {
                        const size_t q = ((size_t)o * H + h) * Wd + w;
                        const double dz = a[l + 1][q] > 0 ? da[l + 1][q] : 0.0;  /* ReLU */
                        if (dz == 0.0) continue;
                        db[o] += dz;
                        for (int c = 0; c < ci; ++c)
                            for (int dh = 0; dh < 3; ++dh)
                                for (int dw = 0; dw < 3; ++dw) {
                                    const int hh = h + dh - 1, ww = w + dw - 1;
                                    if (hh < 0 || hh >= H || ww < 0 || ww >= Wd) continue;
                                    const size_t xi = ((size_t)c * H + hh) * Wd + ww;
                                    const int wi = ((o * ci + c) * 3 + dh) * 3 + dw;
                                    dW[wi] += dz * a[l][xi];
                                    da[l][xi] += dz * n.W[l][wi];
                                }
                    }
        }
    }
    *loss = L * inv;
    for (int l = 0; l <= NL; ++l) {
        free(a[l]);
        free(da[l]);
    }
    return 0;
}
