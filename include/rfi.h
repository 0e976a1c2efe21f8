/*
 * rfi.h -- C ABI of the RFI-flagging stage of the GB300 FX correlator.
 *
 * Sec. 5 of Roy et al. (arXiv:0910.1517) flags RFI with a median-absolute-
 * deviation threshold (Eq. 3: MAD = median |x - median(x)|; Eq. 4: flag
 * |x - median| > M MAD / 0.6745) and studies the total intensity at 1 ms
 * resolution.  Here the flagged quantity is a patch of auto-power dumps
 * (64 dumps x 64 channels of one input, from corr_set_power_dump), and two
 * flaggers are offered:
 *   - rfi_patches: per patch median/MAD statistics, Eq. 4 flags (the fallback
 *     and the judge), and the normalised network input
 *     z = sign(u) log(1 + |u|),  u = (x - median) / (MAD / 0.6745), as FP16;
 *   - a learned flagger: three 3x3 convolutions (1 -> 16 -> 32 -> 16 channels,
 *     zero "same" padding, bias, ReLU) and a 1x1 convolution to one logit per
 *     pixel; FP16 weights and activations, FP32 accumulation and gradients,
 *     Adam on FP32 master weights; loss = mean binary cross-entropy of
 *     sigmoid(logit) against the RFI mask.
 * Parameter vector (n = rfi_n_params() = 9441 floats), in order:
 *   W1[16][1][3][3] b1[16] W2[32][16][3][3] b2[32] W3[16][32][3][3] b3[16] W4[16] b4[1]
 * Device tensors: patches x as IEEE binary16 bits [B][64][64] (row = dump,
 * column = channel), masks and flags uint8 [B][64][64], probabilities float
 * [B][64][64].  Return codes are those of corr.h (CORR_OK = 0, CORR_E_*);
 * corr_last_error() describes a failure.
 */
#ifndef GB300_RFI_H
#define GB300_RFI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct rfi_net rfi_net_t;

/* Number of network parameters (9441). */
int rfi_n_params(void);

/* A network with buffers for batches of up to max_batch patches; parameters zero. */
int rfi_create(rfi_net_t** out, int max_batch);
/* The same network built with FP32 weights and activations (FP32 accumulation and gradients
 * as in rfi_create, FP16 patches in): the build whose forward pass and gradients are checked
 * against the FP64 oracle to 1e-5, which proves the kernels' arithmetic apart from FP16
 * rounding.  Every other call works on it unchanged. */
int rfi_create_fp32(rfi_net_t** out, int max_batch);
int rfi_destroy(rfi_net_t* net);

/* Host FP32 parameter vector in / out (set also resets the Adam moments). */
int rfi_set_params(rfi_net_t* net, const float* params);
int rfi_get_params(rfi_net_t* net, float* params);

/* Forward + backward on a batch without updating: *loss (host) receives the
 * mean BCE and grad (host, may be NULL) d loss / d params.  Synchronous. */
int rfi_loss_grad(rfi_net_t* net, const uint16_t* x, const uint8_t* mask, int B, float* loss, float* grad,
                  void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on a
 * batch, queued on stream; loss (host, may be NULL) receives the batch loss
 * and makes the call synchronous. */
int rfi_train_step(rfi_net_t* net, const uint16_t* x, const uint8_t* mask, int B, float lr, float* loss,
                   void* stream);

/* Flag probabilities sigmoid(logit) for a batch (device out [B][64][64]). */
int rfi_infer(rfi_net_t* net, const uint16_t* x, int B, float* prob, void* stream);

/* Cut power dumps P [n_in][n_dump][n_chan] (device, float) into 64 x 64 patches
 * b = (i * (n_dump/64) + d/64) * (n_chan/64) + k/64 and, per patch, compute the
 * Eq. 3 statistics, Eq. 4 flags with threshold M (mad_flags, may be NULL), the
 * network input x (may be NULL) and (median, MAD) pairs stats [B][2] (may be NULL). */
int rfi_patches(const float* power, int n_in, int n_dump, int n_chan, float M, uint16_t* x,
                uint8_t* mad_flags, float* stats, void* stream);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif
