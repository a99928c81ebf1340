/*
 * warmstart.h -- C ABI of the learned initial guess for the backward-Euler + PCG solve
 * of rklpcg.h (same library, librklpcg.so).
 *
 * The PCG of Fig. 1 of arXiv:1610.01265 starts from an arbitrary x0 and stops on the
 * residual alone, so a better x0 saves iterations without changing what the solve
 * converges to.  This part of the library supplies x0 = T + scale * y(T, bhat, dt)
 * from a small 3-D convolutional net trained on the solver's own solutions; the paper
 * itself has no such net (its PCG starts from the previous time level).  be_pcg_solve
 * (rklpcg.h) takes the guess through its x0 argument and still iterates to rtol.
 *
 * Net (fixed architecture): 3x3x3 convolutions 5 -> 32 -> 32 -> 32 -> 1 channels with
 * ReLU after the first three, cross-correlation with taps ordered (dphi, dtheta, dr),
 * dr fastest.  A "box" is a block of nr x nth x nph cells laid out like every field of
 * rklpcg.h (r fastest); outside a box the input of every layer is zero in r and theta,
 * and in phi either periodic (a whole grid: periodic_phi = 1) or zero (a detached block:
 * periodic_phi = 0).  nbox boxes of the same shape are stored back to back.
 * Input channels: (T - 1e6 K)/1e6 K, bhat_r, bhat_theta, bhat_phi, log10(dt / 1 s).
 *
 * Parameters: ws_num_params() float32 values, for each layer its weights
 * W[Cout][Cin][3][3][3] then its biases b[Cout].  Forward and backward passes run on the
 * tensor cores with BF16 copies of the weights, BF16 activations and FP32 accumulation;
 * the loss gradient dy and the back-propagated activation gradients are BF16 too, the
 * parameter gradients are summed in FP32 per CTA and in FP64 across CTAs (fixed order,
 * run-to-run deterministic).  The optimiser is Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected), parameters and moments in FP32.
 *
 * Memory: arguments named "device" must be CUDA device pointers; parameter and
 * gradient vectors may be host or device (copied).  Activation buffers are owned by the
 * handle and grow to the largest pass seen.  Every call is asynchronous on the handle's
 * stream except ws_create, ws_set_params, ws_get_params, ws_get_grads, ws_check and
 * ws_loss_grad with loss_out != NULL, which return after the stream has drained.
 * Errors: RKL_OK or a negative RKL_E* code of rklpcg.h; ws_last_error() gives the last
 * CUDA message.  A handle is not thread-safe.
 */
#ifndef WARMSTART_H
#define WARMSTART_H

#include "rklpcg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rkl_ws rkl_ws;

/* Number of float32 parameters of the net (constant). */
int ws_num_params(void);

/* New handle on the current device, parameters He-uniform: weight q of the parameter
 * vector = (2u - 1) sqrt(6 / (27 Cin)), u = SplitMix64(seed, q) >> 11 times 2^-53
 * (counter-based, one SplitMix64 step from state seed + (q + 1) * 0x9E3779B97F4A7C15),
 * biases zero, Adam moments zero.  cuda_stream may be NULL (legacy default stream). */
int ws_create(rkl_ws **ws, unsigned long long seed, void *cuda_stream);
int ws_destroy(rkl_ws *ws);
int ws_set_stream(rkl_ws *ws, void *cuda_stream);
const char *ws_last_error(const rkl_ws *ws);
/* Kernels this handle has launched so far. */
long long ws_kernel_launches(const rkl_ws *ws);

/* Copy n = ws_num_params() parameters in (resets the Adam moments and step count) or
 * out; copy the last computed gradient out, or set it (e.g. after averaging the
 * gradients of several replicas) before ws_adam. */
int ws_set_params(rkl_ws *ws, const float *params, int n);
int ws_get_params(rkl_ws *ws, float *params, int n);
int ws_get_grads(rkl_ws *ws, float *grads, int n);
int ws_set_grads(rkl_ws *ws, const float *grads, int n);

/* y [nbox * cells] (device, FP32) of the net on inputs in (device, FP32, channel-major
 * [5][nbox * cells]).  box = {nr, nth, nph}. */
int ws_forward(rkl_ws *ws, const int box[3], int nbox, int periodic_phi, const float *in,
               float *y);

/* Loss L = sum w (y - t)^2 / sum w over nbox boxes and its gradient with respect to the
 * parameters (kept in the handle for ws_adam / ws_get_grads).  in as ws_forward, target
 * (device, FP32 [nbox * cells]), weight (device, FP32, >= 0, or NULL for all ones).
 * loss_out (host, may be NULL) receives L. */
int ws_loss_grad(rkl_ws *ws, const int box[3], int nbox, int periodic_phi, const float *in,
                 const float *target, const float *weight, double *loss_out);

/* One Adam step with learning rate lr on the current gradient. */
int ws_adam(rkl_ws *ws, double lr);

/* Net inputs of one whole grid from T [N] and bhat [3N] (device, float64) and dt > 0:
 * feat (device, FP32 [5][N]) in the layout ws_forward and ws_loss_grad take. */
int ws_features(rkl_ws *ws, const rkl_grid *grid, const double *T, const double *bhat,
                double dt, float *feat);

/* Initial guess for be_pcg_solve on a whole grid (phi periodic):
 * x0 = T + scale * y(features(T, bhat, dt)); T, bhat, x0 device float64, x0 may not
 * alias T.  grid->r_faces is not used. */
int ws_guess(rkl_ws *ws, const rkl_grid *grid, const double *T, const double *bhat,
             double dt, double scale, double *x0);

/* Drain the handle's stream and report whether every tensor-core convolution since the
 * last check finished: RKL_ECUDA (message in ws_last_error, flag cleared) if one gave up
 * waiting for its MMAs after about two seconds, in which case the outputs of the calls
 * since the last check are not valid.  ws_loss_grad with loss_out != NULL checks too. */
int ws_check(rkl_ws *ws);

/* Training target of one solve: target[i] = (x[i] - base[i]) / unit in FP32 for n cells
 * (x, base device float64, target device float32), e.g. x = the PCG solution and
 * base = the field the step started from, so that the guess is base + unit * y. */
int ws_target(rkl_ws *ws, long long n, const double *x, const double *base, double unit,
              float *target);

#ifdef __cplusplus
}
#endif

#endif /* WARMSTART_H */
