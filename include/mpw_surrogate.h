/*
 * mpw_surrogate.h -- C ABI of the learned part of libmpw: a 3D convolutional
 * surrogate that advances the global patch of the multipatch scalar-wave
 * method several RK4 steps per call, trained on trajectories of the method
 * itself.  The paper has no learned component; everything in this header is
 * an extension of the method of Sec. 2 (its RK4 step, Table 1, and the
 * 4th-order centred Laplacian of its stencil, Sec. 2.2), defined here.
 *
 * Network (fixed shape): four 3x3x3 convolutions on a periodic box,
 * channels-last, 7 -> 32 -> 32 -> 32 -> 2, ReLU after layers 1-3, no
 * activation after layer 4.  Tensor-core arithmetic: BF16 operands, FP32
 * accumulation, FP32 bias added after the contraction.
 *
 * Conventions shared by every entry point
 *  - Every call returns mpw_status (include/mpw.h); on error
 *    mpw_last_error() holds a message.
 *  - All tensor pointers are CUDA device pointers on the current device,
 *    enqueued on `stream` (NULL = the legacy default stream).  The library
 *    never keeps or frees a caller pointer.
 *  - A volume is [batch][n2][n1][n0][C] (x fastest, channel innermost),
 *    periodic in x, y and z.  n0 must be a multiple of 16 and n1 of 8;
 *    every n >= 3.
 *  - BF16 tensors are passed as uint16_t (IEEE bfloat16 bit patterns).
 *    Channel counts are 8 or 32: the 7 input features and the 2 outputs are
 *    stored in 8-channel tensors whose extra channels are zero.
 *  - Weights of one layer: W[co][tap][ci], tap = (dz*3 + dy)*3 + dx with
 *    offsets dz-1, dy-1, dx-1 in {-1, 0, 1}:
 *        y[p][co] = b[co] + sum_{tap, ci} x[p + off(tap)][ci] * W[co][tap][ci]
 *    (a cross-correlation, indices taken modulo n).
 */
#ifndef MPW_SURROGATE_H
#define MPW_SURROGATE_H

#include <stddef.h>
#include <stdint.h>

#include "mpw.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- layer primitives (device pointers) -------------------------------- */

/* y = act(conv(x, W) + b).  cin, cout in {8, 32} ((8, 8) is rejected).
 * relu = 1 applies max(0, .); mask (optional, [..][cout] BF16) zeroes every
 * output whose mask value is <= 0.  Either output may be NULL: y (BF16, RNE
 * rounding of the FP32 result) and y32 (the FP32 result).  bias may be NULL.
 * MPW_ERR_ARG on an unsupported shape or a NULL input. */
mpw_status mpw_conv3_forward(const uint16_t* x, int cin, const uint16_t* w, const float* bias, int cout,
                             int batch, const int n[3], int relu, const uint16_t* mask, uint16_t* y, float* y32,
                             void* stream);

/* Forward kernel selection (process-wide; no counterpart in the paper).
 * kernel = 0 (default): volumes with n0 = 128 run on the tcgen05 tensor-core
 * kernel (TMEM accumulators, one x-row of 128 points per MMA), every other
 * volume on the mma.sync kernel; kernel = 1: the mma.sync kernel always (the
 * parity reference of the tcgen05 one).  Applies to mpw_conv3_forward,
 * mpw_conv3_backward_data and everything built on them.  Not thread-safe
 * against concurrent launches.  Errors: MPW_ERR_ARG for another value. */
mpw_status mpw_conv3_select(int kernel);

/* Gradient with respect to the input of a layer with weights W[cout][27][cin]:
 *     gx[p][ci] = sum_{tap, co} gy[p - off(tap)][co] * W[co][tap][ci]
 * multiplied by 1[mask[p][ci] > 0] when mask (the layer's input activation,
 * [..][cin] BF16) is given.  gy is [..][cout] BF16; gx is written as BF16
 * (gx) and/or FP32 (gx32). */
mpw_status mpw_conv3_backward_data(const uint16_t* gy, int cout, const uint16_t* w, int cin, int batch,
                                   const int n[3], const uint16_t* mask, uint16_t* gx, float* gx32, void* stream);

/* Gradients with respect to the weights and the bias:
 *     gw[co][tap][ci] = sum_p gy[p][co] * x[p + off(tap)][ci],   gb[co] = sum_p gy[p][co]
 * (FP32, overwritten).  scratch: device workspace of at least
 * mpw_conv3_wgrad_scratch_bytes(cin, cout) bytes. */
size_t mpw_conv3_wgrad_scratch_bytes(int cin, int cout);
mpw_status mpw_conv3_backward_weights(const uint16_t* x, int cin, const uint16_t* gy, int cout, int batch,
                                      const int n[3], float* gw, float* gb, void* scratch, size_t scratch_bytes,
                                      void* stream);

/* One Adam update (Kingma & Ba, Algorithm 1) of `count` FP32 parameters:
 *     m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *     w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * with t >= 1 the 1-based step number; w16 (optional) receives the BF16 (RNE)
 * copy of the updated w. */
mpw_status mpw_adam_step(float* w, uint16_t* w16, const float* g, float* m, float* v, long long count, float lr,
                         float b1, float b2, float eps, int t, void* stream);

/* Mean-squared error of the first `used` channels of y ([points][cy] FP32)
 * against t ([points][used] FP32): loss = sum (y - t)^2 / (points * used).
 * gy ([points][cy] BF16) receives d loss / d y (zero in channels >= used).
 * loss (device double, may be NULL) is overwritten. */
mpw_status mpw_mse_grad(const float* y, int cy, const float* t, int used, long long points, uint16_t* gy,
                        double* loss, void* stream);

/* ---- the surrogate (network, trainer, inference) ----------------------- */

/* What the network learns.  With Delta = 4 dt (one call replaces four RK4
 * steps of the method) and L the method's 4th-order centred Laplacian
 * (Sec. 2.2: 12 h^2 L u = sum over axes of -u[-2] + 16 u[-1] - 30 u + 16 u[1]
 * - u[2], periodic), the state advances as
 *     psi1 = psi0 + D Pi0 + D^2/2 L psi0 + D^3/6 L Pi0 + D^4/24 L^2 psi0 + (sigma / s) N_0
 *     Pi1  = Pi0 + D L psi0 + D^2/2 L Pi0 + D^3/6 L^2 psi0 + D^4/24 L^2 Pi0 + (sigma / (s D)) N_1
 * (D = Delta): the fourth-order Taylor step of d psi/dt = Pi, d Pi/dt = L psi
 * (for this linear system, one RK4 step of size Delta; stable while Delta
 * times the largest frequency stays below 2.8) plus a learned remainder
 * N = net(x) (channels 0, 1 of the last layer).  Every sum is taken left to
 * right, each operation rounded once.  Per sample the scale
 * s = 1 / max_p max(|psi0|, Delta |Pi0|) (binary32: the maximum is rounded to
 * binary32, then s = 1/max rounded to binary32; 1 if the state is 0).  Input
 * features (BF16 of the binary32 rounding of the FP64 value):
 *     x = (s psi0, s Delta Pi0, s Delta^2 L psi0, s Delta^3 L Pi0, 0, 0, 0, 0)
 * Training targets (binary32): the remainder of the method's own four steps
 * over the Taylor step,
 *     t_0 = (s / sigma) (psi1 - psi0 - D Pi0 - D^2/2 L psi0 - D^3/6 L Pi0 - D^4/24 L^2 psi0)
 *     t_1 = (s / sigma) D (Pi1 - Pi0 - D L psi0 - D^2/2 L Pi0 - D^3/6 L^2 psi0 - D^4/24 L^2 Pi0).
 * The loss is the mean squared error of (N_0, N_1) against t. */
typedef struct mpw_sur mpw_sur;

/* Parameters, binary32, in this order for layers l = 1..4 (channel counts
 * padded as above: cin 8,32,32,32; cout 32,32,32,8): W_l[cout][27][cin], then
 * b_l[cout].  The padded entries (W_1 for ci >= 7, W_4 and b_4 for co >= 2)
 * must be zero; their gradients are zero, so training keeps them zero. */
long long mpw_sur_param_count(void);

/* dt: the method's step (Delta = 4 dt); h: the global spacing (isotropic);
 * sigma: the remainder scale.  Work is enqueued on `stream` of `device`.
 * Parameters start at zero (call mpw_sur_set_params).  Errors: MPW_ERR_ARG,
 * MPW_ERR_CUDA. */
mpw_status mpw_sur_create(int device, void* stream, double dt, double h, double sigma, mpw_sur** out);
void mpw_sur_destroy(mpw_sur* s);

/* Host copies of the parameters; set also resets Adam's moments and step. */
mpw_status mpw_sur_set_params(mpw_sur* s, const float* params, long long count);
mpw_status mpw_sur_get_params(mpw_sur* s, float* params, long long count);
/* Host copy of the gradient of the last mpw_sur_train_step (same layout). */
mpw_status mpw_sur_get_grads(mpw_sur* s, float* grads, long long count);

/* Features x ([batch][n2][n1][n0][8] BF16) and scales ([batch] binary32) of
 * dense periodic FP64 fields psi0, Pi0 ([batch][n2][n1][n0], device). */
mpw_status mpw_sur_features(mpw_sur* s, const double* psi0, const double* pi0, int batch, const int n[3],
                            uint16_t* x, float* scale);
/* Targets t ([..][2] binary32) of the pair (psi0, Pi0) -> (psi1, Pi1). */
mpw_status mpw_sur_targets(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1,
                           const double* pi1, int batch, const int n[3], const float* scale, float* t);
/* One training step on a batch: forward, loss, backward, Adam (lr, betas
 * 0.9 and 0.999, eps 1e-8).  loss (host, optional) receives the batch loss
 * before the update; passing it synchronises the stream. */
mpw_status mpw_sur_train_step(mpw_sur* s, const uint16_t* x, const float* t, int batch, const int n[3], float lr,
                              double* loss);
/* Network output y ([..][8] binary32; channels 0, 1 are N) for features x. */
mpw_status mpw_sur_forward(mpw_sur* s, const uint16_t* x, int batch, const int n[3], float* y);
/* One surrogate call: (psi0, Pi0) -> (psi1, Pi1) = the state 4 dt later
 * (outputs may not alias inputs). */
mpw_status mpw_sur_predict(mpw_sur* s, const double* psi0, const double* pi0, int batch, const int n[3],
                           double* psi1, double* pi1);

/* Residual check of a call (psi0, Pi0) -> (psi1, Pi1) against the method's
 * RHS: with the two-point quadrature with end corrections,
 *   R_psi = psi1 - psi0 - Delta/2 (Pi0 + Pi1) + Delta^2/12 (L psi1 - L psi0)
 *   R_Pi  = Pi1 - Pi0 - Delta/2 (L psi0 + L psi1) + Delta^2/12 (L Pi1 - L Pi0)
 * which the exact evolution meets to O(Delta^5).  out ([batch][2] binary32,
 * device) receives max_p max(|R_psi|, Delta |R_Pi|) (rounded up) and
 * max_p max(|psi0|, Delta |Pi0|) per sample; lap (optional, device,
 * 4 * batch * points doubles) receives L psi0, L Pi0, L psi1, L Pi1. */
mpw_status mpw_sur_check(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1, const double* pi1,
                         int batch, const int n[3], double* lap, float* out);

/* Hybrid stepping of a multipatch context: `calls` surrogate calls of four
 * steps of dt each.  Per call, from the state at t_n (its covered global cells
 * refilled from the local patches, Sec. 2.4.2): the surrogate's global state
 * four steps later and its residual r = max(|R_psi|, Delta |R_Pi|) /
 * max(|psi0|, Delta |Pi0|) (mpw_sur_check).  r <= tol: the global patch takes
 * that state, and the local patches take their four RK4 steps of the method,
 * their ghost zones filled from a global patch that holds, at every substage,
 * the stage input the method would have formed there: for the linear system,
 * u, u + dt/2 u', u + dt/2 u' + dt^2/4 u'', u + dt u' + dt^2/2 u'' + dt^3/4 u'''
 * with u and its time derivatives taken from the quintic Hermite interpolant
 * in time of (psi, Pi) between the two global states (values, d/dt and
 * d^2/dt^2 from Pi, L psi and L Pi).
 * Otherwise (or r not finite) the call is discarded and the four steps are
 * the method's own (mpw_step).  Every call starts from the global state with
 * its covered cells refilled from the local patches (Local-to-Global,
 * Sec. 2.4.2), as the method refills them at every substage, so local-patch
 * data flows back into the global patch once per call.  Needs a
 * binary64 context whose global patch is periodic with the surrogate's
 * spacing, translating Cartesian local patches, and the surrogate's dt; the
 * surrogate's stream is synchronised with the context's when they differ.
 * accepted, max_residual (optional): calls taken, largest r.  Errors: those
 * of mpw_step, MPW_ERR_ARG. */
mpw_status mpw_step_surrogate(mpw_ctx* ctx, mpw_sur* s, double dt, int calls, double tol, int* accepted,
                              double* max_residual);

/* The weights that mpw_step_surrogate gives (y0, y0', y0'', y1, y1', y1''),
 * the global state at both ends of a call and its first two time derivatives,
 * to build the input of RK4 stage l (0..3) of step m (0..3) of the call, for
 * a call of length delta = 4 dt (host only; no device work).  w6 receives six
 * doubles.  MPW_ERR_ARG for m or l outside 0..3 or a NULL w6. */
mpw_status mpw_sur_stage_weights(int m, int l, double delta, double* w6);

#ifdef __cplusplus
}
#endif

#endif /* MPW_SURROGATE_H */
