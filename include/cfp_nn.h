/*
 * cfp_nn.h -- C ABI of the learned part: a small 3x3x3 convolutional network
 * on a context's grid, trained on residual/error pairs the solver produces
 * and used to supply an initial guess (an extension of the method, not in
 * arXiv 1901.08269).
 *
 * Conventions (beyond those of cfp.h):
 *  - An activation is a device array of N x 16 BF16 values (uint16_t bit
 *    patterns), channels last: channel c of node (i,j,k) at
 *    16*(i + nx*(j + ny*k)) + c.  N, nx, ny, nz are the context's.
 *  - Weights of a layer are 16 x 27 x 16 BF16 values [co][tap][ci], tap t for
 *    the offset (dz, dy, dx) = (t/9 - 1, (t/3)%3 - 1, t%3 - 1); a bias is 16
 *    FP32 values.  A layer computes, with zero padding outside the grid,
 *        out[v][co] = bias[co] + sum_t sum_ci W[co][t][ci] * in[v + off(t)][ci].
 *    Narrower layers keep their unused channels at zero weight.
 *  - The convolutions run on the tensor cores in BF16 with FP32 accumulation.
 *  - Every call is ordered on the context's stream; cfp_nn_mse synchronises.
 *    Errors as in cfp.h (CFP_EINVAL for NULL or inconsistent arguments).
 */
#ifndef CFP_NN_H
#define CFP_NN_H
#include <stdint.h>

#include "cfp.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Network input and training target from FP64 fields.  x (N x 16 BF16):
 * channel 0 = scale * r at the unknowns, channel 1 = 1 at the unknowns, 0
 * elsewhere.  scale <= 0: scale = 1 / max |r| over the unknowns (1 if r is
 * 0 there), computed on the device (the call then synchronises); the scale
 * used goes to *scale_used_host (NULL: not returned).  target (NULL or N
 * FP32) = scale * escale * e at the unknowns (0 where e is NULL or off the
 * unknowns), so the network's output y predicts e = y / (scale * escale);
 * mask (NULL or N FP32) = 1 at the unknowns.  Requires classification
 * (CFP_ESTATE otherwise).
 */
cfp_status cfp_nn_pack(cfp_ctx* ctx, const double* r_dev, const double* e_dev, double scale, double escale,
                       uint16_t* x_dev, float* target_dev, float* mask_dev, double* scale_used_host);

/*
 * One layer: out = conv(in, w) + bias (bias NULL: none), then ReLU if relu.
 * Exactly one of out_bf16 (N x 16 BF16) and out_f32 (N x 16 FP32) is given.
 */
cfp_status cfp_nn_conv3d(cfp_ctx* ctx, const uint16_t* in_dev, const uint16_t* w_dev, const float* bias_dev,
                         int relu, uint16_t* out_bf16_dev, float* out_f32_dev);

/*
 * Input gradient of a layer: din[v][ci] = sum_t sum_co w[co][t][ci] *
 * dout[v - off(t)][co], multiplied by [act[v][ci] > 0] when act (the layer's
 * input activation, post-ReLU) is given, which folds in the previous layer's
 * ReLU.  din must not alias dout.
 */
cfp_status cfp_nn_conv3d_dgrad(cfp_ctx* ctx, const uint16_t* dout_dev, const uint16_t* w_dev,
                               const uint16_t* act_dev, uint16_t* din_dev);

/*
 * Weight and bias gradients, ADDED to dw (16 x 27 x 16 FP32) and db (NULL or
 * 16 FP32): dw[co][t][ci] += sum_v dout[v][co] * in[v + off(t)][ci],
 * db[co] += sum_v dout[v][co].
 */
cfp_status cfp_nn_conv3d_wgrad(cfp_ctx* ctx, const uint16_t* in_dev, const uint16_t* dout_dev, float* dw_dev,
                               float* db_dev);

/*
 * Masked mean squared error of channel 0 of y (N x 16 FP32) against target
 * (N FP32) with mask (N FP32): loss = inv_count * sum mask (y - target)^2,
 * returned in *loss_host; dout (N x 16 BF16) = its gradient (channel 0 =
 * 2 inv_count mask (y - target), other channels 0).  Synchronises.
 */
cfp_status cfp_nn_mse(cfp_ctx* ctx, const float* y_dev, const float* target_dev, const float* mask_dev,
                      double inv_count, uint16_t* dout_dev, double* loss_host);

/*
 * Adam step (Kingma & Ba, beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on n FP32
 * master weights w with gradient grad and moments m, v (all device, n each);
 * step counts from 1.  Writes the BF16 copy w_bf16 (NULL: none) and clears
 * grad for the next accumulation.
 */
cfp_status cfp_nn_adam(cfp_ctx* ctx, int64_t n, float* w_dev, float* grad_dev, float* m_dev, float* v_dev,
                       int step, double lr, uint16_t* w_bf16_dev);

/*
 * u = inv_scale * y[v][0] at the unknowns, 0 elsewhere (y N x 16 FP32, u an
 * FP64 field): the network's output as an initial guess for cfp_solve.
 * Requires classification.
 */
cfp_status cfp_nn_unpack(cfp_ctx* ctx, const float* y_dev, double inv_scale, double* u_dev);

#ifdef __cplusplus
}
#endif
#endif
