/*
 * cfp_nn.h -- C ABI of the learned part (an extension of the method, not in
 * arXiv 1901.08269): a 3D convolutional U-Net on the solver's grid that maps
 * a residual of Eq. Bu=q to its error, trained on residual / error pairs the
 * solver generates, and a flexible GMRES that uses it as a preconditioner.
 *
 * Network: four levels (16, 32, 64, 128 channels), 3x3x3 convolutions with
 * BF16 weights and activations and FP32 accumulation on the tcgen05 tensor
 * cores, injection down and linear interpolation up, skips by addition; 13
 * convolution layers, cfp_unet_param_count() FP32 parameters (per layer the
 * weights [Cout][27][Cin], then the bias [Cout]).  The encoder runs on all
 * four levels, the decoder up to level 1, and the output (channel 0 of the
 * last layer) is interpolated to the grid: a coarse-grid correction, smooth
 * by construction.  Inputs: the residual
 * scaled by 1 / its maximum over the unknowns, the unknowns' mask, a signed
 * distance to the bodies, the local grid spacing per axis.  Output: the
 * error, times 32 and the same scale.  The network needs 4 m + 1 (>= 9) nodes on
 * every axis of the grid it runs on (levels 0 to 2 then have odd sizes).
 *
 * Conventions (beyond those of cfp.h):
 *  - An activation on a grid of nx x ny x nz nodes is a device array of
 *    (nx + 2)(ny + 2)(nz + 2) x C BF16 values (uint16_t bit patterns): the
 *    grid padded by one node on every side, channels last, channel c of
 *    padded node (i, j, k) at ((k (ny + 2) + j)(nx + 2) + i) C + c.  The
 *    padding nodes hold zeros (every kernel here writes zeros there).
 *    Arrays are 16-byte aligned.
 *  - Weights of a layer: Cout x 27 x Cin BF16 values [co][tap][ci], tap t for
 *    the offset (dz, dy, dx) = (t/9 - 1, (t/3)%3 - 1, t%3 - 1):
 *        out[v][co] = bias[co] + sum_t sum_ci W[co][t][ci] in[v + off(t)][ci].
 *  - Calls are ordered on the context's stream; the ones that return host
 *    values synchronise.  Errors as in cfp.h; CFP_ECUDA also when a bounded
 *    (one second) pipeline wait of a tensor-core kernel timed out.
 */
#ifndef CFP_NN_H
#define CFP_NN_H
#include <stdint.h>

#include "cfp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------ single kernels */
enum { CFP_NN_RELU = 1,     /* max(., 0) after the bias                        */
       CFP_NN_MASK = 2,     /* times [act > 0] (the ReLU of the layer before)  */
       CFP_NN_OUT_F32 = 4,  /* FP32 output (Np x cout floats)                  */
       CFP_NN_ACCUM = 8,    /* add to the values already in out                */
       CFP_NN_DGRAD = 16    /* input gradient: w is the forward layer's weights
                               (cin x 27 x cout as [co_f][tap][ci_f], i.e. this
                               call's cout and cin swapped) and the call
                               computes out[v][c] = sum_t sum_k
                               w[k][t][c] in[v - off(t)][k]                   */ };

/*
 * One 3x3x3 convolution with zero padding on an nx x ny x nz grid:
 * out = epilogue(conv(in, w) + bias), cin -> cout channels, (cin, cout) one
 * of (16,16) (16,32) (32,16) (32,32) (32,64) (64,32) (64,64) (64,128)
 * (128,64) (128,128).  bias (cout FP32) may be NULL; act (Np x cout BF16) is
 * read with CFP_NN_MASK.  Tensor-core implicit GEMM (tcgen05, operands staged
 * by TMA).  Synchronises.  Errors: CFP_EINVAL, CFP_ECUDA.
 */
cfp_status cfp_nn_conv3d(cfp_ctx* ctx, int nx, int ny, int nz, int cin, int cout, const uint16_t* in_dev,
                         const uint16_t* w_dev, const float* bias_dev, const uint16_t* act_dev, int flags,
                         void* out_dev);

/*
 * Weight and bias gradients of a convolution, ADDED to dw (cout x 27 x cin
 * FP32, [co][tap][ci]) and db (NULL or cout FP32):
 *   dw[co][t][ci] += sum_v gout[v][co] in[v + off(t)][ci],
 *   db[co] += sum_v gout[v][co].
 * Tensor cores (tcgen05); partial sums per voxel chunk are added in a fixed
 * order, so the result is the same on every run.  Synchronises.
 */
cfp_status cfp_nn_conv3d_wgrad(cfp_ctx* ctx, int nx, int ny, int nz, int cin, int cout, const uint16_t* in_dev,
                               const uint16_t* gout_dev, float* dw_dev, float* db_dev);

/* Transfers between a fine grid (nx x ny x nz, odd sizes) and its coarse
 * grid ((nx + 1) / 2 x ...), coarse node I on fine node 2I, c channels
 * (a multiple of 8), padded activations:
 *   CFP_NN_INJECT       out (coarse) = a (fine) at the even nodes
 *   CFP_NN_PROLONG_ADD  out (fine) = P a (coarse) + b (fine): per axis fine
 *                       2I takes coarse I, fine 2I + 1 the mean of I, I + 1
 *   CFP_NN_PROLONG_T    out (coarse) = P^T a (fine)
 *   CFP_NN_SKIP_GRAD    out (fine) = (a + R^T b) [act > 0], b coarse, R^T
 *                       putting coarse I on fine 2I                       */
enum { CFP_NN_INJECT = 0, CFP_NN_PROLONG_ADD = 1, CFP_NN_PROLONG_T = 2, CFP_NN_SKIP_GRAD = 3 };
cfp_status cfp_nn_transfer(cfp_ctx* ctx, int kind, int nx, int ny, int nz, int c, const uint16_t* a_dev,
                           const uint16_t* b_dev, const uint16_t* act_dev, uint16_t* out_dev);

/* ------------------------------------------------ the network */
typedef struct cfp_unet cfp_unet;

/* Number of FP32 parameters. */
int64_t cfp_unet_param_count(void);

/*
 * A network with He-initialised weights from `seed` (zero biases), its
 * optimiser state and work space on the device of ctx, whose stream it uses.
 * Activation buffers follow the grids it is given.  The network must be
 * destroyed before ctx.  Errors: CFP_EINVAL, CFP_ENOMEM, CFP_ECUDA.
 */
cfp_status cfp_unet_create(cfp_ctx* ctx, uint64_t seed, cfp_unet** out);
void cfp_unet_destroy(cfp_unet* net);

/* Parameters and accumulated gradients as host copies (either may be NULL),
 * cfp_unet_param_count() floats each; set_params also clears the gradients.
 * Synchronise. */
cfp_status cfp_unet_get_params(cfp_unet* net, float* params_host, float* grads_host);
cfp_status cfp_unet_set_params(cfp_unet* net, const float* params_host);

/*
 * The network on a packed input x (16-channel padded activation on an
 * nx x ny x nz grid): y (NULL or Np x 16 FP32) = its output.  With target
 * (Np FP32), mask (Np FP32) and count (> 0): also the loss, the energy
 * norm of the error d = mask (y[.][0] - target) (d = 0 at the padding):
 *   L = (1 / count) sum over the edges (p, q) of the padded grid (d_p - d_q)^2
 * into *loss_host (NULL allowed) and the gradients of L with respect to every
 * parameter ADDED to the network's gradient accumulators (no optimiser step).
 * Synchronises.
 */
cfp_status cfp_unet_forward_raw(cfp_unet* net, int nx, int ny, int nz, const uint16_t* x_dev,
                                const float* target_dev, const float* mask_dev, int count, float* y_dev,
                                double* loss_host);

/*
 * One training step on a pair of FP64 fields of the classified context g:
 * input from r (residual) with scale s = 1 / max |r| over the unknowns,
 * target 32 s e (e the error), loss as above over the unknowns, backward pass,
 * one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr).
 * loss_host: NULL (no synchronisation) or receives the loss (synchronises).
 */
cfp_status cfp_unet_train_step(cfp_unet* net, cfp_ctx* g, const double* r_dev, const double* e_dev, double lr,
                               double* loss_host);

/*
 * z = the network's error estimate for the residual r (FP64 fields of the
 * classified context g): z = y[.][0] / (32 s) at the unknowns, 0 elsewhere.
 * Enqueues only (no synchronisation; may be captured in a CUDA graph once
 * the grid's buffers exist, i.e. after one call on that grid).
 */
cfp_status cfp_unet_apply(cfp_unet* net, cfp_ctx* g, const double* r_dev, double* z_dev);

/* CFP_ECUDA if a bounded wait of one of the network's kernels timed out
 * since the last check.  Synchronises. */
cfp_status cfp_unet_check(cfp_unet* net);

/*
 * Flexible GMRES(m) (Saad, SIAM J. Sci. Comput. 14, 1993) for Eq. Bu=q,
 * right-preconditioned with a preconditioner that may change from step to
 * step: z_j = M(v_j), x = x0 + Z y.
 *   net == NULL: M = P, the inner preconditioner of opts (opts->precond,
 *     sweeps, mg_*; opts->precision CFP_PREC_MIXED applies it in FP32); P is
 *     linear, so this is plain right-preconditioned GMRES.
 *   net != NULL: each step forms the plain direction z1 = P v and a
 *     two-grid cycle whose coarse correction is the network: r1 = v - B z1,
 *     y = net(r1), alpha = (y, r1) / (y, B y) (the step in the energy norm;
 *     0 unless (y, B y) < 0), z2 = z1 + alpha y, zn = z2 + P(v - B z2); it
 *     keeps zn if ||v - B zn|| < ||v - B z1||, else z1 (the plain
 *     preconditioner as fallback and arbiter at every step).  Not linear in
 *     v, hence the flexible method.  info->refinements counts the steps that
 *     kept the network's direction.
 *   net_guess: with net, the initial iterate is u0 = alpha net(rhs) with the
 *     same step (else u_dev).
 *   m: restart length, 1 .. 64.  tol: stop when the true relative residual
 *   ||rhs - B u||_2 / ||rhs||_2 <= tol (the cycle's estimate ends a cycle
 *   early, the true residual is recomputed at every restart).  maxit:
 *   opts->maxit steps.  Other arguments as cfp_solve; info->iterations counts
 *   GMRES steps, info->restarts the cycles.
 * Vectors, the Hessenberg matrix, the rotations and every scalar stay on the
 * device; each step is one CUDA graph launch (captured at the first step of
 * a solve), after which the host reads one flag.  Synchronises.  Errors: as
 * cfp_solve.
 */
cfp_status cfp_solve_fgmres(cfp_ctx* ctx, cfp_unet* net, const double* f_dev, const double* g_nodes_dev,
                            const double* g_ibi_dev, double* u_dev, double tol, const cfp_opts* opts, int m,
                            int net_guess, cfp_info* info);

#ifdef __cplusplus
}
#endif
#endif
