/* Learned initial guess of the Picard iteration (C ABI).
 *
 * Sec. 2.1 solves each implicit step by a nonlinear fixed-point (Picard)
 * iteration whose start the paper leaves open; the plain start is
 * E^{n+1,0} = E^n.  This interface adds two better starts without touching the
 * convergence test (still |E^{k+1} - E^k| / |E^{k+1}| < picard_tol), so charge
 * and energy conservation are exactly those of the plain method:
 *   PIC_GUESS_EXTRAP  quadratic time extrapolation G = 3E^n - 3E^{n-1} + E^{n-2}
 *   PIC_GUESS_CNN     G + s_d * f(x): a stack of 3x3 convolutions f (BF16
 *                     weights and activations, FP32 accumulation, tensor cores)
 *                     applied to 14 input channels x built from the last four
 *                     fields, H^n and the last step's crossed charge, s_d the
 *                     RMS of the last field increment.
 * Both fall back to the plain start until four field levels exist, and the
 * CNN start falls back to the plain one when its output is not finite or when
 * the Picard iteration from it does not converge (the step is then redone
 * from E^n; pic_step_stats.guess reports the start that was used).
 *
 * Grid of the network: the (nr+1) x (nz+1) points that hold E_r (rows < nr),
 * E_z (columns < nz) and H_theta (rows < nr, columns < nz) at their own
 * indices; tensors at this interface are FP32, NCHW, device pointers.
 * Channels of x (all fields divided by the RMS over their valid points):
 *   0-5 field increments E^{n-k} - E^{n-k-1}, k = 0..2 (E_r, E_z) / s_d;
 *   6-7 E^n; 8 H^n; 9-10 crossed charge (E_r, E_z layouts); 11-12 validity
 *   masks of the E_r and E_z points; 13 r / R of the row.
 * Output / target channels: 0 = E_r, 1 = E_z correction, (E^{n+1} - G) / s_d.
 * The training loss is the mean over the batch of
 * sum_valid (y - t)^2 / (number of valid points).
 *
 * Errors: every call returns PIC_OK or a negative PIC_E_* code of pic.h and
 * never aborts.  The network owns no memory: pic_cnn_init carves the
 * caller's device workspace (pic_cnn_workspace_size bytes, 256-byte aligned),
 * which must outlive the handle.  All work runs on the stream given at init.
 */
#ifndef PIC_GUESS_H
#define PIC_GUESS_H

#include <stddef.h>

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_GUESS_PLAIN 0
#define PIC_GUESS_EXTRAP 1
#define PIC_GUESS_CNN 2

#define PIC_CNN_IN 14  /* input channels */
#define PIC_CNN_OUT 2  /* output channels */

typedef struct pic_cnn pic_cnn;

typedef struct {
  int nr, nz;              /* reactor grid; the network works on (nr+1) x (nz+1) */
  int width;               /* hidden channels: 64 (the only width built) */
  int depth;               /* convolution layers, 2..8 (5: 14-64-64-64-64-2) */
  int batch;               /* largest batch of forward / training calls */
  unsigned long long seed; /* He-normal initial weights, zero biases */
} pic_cnn_config;

/* Device bytes the network needs for cfg; 0 on an invalid cfg. */
size_t pic_cnn_workspace_size(const pic_cnn_config *cfg);

/* Creates the network in ws_dev (bytes >= pic_cnn_workspace_size) on the
 * CUDA stream `stream` (cudaStream_t, NULL = default stream).
 * PIC_E_CONFIG on an invalid cfg, PIC_E_WORKSPACE if bytes is too small. */
int pic_cnn_init(const pic_cnn_config *cfg, void *ws_dev, size_t bytes, void *stream,
                 pic_cnn **out);
void pic_cnn_destroy(pic_cnn *cnn);

/* Number of parameters: per layer the weights (out, in, 3, 3) then the biases. */
long long pic_cnn_num_params(const pic_cnn *cnn);
/* Copies the FP32 master parameters to / from host memory (num_params floats). */
int pic_cnn_get_params(pic_cnn *cnn, float *host);
int pic_cnn_set_params(pic_cnn *cnn, const float *host);

/* y[batch][2][nr+1][nz+1] = f(x[batch][14][nr+1][nz+1]); synchronous. */
int pic_cnn_forward(pic_cnn *cnn, const float *x_dev, int batch, float *y_dev);

/* Loss of f(x) against the target t (same shape as y), and its gradient with
 * respect to the parameters (num_params floats, host, nullable); synchronous. */
int pic_cnn_loss_grad(pic_cnn *cnn, const float *x_dev, const float *t_dev, int batch,
                      double *loss_host, float *grad_host);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on the
 * batch; *loss_host (nullable) receives the loss before the step. */
int pic_cnn_train_step(pic_cnn *cnn, const float *x_dev, const float *t_dev, int batch, float lr,
                       double *loss_host);

/* Selects the Picard start of the following steps (PIC_GUESS_*); cnn is
 * required for PIC_GUESS_CNN, must match the grid and outlive its use. */
int pic_set_guess(pic_ctx *ctx, int mode, pic_cnn *cnn);

/* The (input, target) pair of the last completed step, for training:
 * x_dev [14][nr+1][nz+1] (the inputs at the start of that step) and t_dev
 * [2][nr+1][nz+1] ((E^{n+1} - G) / s_d); *valid = 0 until four field levels
 * preceded the step. */
int pic_guess_sample(pic_ctx *ctx, float *x_dev, float *t_dev, int *valid);

#ifdef __cplusplus
}
#endif

#endif /* PIC_GUESS_H */
