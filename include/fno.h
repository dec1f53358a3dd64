/*
 * fno.h -- C ABI of the learned warm start: a small Fourier neural operator
 * that maps the problem parameters (wall speed U_w, potential amplitude A0,
 * wavelength lambda, reduced temperature T_r) to the steady fields of the
 * lattice Boltzmann solver (include/lb.h) -- density and velocity,
 * `outputs` channels -- used as its initial condition.  The paper has no
 * counterpart: its steady states come from running the scheme of Sec. II;
 * the network only shortens that run, and the solver's own run still
 * decides the result.
 *
 * Network (all sizes from fno_config; FP32 parameters and activations,
 * GEMMs in BF16 with FP32 accumulation unless gemm_bf16 = 0):
 *   features  x[b, 5, y, x]:  A0/1e-3 sin(2 pi x/lambda), A0/1e-3 cos(2 pi x/lambda),
 *             U_w/0.05 (2y/(ny-1) - 1), (T_r - 0.94)/0.02, 2y/(ny-1) - 1
 *   lift      v0 = P x + p
 *   layer l   z = W_l v + w_l + IDFT_m(R_l[m] DFT_m(v)),  v' = gelu(z)
 *             (no gelu after the last layer).  DFT_m keeps x-modes
 *             kx = 0..modes_x-1 and y-modes 0..modes_y/2-1, -modes_y/2..-1;
 *             the inverse is the real transform of the kept modes with kx > 0
 *             counted twice and scale 1/(nx ny).
 *   project   out = Q2 gelu(Q1 v_L + q1) + q2  (`outputs` channels);
 *             loss = mean over fields, channels and sites of (out - target)^2
 * gelu(z) = z Phi(z), Phi the standard normal distribution function.
 *
 * Parameter vector (FP32, this order): P [width][5], p [width]; for each
 * layer: W [width][width], w [width], Rr [modes_y][modes_x][width(in)][width(out)],
 * Ri (same shape); Q1 [hidden][width], q1 [hidden], Q2 [outputs][hidden], q2 [outputs].
 *
 * Layouts: params_dev [batch][4] = (U_w, A0, lambda, T_r) as float;
 * fields [batch][outputs][ny][nx] float, x fastest.  All field and parameter
 * pointers of fno_forward / fno_backward are DEVICE pointers; the calls
 * enqueue work on the handle's stream.  Return values are the LB_* codes
 * of lb.h (0 = success).
 */
#ifndef FNO_H
#define FNO_H

#include <stdint.h>

#include "lb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t width, hidden, layers, modes_x, modes_y, outputs;
  int32_t batch_max, nx_max, ny_max; /* workspace bounds                   */
  int32_t gemm_bf16;                 /* 1: BF16 GEMM inputs; 0: FP32       */
  void *stream;                      /* cudaStream_t; NULL = default       */
} fno_config;

typedef struct fno_handle fno_handle;

/* Allocate the network (parameters zeroed), its gradients, Adam moments and
 * the activation workspace for batch_max fields of nx_max x ny_max.
 * Errors: LB_ERR_ARG (sizes: modes_x <= nx_max/2, modes_y even and
 * <= ny_max, modes_x * modes_y <= 512, and the per-mode mixing's shared
 * memory 4 (4 batch_max width + 2 width^2) bytes at most 48 KB),
 * LB_ERR_CUDA, LB_ERR_OOM.                                                  */
int fno_create(const fno_config *cfg, fno_handle **out);

/* Number of FP32 parameters (the vector described above). */
int64_t fno_param_count(const fno_handle *h);

/* Copy parameters / gradients to or from HOST float arrays of
 * fno_param_count entries (synchronises the stream).                     */
int fno_set_params(fno_handle *h, const float *host);
int fno_get_params(fno_handle *h, float *host);
int fno_get_grads(fno_handle *h, float *host);

/* Forward pass over `batch` fields of nx x ny: out[batch][outputs][ny][nx]
 * (device).  Keeps the activations for fno_backward.                       */
int fno_forward(fno_handle *h, int32_t batch, int32_t nx, int32_t ny, const float *params_dev, float *out);

/* Loss of the last forward pass against target[batch][outputs][ny][nx]
 * (device), and its gradient with respect to every parameter, which
 * REPLACES the gradient buffer.  *loss (host, may be NULL) receives the loss
 * (synchronises the stream when non-NULL).                                */
int fno_backward(fno_handle *h, const float *target, double *loss);

/* One Adam step on the parameters with the current gradients
 * (t = 1, 2, ... is the step number for the bias corrections).            */
int fno_adam(fno_handle *h, float lr, float beta1, float beta2, float eps, int32_t t);

/* Initial fields of the solver (lb_init, mode 1) from the network output,
 * on the device.  For each of `batch` fields out[b] ([outputs][ny][nx]
 * FP32, DEVICE, outputs >= 3, the layout of fno_forward): density
 * n = 1 + s0 out[b][0] + c_b with the constant c_b that makes its mean over
 * the nx ny sites rho_mean (the solver conserves mass, so a prediction must
 * carry the mass of the state it replaces), u_x = s1 out[b][1],
 * u_y = s2 out[b][2], written to fields[b][3][ny][nx] (FP64, DEVICE: rho0,
 * ux0, uy0 of lb_init at fields + 3 b nx ny, + nx ny, + 2 nx ny).
 * scales = (s0, s1, s2), a HOST array.  FP64 arithmetic, each operation
 * rounded once; the mean is a fixed-order sum.  Enqueued on the handle's
 * stream.  Errors: LB_ERR_ARG (null pointers, batch outside 1..8192,
 * fewer than 3 outputs), LB_ERR_CUDA.                                      */
int fno_fields(fno_handle *h, const float *out, int32_t batch, int32_t nx, int32_t ny, const double *scales,
               double rho_mean, double *fields);

int fno_destroy(fno_handle *h);
const char *fno_last_error(const fno_handle *h);

/* The network's matrix product on the tensor cores, as a building block
 * (the paper has no counterpart): for b = 0 .. batch-1,
 *   C[b](m, n) = sum_k X[b](m, k) Y[b](n, k) + beta C[b](m, n)
 * with BF16 operands and FP32 accumulation.  X is M x K with row pitch ldx,
 * Y is N x K with row pitch ldy (k contiguous in both), batch strides sX,
 * sY in elements (0: one matrix shared by every batch); pitches and strides
 * multiples of 8 elements, ldx, ldy >= K, bases 16-byte aligned.  C is FP32,
 * element (b, m, n) at C + b sC + m cm + n cn (any strides, so C or its
 * transpose).  X, Y, C and err are DEVICE pointers; err points to an int the
 * kernel sets to 1 when one of its bounded waits gave up (results then
 * meaningless).  Enqueued on `stream` (cudaStream_t, NULL = default) without
 * synchronising.  Errors: LB_ERR_ARG (shapes, pitches, alignment, null
 * pointers), LB_ERR_CUDA.                                                  */
int fno_gemm_bf16(const void *X, int32_t ldx, int64_t sX, const void *Y, int32_t ldy, int64_t sY, float *C,
                  int64_t cm, int64_t cn, int64_t sC, int32_t M, int32_t N, int32_t K, int32_t batch, float beta,
                  int *err, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FNO_H */
