// lb_internal.h -- launchers shared between the translation units of the
// library (FP64 parity build, FP32 build, host API).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace lbk {

// Arguments of the FP32 strip-sweep kernel (lb_sweep.cu).  The state buffers
// use the padded layout: plane q, interior site (x, y) at element
// q * plane + off + y * pitch + x, with 4 ghost columns and 4 ghost rows on
// each side.
struct SweepArgs {
  int nx, ny, walls;
  int pitch;
  long long plane, off;
  int seg_h, nseg, nstrips, base_w, extra;
  float T, a, b, kappa, omega, one_minus_omega, g, th, A0, u_bot, u_top;
  float N, M, Q, R, four_QR;
  float A_rest, A_ax, A_diag;  // rest factors 1 + (T - T0)(c.c - 2 T0) / (2 T0^2)
  float nmax;                  // 1/b (upper bound of a valid density)
  const float *sinx;
  float *fout;
  double *partials;            // 4 doubles per CTA: mass, J_x, J_y, bad-site flag
  int *err;                    // set when a bounded wait gave up
};

cudaError_t sweep_prepare(size_t *smem_bytes);
// Strips (widths base_w or base_w + 4; the first `extra` are wider) and
// row segments of the sweep kernel for an nx x ny lattice.
void sweep_plan(int nx, int ny, int *nstrips, int *base_w, int *extra, int *seg_h, int *nseg);
// TMA descriptor of one padded FP32 state buffer, with the box the sweep
// kernel's ring expects (built next to the kernel so the two cannot differ).
cudaError_t sweep_make_map(void *base, int pitch, int ny, long long plane, CUtensorMap *map);
cudaError_t launch_sweep(const CUtensorMap &tin, const SweepArgs &A, size_t smem, cudaStream_t st);
cudaError_t launch_ghost_fill(float *f, int nx, int ny, int pitch, long long plane, long long off,
                              int walls, cudaStream_t st);

template <typename real_t>
struct StepArgs;

// One fused time step fin -> fout.
cudaError_t launch_step(const double *fin, double *fout, const StepArgs<double> &A, cudaStream_t st);
cudaError_t launch_step(const float *fin, float *fout, const StepArgs<float> &A, cudaStream_t st);

// Moments (n, u*) of the stored state; dtype 0 = double, 1 = float outputs.
cudaError_t launch_moments(const double *fin, const StepArgs<double> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);
cudaError_t launch_moments(const float *fin, const StepArgs<float> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);

// Equilibrium initial state from noise (mode 0) or device fields (mode 1).
cudaError_t launch_init(double *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);
cudaError_t launch_init(float *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);

}  // namespace lbk
