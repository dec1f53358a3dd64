// lb_f64.cu -- FP64 instantiation of the fused step (parity mode).
// Compiled with --fmad=false: every multiply and add is rounded separately,
// in the order written in lb_device.cuh.
#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbk {

static dim3 tile_grid(int nx, int ny) {
  return dim3((unsigned)((nx + TX - 1) / TX), (unsigned)((ny + TY - 1) / TY));
}

cudaError_t launch_step(const double *fin, double *fout, const StepArgs<double> &A, cudaStream_t st) {
  tile_step_kernel<double, 0, double><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
      fin, fout, nullptr, nullptr, nullptr, A);
  return cudaGetLastError();
}

cudaError_t launch_moments(const double *fin, const StepArgs<double> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st) {
  if (dtype == 0)
    tile_step_kernel<double, 1, double><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
        fin, nullptr, (double *)n, (double *)ux, (double *)uy, A);
  else
    tile_step_kernel<double, 1, float><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
        fin, nullptr, (float *)n, (float *)ux, (float *)uy, A);
  return cudaGetLastError();
}

cudaError_t launch_init(double *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st) {
  init_kernel<double><<<init_grid(nx, ny), 256, 0, st>>>(f, nx, ny, pitch, plane, off, mode, seed, rho_mean, amp, rho0, ux0, uy0, T);
  return cudaGetLastError();
}

}  // namespace lbk
