// lb_f32.cu -- FP32 instantiation of the fused tile step.
#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbk {

static dim3 tile_grid(int nx, int ny) {
  return dim3((unsigned)((nx + TX - 1) / TX), (unsigned)((ny + TY - 1) / TY));
}

cudaError_t launch_step(const float *fin, float *fout, const StepArgs<float> &A, cudaStream_t st) {
  tile_step_kernel<float, 0, float><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
      fin, fout, nullptr, nullptr, nullptr, A);
  return cudaGetLastError();
}

cudaError_t launch_moments(const float *fin, const StepArgs<float> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st) {
  if (dtype == 0)
    tile_step_kernel<float, 1, double><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
        fin, nullptr, (double *)n, (double *)ux, (double *)uy, A);
  else
    tile_step_kernel<float, 1, float><<<tile_grid(A.nx, A.ny), TTHREADS, 0, st>>>(
        fin, nullptr, (float *)n, (float *)ux, (float *)uy, A);
  return cudaGetLastError();
}

cudaError_t launch_init(float *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st) {
  const size_t S = (size_t)nx * ny;
  const unsigned blocks = (unsigned)((S + 255) / 256 < 4096 ? (S + 255) / 256 : 4096);
  init_kernel<float><<<blocks, 256, 0, st>>>(f, nx, ny, pitch, plane, off, mode, seed, rho_mean, amp, rho0, ux0, uy0, T);
  return cudaGetLastError();
}

}  // namespace lbk
