// lb_f32.cu -- FP32 instantiation of the fused tile step, and the ghost-band
// copy of the padded sweep planes (FP32 and 16-bit).
#include <algorithm>

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
  init_kernel<float><<<init_grid(nx, ny), 256, 0, st>>>(f, nx, ny, pitch, plane, off, mode, seed, rho_mean, amp, rho0, ux0, uy0, T);
  return cudaGetLastError();
}

// Copy the periodic images into the ghost band of nplanes padded planes.
// Only band elements are visited (blockIdx.y is the plane): first the
// 4 + 4 ghost columns of rows -4 .. ny+3 (with walls rows 0 .. ny-1 only:
// wall lattices have no ghost rows), then, periodic in y, the 4 + 4 ghost
// rows of the interior columns.  Every source is an interior site.
template <typename E>
__global__ void ghost_fill_kernel(E *f, int nx, int ny, int pitch, long long plane, long long off, int walls) {
  const int y0 = walls ? 0 : -4, rows = walls ? ny : ny + 8;
  const long long ncol = 8ll * rows, total = ncol + (walls ? 0ll : 8ll * nx);
  E *p = f + blockIdx.y * plane + off;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total;
       j += (long long)gridDim.x * blockDim.x) {
    int x, y;
    if (j < ncol) {
      const int c = (int)(j & 7);
      y = y0 + (int)(j >> 3);
      x = c < 4 ? c - 4 : nx + c - 4;
    } else {
      const long long r = (j - ncol) / nx;
      x = (int)(j - ncol - r * nx);
      y = r < 4 ? (int)r - 4 : ny + (int)r - 4;
    }
    const int sx = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    const int sy = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    p[(long long)y * pitch + x] = p[(long long)sy * pitch + sx];
  }
}

cudaError_t launch_ghost_fill(void *f, int elem_bytes, int nplanes, int nx, int ny, int pitch, long long plane,
                              long long off, int walls, cudaStream_t st) {
  if (nplanes < 1 || nplanes > 65535) return cudaErrorInvalidValue;
  const long long band = 8ll * (ny + 8) + (walls ? 0ll : 8ll * nx);
  const dim3 grid((unsigned)std::min<long long>((band + 255) / 256, 1024), nplanes);
  if (elem_bytes == 4)
    ghost_fill_kernel<uint32_t><<<grid, 256, 0, st>>>((uint32_t *)f, nx, ny, pitch, plane, off, walls);
  else if (elem_bytes == 2)
    ghost_fill_kernel<uint16_t><<<grid, 256, 0, st>>>((uint16_t *)f, nx, ny, pitch, plane, off, walls);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lbk
