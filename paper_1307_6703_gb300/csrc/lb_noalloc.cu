// lb_noalloc.cu -- lb_reduce_noalloc: the FP64 mass / momentum / stability
// reduction of lb_reduce for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at the point where they want these
// sums: code running under a host application that owns all device memory
// (a plugin or an embedded solver with a fixed memory budget), code in a
// real-time loop where an allocation could block, or code that runs after the
// device allocator has been locked down.  This variant keeps its scratch (one
// partial sum per lattice row) in a fixed file-scope device array instead of
// a buffer from cudaMalloc, and reads and writes only caller-owned buffers.
//
// The scratch array is shared by every call in the process: calls that
// overlap on the GPU (two streams, or two host threads) race on it and must
// be serialised by the caller.  Each call overwrites every entry it later
// reads, so nothing has to be cleared between calls.
#include <cmath>
#include <mutex>

#include <cuda_runtime.h>

#include "lb.h"

namespace {

constexpr int kThreads = 256;

// One (mass, momx, momy, flag) record per lattice row.
struct RowPartial {
  double m, jx, jy;
  int bad;
  int pad;
};

static __device__ __align__(256) RowPartial g_row_scratch[LB_NOALLOC_MAX_ROWS];

// Host-side addresses of g_row_scratch, resolved once per device.  In host
// code the symbol itself is only a stand-in, never a device address.
constexpr int kMaxDevices = 64;
RowPartial *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Pass 1: block r sums row r of the populations (FP64, fixed order).
template <typename real_t>
__global__ void __launch_bounds__(kThreads)
rows_pass(const real_t *__restrict__ f, int nx, int ny, double nmax, RowPartial *__restrict__ rows) {
  __shared__ double sm[3][kThreads];
  __shared__ int sbad;
  const size_t S = (size_t)nx * ny;
  for (int y = blockIdx.x; y < ny; y += gridDim.x) {
    if (threadIdx.x == 0) sbad = 0;
    double m = 0.0, jx = 0.0, jy = 0.0;
    int bad = 0;
    for (int x = threadIdx.x; x < nx; x += kThreads) {
      const size_t s = (size_t)y * nx + x;
      double v[9];
#pragma unroll
      for (int i = 0; i < 9; i++) v[i] = (double)f[i * S + s];
      double ms = 0.0;
#pragma unroll
      for (int i = 0; i < 9; i++) ms += v[i];
      const double xs = ((((v[1] - v[3]) + v[5]) - v[6]) - v[7]) + v[8];
      const double ys = ((((v[2] - v[4]) + v[5]) + v[6]) - v[7]) - v[8];
      if (!(ms > 0.0 && ms < nmax) || !isfinite(xs) || !isfinite(ys)) bad = 1;
      m += ms;
      jx += xs;
      jy += ys;
    }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = jx;
    sm[2][threadIdx.x] = jy;
    __syncthreads();
    if (bad) sbad = 1;
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
#pragma unroll
        for (int c = 0; c < 3; c++) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      rows[y].m = sm[0][0];
      rows[y].jx = sm[1][0];
      rows[y].jy = sm[2][0];
      rows[y].bad = sbad;
    }
    __syncthreads();
  }
}

// Pass 2: one block adds the row partials in a fixed order.
__global__ void __launch_bounds__(kThreads)
rows_total(const RowPartial *__restrict__ rows, int ny, double *__restrict__ out, int *__restrict__ flag) {
  __shared__ double sm[3][kThreads];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  double acc[3] = {0.0, 0.0, 0.0};
  int bad = 0;
  for (int r = threadIdx.x; r < ny; r += kThreads) {
    acc[0] += rows[r].m;
    acc[1] += rows[r].jx;
    acc[2] += rows[r].jy;
    bad |= rows[r].bad;
  }
#pragma unroll
  for (int c = 0; c < 3; c++) sm[c][threadIdx.x] = acc[c];
  __syncthreads();
  if (bad) sbad = 1;
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int c = 0; c < 3; c++) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sm[0][0];
    out[1] = sm[1][0];
    out[2] = sm[2][0];
    if (flag) *flag = sbad;
  }
}

// Resolve the device address of the scratch array for the current device.
int scratch_for_current_device(RowPartial **ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LB_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LB_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_row_scratch) != cudaSuccess || !p) return LB_ERR_CUDA;
    g_scratch_ptr[dev] = (RowPartial *)p;
  }
  *ptr = g_scratch_ptr[dev];
  return LB_OK;
}

}  // namespace

extern "C" int lb_reduce_noalloc(const void *f, int precision, int32_t nx, int32_t ny, double b,
                                 double *out, int *flag, void *stream) {
  if (!f || !out) return LB_ERR_ARG;
  if (precision != LB_FP64 && precision != LB_FP32) return LB_ERR_ARG;
  if (nx < 1 || ny < 1 || ny > LB_NOALLOC_MAX_ROWS) return LB_ERR_ARG;
  RowPartial *rows = nullptr;
  const int rc = scratch_for_current_device(&rows);
  if (rc != LB_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const double nmax = b > 0.0 ? 1.0 / b : INFINITY;
  const int blocks = ny < 2048 ? ny : 2048;
  // Each launch reports its own error: the caller's pending error state is
  // neither read nor cleared.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaError_t e = precision == LB_FP64
                      ? cudaLaunchKernelEx(&cfg, rows_pass<double>, (const double *)f, (int)nx, (int)ny, nmax, rows)
                      : cudaLaunchKernelEx(&cfg, rows_pass<float>, (const float *)f, (int)nx, (int)ny, nmax, rows);
  if (e != cudaSuccess) return LB_ERR_CUDA;
  cfg.gridDim = dim3(1);
  e = cudaLaunchKernelEx(&cfg, rows_total, (const RowPartial *)rows, (int)ny, out, flag);
  return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
