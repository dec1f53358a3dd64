// lb_api.cu -- host side of the C ABI declared in include/lb.h, plus the
// deterministic FP64 reduction kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_device.cuh"
#include "lb_internal.h"

using lbk::StepArgs;

struct lb_handle {
  lb_params p{};
  cudaStream_t st = nullptr;
  int device = 0;
  size_t S = 0;          // sites
  size_t elem = 0;       // bytes per stored population
  // Layout of a state buffer: plane q, site (x, y) at element
  // q * plane + off + y * pitch + x.  Compact (pitch = nx, off = 0) for the
  // tile kernel; padded with 4 ghost columns / rows for the sweep kernel.
  int pitch = 0;
  long long plane = 0, off = 0;
  bool sweep = false;            // strip-sweep kernel in use
  int store = 0;                 // its storage format (lbk::kStoreF32, kStoreBF16, kStoreFP16)
  CUtensorMap tmap[2][2];        // TMA descriptors of the two state buffers
  float ref_ax = 0.f, ref_dg = 0.f;  // reference populations of 16-bit storage
  float *wide = nullptr;         // 16-bit storage: nine float planes (moments, reductions, init)
  size_t sweep_smem = 0;
  int sweep_seg = 64, sweep_nstrips = 0, sweep_nseg = 0, sweep_base = 0, sweep_extra = 0;
  double *d_cta = nullptr;       // per-CTA partials written by the sweep kernel
  size_t cta_bytes = 0;
  int plan_gen = 0;              // bumped when the tiling or the record array changes
  bool cta_valid = false;        // d_cta describes the current state
  bool total_valid = false;      // d_out holds the current state's sums (fused)
  int *d_err = nullptr;          // bounded-wait failure flag
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  void *sinx = nullptr;  // device table, storage type
  double *d_fields = nullptr;   // 3*S doubles, staging for lb_init mode 1
  void *d_mom = nullptr;        // 3*S doubles, staging for host moments
  double *d_partials = nullptr; // reduction scratch
  int *d_flag = nullptr;
  double *d_out = nullptr;       // 5 doubles: mass, J_x, J_y, unstable, wait error
  unsigned *d_arrive = nullptr;  // CTA arrival counter of the fused sums
  double *mon_ring = nullptr;    // device address of the monitoring ring (lb_monitor)
  int mon_cap = 0;
  // Multi-step launches (lb_step with nsteps >= 2 while not monitoring):
  // per-tile completion counters and dependency lists of the current tiling.
  int persist_cap = 0;           // resident CTAs of that kernel (0: not queried, < 0: unavailable)
  unsigned *d_done = nullptr;
  int *d_dep = nullptr;          // CSR: ntiles + 1 offsets, then indices
  unsigned *d_ticket = nullptr;  // ticket counter of a launch
  int deps_gen = -1;             // plan_gen the lists were built for
  int deps_ntiles = 0;
  unsigned epoch = 0;            // value of every counter between launches
  double *d_mon_recs = nullptr;  // per-step record slots of a monitored multi-step launch
  unsigned *d_mon_arr = nullptr; // their arrival counters (zero between launches)
  int mon_tiles = 0;             // tiles the slots were sized for
  bool in_batch = false;         // instance of an lb_batch
  int red_blocks = 0;
  int64_t step = 0;
  bool initialised = false;
  std::string err;
};

namespace {

thread_local std::string g_create_err;

int fail(lb_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_fail(lb_handle *h, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, m);
}

#define LB_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// Address under which the current device's kernels can read and write p:
// page-locked host memory (mapped into the device's address space under
// unified addressing) or memory of the current device itself; nullptr for
// pageable memory, another device's memory and anything else.  Asked
// through the driver, so that the runtime's last-error state is left as
// the caller had it.
void *device_view(const void *p, bool host_only = false) {
  typedef CUresult (*get_attr_fn)(void *, CUpointer_attribute, CUdeviceptr);
  static get_attr_fn get = nullptr;
  if (!p) return nullptr;
  if (!get) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    get = (get_attr_fn)fn;
  }
  unsigned type = 0;
  if (get(&type, CU_POINTER_ATTRIBUTE_MEMORY_TYPE, (CUdeviceptr)p) != CUDA_SUCCESS) return nullptr;
  if (type == CU_MEMORYTYPE_DEVICE && !host_only) {
    int ord = -1, cur = -2;
    if (get(&ord, CU_POINTER_ATTRIBUTE_DEVICE_ORDINAL, (CUdeviceptr)p) != CUDA_SUCCESS ||
        cudaGetDevice(&cur) != cudaSuccess || ord != cur)
      return nullptr;
    return const_cast<void *>(p);
  }
  if (type != CU_MEMORYTYPE_HOST) return nullptr;
  CUdeviceptr d = 0;
  if (get(&d, CU_POINTER_ATTRIBUTE_DEVICE_POINTER, (CUdeviceptr)p) != CUDA_SUCCESS || !d) return nullptr;
  return (void *)d;
}

template <typename real_t>
StepArgs<real_t> make_args(const lb_handle *h) {
  const lb_params &p = h->p;
  StepArgs<real_t> A;
  A.nx = p.nx;
  A.ny = p.ny;
  A.walls = p.walls;
  A.plane = (size_t)h->plane;
  A.pitch = h->pitch;
  A.off = h->off;
  A.T = (real_t)p.T;
  A.a = (real_t)p.a;
  A.b = (real_t)p.b;
  A.kappa = (real_t)p.kappa;
  A.omega = (real_t)(1.0 / p.tau);
  A.g = (real_t)(1.0 - 1.0 / (2.0 * p.tau));
  A.th = (real_t)(1.0 / 3.0 - p.T);
  A.A0 = (real_t)p.A0;
  A.u_bot = (real_t)p.u_bot;
  A.u_top = (real_t)p.u_top;
  A.N = (real_t)p.N;
  A.M = (real_t)((1.0 - 2.0 * p.N) / 4.0);
  A.Q = (real_t)p.Q;
  const double R = (1.0 - p.Q) / 2.0;
  A.R = (real_t)R;
  A.four_QR = (real_t)(4.0 * (p.Q + R));
  A.sinx = (const real_t *)h->sinx;
  return A;
}

// ------------------------------------------------------------ reductions

constexpr int RED_THREADS = 256;

// Pass 1: each block sums mass and momentum of its grid-stride share of the
// sites in FP64 (fixed order) and flags non-finite or out-of-range sites.
template <typename real_t>
__global__ void __launch_bounds__(RED_THREADS)
reduce_pass1(const real_t *__restrict__ f, int nx, size_t S, int pitch, long long plane,
             long long off, double nmax, double *__restrict__ partials, int *__restrict__ flag) {
  __shared__ double sm[3][RED_THREADS];
  double m = 0.0, jx = 0.0, jy = 0.0;
  int bad = 0;
  for (size_t s = blockIdx.x * (size_t)RED_THREADS + threadIdx.x; s < S;
       s += (size_t)gridDim.x * RED_THREADS) {
    const long long e = off + (long long)(s / (size_t)nx) * pitch + (long long)(s % (size_t)nx);
    double v[9];
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = (double)f[i * plane + e];
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
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int c = 0; c < 3; c++) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x + 0] = sm[0][0];
    partials[3 * blockIdx.x + 1] = sm[1][0];
    partials[3 * blockIdx.x + 2] = sm[2][0];
  }
  if (bad) atomicOr(flag, 1);
}

// Pass 2: one block adds the block partials in a fixed order; out[3] and
// out[4] receive the instability flag pass 1 raised and the step kernels'
// wait/layout error flag (1.0 or 0.0).
__global__ void __launch_bounds__(RED_THREADS)
reduce_pass2(const double *__restrict__ partials, int nblocks, double *__restrict__ out,
             const int *__restrict__ flag, const int *__restrict__ err) {
  __shared__ double sm[3][RED_THREADS];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += RED_THREADS)
#pragma unroll
    for (int c = 0; c < 3; c++) acc[c] += partials[3 * b + c];
#pragma unroll
  for (int c = 0; c < 3; c++) sm[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
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
    out[3] = *flag != 0 ? 1.0 : 0.0;
    out[4] = *err != 0 ? 1.0 : 0.0;
  }
}

// Pass 2 over the sweep kernel's per-CTA records (mass, J_x, J_y, flag);
// out[3], out[4] as in reduce_pass2.
__global__ void __launch_bounds__(RED_THREADS)
reduce_cta(const double *__restrict__ cta, int nblocks, double *__restrict__ out, const int *__restrict__ err) {
  __shared__ double sm[3][RED_THREADS];
  double acc[3] = {0.0, 0.0, 0.0};
  int bad = 0;
  for (int b = threadIdx.x; b < nblocks; b += RED_THREADS) {
#pragma unroll
    for (int c = 0; c < 3; c++) acc[c] += cta[4 * b + c];
    if (!(cta[4 * b + 3] == 0.0)) bad = 1;
  }
#pragma unroll
  for (int c = 0; c < 3; c++) sm[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int c = 0; c < 3; c++) sm[c][threadIdx.x] += sm[c][threadIdx.x + w];
    }
    __syncthreads();
  }
  const int any_bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    out[0] = sm[0][0];
    out[1] = sm[1][0];
    out[2] = sm[2][0];
    out[3] = any_bad ? 1.0 : 0.0;
    out[4] = *err != 0 ? 1.0 : 0.0;
  }
}

bool fp64(const lb_handle *h) { return h->p.precision == LB_FP64; }
bool dev16(const lb_handle *h) { return h->p.precision == LB_BF16DEV || h->p.precision == LB_FP16DEV; }

// Bytes of the compact state of lb_get_state / lb_set_state.
size_t state_bytes(const lb_handle *h) {
  return dev16(h) ? h->S * (sizeof(float) + 8 * 2) : 9 * h->S * h->elem;
}

// Plane q of state buffer b: first interior element and element size.
char *plane_ptr(const lb_handle *h, int b, int q, size_t *esize) {
  char *base = (char *)h->f[b];
  if (!dev16(h)) {
    *esize = h->elem;
    return base + ((size_t)q * h->plane + h->off) * h->elem;
  }
  if (q == 0) {
    *esize = sizeof(float);
    return base + (size_t)h->off * sizeof(float);
  }
  *esize = 2;
  return base + (size_t)h->plane * sizeof(float) + ((size_t)(q - 1) * h->plane + h->off) * 2;
}

// The nine float planes of the current state: the state buffer itself for
// FP32, else the widened copy.
cudaError_t current_f32(lb_handle *h, const float **out) {
  if (!dev16(h)) {
    *out = (const float *)h->f[h->cur];
    return cudaSuccess;
  }
  *out = h->wide;
  return lbk::launch_widen(h->store, h->f[h->cur], h->wide, h->plane, h->ref_ax, h->ref_dg, h->st);
}

lbk::SweepArgs sweep_args(const lb_handle *h, float *fout) {
  const lb_params &p = h->p;
  lbk::SweepArgs A;
  A.nx = p.nx;
  A.ny = p.ny;
  A.walls = p.walls;
  A.pitch = h->pitch;
  A.plane = h->plane;
  A.off = h->off;
  A.seg_h = h->sweep_seg;
  A.nseg = h->sweep_nseg;
  A.nstrips = h->sweep_nstrips;
  A.base_w = h->sweep_base;
  A.extra = h->sweep_extra;
  const double T0 = 1.0 / 3.0;
  A.T = (float)p.T;
  A.a = (float)p.a;
  A.b = (float)p.b;
  A.kappa = (float)p.kappa;
  A.omega = (float)(1.0 / p.tau);
  A.one_minus_omega = (float)(1.0 - 1.0 / p.tau);
  A.g = (float)(1.0 - 1.0 / (2.0 * p.tau));
  A.th = (float)(T0 - p.T);
  A.A0 = (float)p.A0;
  A.u_bot = (float)p.u_bot;
  A.u_top = (float)p.u_top;
  A.N = (float)p.N;
  A.M = (float)((1.0 - 2.0 * p.N) / 4.0);
  A.Q = (float)p.Q;
  A.R = (float)((1.0 - p.Q) / 2.0);
  A.four_QR = (float)(4.0 * (p.Q + (1.0 - p.Q) / 2.0));
  const double k = (p.T - T0) / (2.0 * T0 * T0);
  A.A_rest = (float)(1.0 + k * (0.0 - 2.0 * T0));
  A.A_ax = (float)(1.0 + k * (1.0 - 2.0 * T0));
  A.A_diag = (float)(1.0 + k * (2.0 - 2.0 * T0));
  A.nmax = p.b > 0.0 ? (float)(1.0 / p.b) : 3.0e38f;
  A.ref_ax = h->ref_ax;
  A.ref_dg = h->ref_dg;
  A.sinx = (const float *)h->sinx;
  A.fout = fout;
  A.fdev = dev16(h) ? (void *)((char *)fout + (size_t)h->plane * sizeof(float)) : nullptr;
  A.partials = h->d_cta;
  A.records = 1;
  A.err = h->d_err;
  A.total = nullptr;
  A.arrivals = nullptr;
  A.monitor = nullptr;
  A.mon_step = 0.0;
  return A;
}

// Segment height of a sweep handle; the per-CTA record array must already
// be large enough (see ensure_records).
void set_segments(lb_handle *h, int seg_h) {
  h->sweep_seg = std::max(1, std::min(seg_h, h->p.ny));
  h->sweep_nseg = (h->p.ny + h->sweep_seg - 1) / h->sweep_seg;
  h->cta_valid = false;
  h->total_valid = false;
  h->plan_gen++;
}

// Grow the per-CTA record array to hold `nseg` segments of records.
cudaError_t ensure_records(lb_handle *h, int nseg) {
  const size_t need = 4 * sizeof(double) * (size_t)h->sweep_nstrips * nseg;
  if (need <= h->cta_bytes) return cudaSuccess;
  double *p = nullptr;
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess) e = cudaMalloc((void **)&p, need);
  if (e != cudaSuccess) return e;
  cudaFree(h->d_cta);
  h->d_cta = p;
  h->cta_bytes = need;
  h->cta_valid = false;
  h->total_valid = false;
  h->plan_gen++;
  return cudaSuccess;
}

// Dependency lists and counters of the multi-step kernel for the current
// tiling (rebuilt when the tiling changes; counters then restart at 0).
cudaError_t ensure_deps(lb_handle *h) {
  if (h->deps_gen == h->plan_gen) return cudaSuccess;
  std::vector<int> ofs, idx;
  lbk::sweep_deps(h->store, h->p.nx, h->p.ny, h->p.walls, h->sweep_nstrips, h->sweep_base, h->sweep_extra,
                  h->sweep_seg, ofs, idx);
  const int ntiles = h->sweep_nstrips * h->sweep_nseg;
  std::vector<int> csr(ofs);
  csr.insert(csr.end(), idx.begin(), idx.end());
  cudaError_t e = cudaStreamSynchronize(h->st);  // no launch may still use the old lists
  if (e != cudaSuccess) return e;
  cudaFree(h->d_dep);
  cudaFree(h->d_done);
  h->d_dep = nullptr;
  h->d_done = nullptr;
  h->deps_gen = -1;
  e = cudaMalloc((void **)&h->d_dep, csr.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_dep, csr.data(), csr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_done, (size_t)ntiles * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->d_done, 0, (size_t)ntiles * sizeof(unsigned));
  if (e == cudaSuccess && !h->d_ticket) e = cudaMalloc((void **)&h->d_ticket, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  h->deps_ntiles = ntiles;
  h->epoch = 0;
  h->deps_gen = h->plan_gen;
  return cudaSuccess;
}

constexpr int kMonSlots = 64;  // steps per multi-step launch while monitoring

// Record slots of a monitored multi-step launch (one per step of a launch).
cudaError_t ensure_mon_slots(lb_handle *h, int ntiles) {
  if (h->d_mon_recs && h->mon_tiles >= ntiles) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return e;
  cudaFree(h->d_mon_recs);
  cudaFree(h->d_mon_arr);
  h->d_mon_recs = nullptr;
  h->d_mon_arr = nullptr;
  h->mon_tiles = 0;
  e = cudaMalloc((void **)&h->d_mon_recs, 4 * sizeof(double) * (size_t)ntiles * kMonSlots);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_mon_arr, kMonSlots * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_mon_arr, 0, kMonSlots * sizeof(unsigned), h->st);
  if (e == cudaSuccess) h->mon_tiles = ntiles;
  return e;
}

// nsteps >= 2 steps of a strip-sweep handle in multi-step launches.
// Returns LB_OK, an error code, or 1 when that kernel cannot run here (the
// caller then launches one kernel per step).
int multi_steps(lb_handle *h, int64_t nsteps) {
  if (h->persist_cap == 0) {
    int cap = 0;
    const cudaError_t e = lbk::persist_capacity(h->store, h->sweep_smem, &cap);
    if (e != cudaSuccess) cudaGetLastError();
    h->persist_cap = (e == cudaSuccess && cap > 0) ? cap : -1;
  }
  if (h->persist_cap < 0) return 1;
  LB_CUDA(h, ensure_deps(h));
  const int ntiles = h->deps_ntiles;
  const lbk::SweepArgs A = sweep_args(h, nullptr);
  const int grid = std::min(ntiles, h->persist_cap);
  lbk::MultiOut Q{};
  for (int b = 0; b < 2; ++b) {
    Q.fout[b] = (float *)h->f[b ^ 1];  // a step reading buffer b writes buffer b ^ 1
    Q.fdev[b] = dev16(h) ? (void *)((char *)h->f[b ^ 1] + (size_t)h->plane * sizeof(float)) : nullptr;
  }
  Q.total = h->d_out;
  Q.arrivals = h->d_arrive;
  const bool mon = h->mon_cap > 0;
  if (mon) {
    LB_CUDA(h, ensure_mon_slots(h, ntiles));
    Q.mon_recs = h->d_mon_recs;
    Q.mon_arr = h->d_mon_arr;
    Q.mon_ring = h->mon_ring;
    Q.mon_cap = h->mon_cap;
  }
  // A monitored launch holds at most as many steps as the ring has records,
  // so it writes each ring slot once; launches are stream-ordered, so an
  // earlier step's record never lands after a later one's in the same slot
  // (a tile publishes its completion before its record reduction, so the
  // final sums of different steps of one launch are not ordered).
  const int64_t per_launch = mon ? std::min<int64_t>(kMonSlots, h->mon_cap)
                                 : std::max<int64_t>(2, (1LL << 30) / ntiles);
  for (int64_t done = 0; done < nsteps;) {
    const int chunk = (int)std::min<int64_t>(nsteps - done, per_launch);
    Q.mon_step0 = h->step + 1;  // step number of the first step's result
    lbk::PersistArgs P{};
    P.nitems = ntiles;
    P.nsteps = chunk;
    P.kpar0 = h->cur;
    P.epoch = h->epoch;
    P.done = h->d_done;
    P.dep_ofs = h->d_dep;
    P.dep_idx = h->d_dep + ntiles + 1;
    P.next = h->d_ticket;
    LB_CUDA(h, cudaMemsetAsync(h->d_ticket, 0, sizeof(unsigned), h->st));
    const cudaError_t e = lbk::launch_sweep_multi(h->store, h->tmap, A, P, Q, grid, h->sweep_smem, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_step: multi-step sweep kernel");
    h->cur ^= chunk & 1;
    h->step += chunk;
    h->epoch += (unsigned)chunk;
    h->cta_valid = !mon;  // monitored launches keep their records in the slots
    h->total_valid = true;
    done += chunk;
  }
  return LB_OK;
}

}  // namespace

extern "C" {

int lb_create(const lb_params *p, lb_handle **out) {
  if (!p || !out) return fail(nullptr, LB_ERR_ARG, "lb_create: null argument");
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1) return fail(nullptr, LB_ERR_ARG, "lb_create: nx and ny must be >= 1");
  if (p->walls != 0 && p->walls != 1) return fail(nullptr, LB_ERR_ARG, "lb_create: walls must be 0 or 1");
  if (p->walls && p->ny < 3) return fail(nullptr, LB_ERR_ARG, "lb_create: walls need ny >= 3");
  if (p->precision != LB_FP64 && p->precision != LB_FP32 && p->precision != LB_BF16DEV &&
      p->precision != LB_FP16DEV)
    return fail(nullptr, LB_ERR_ARG, "lb_create: unknown precision");
  if ((p->precision == LB_BF16DEV || p->precision == LB_FP16DEV) &&
      !lbk::sweep_supported(p->precision, p->nx, p->ny))
    return fail(nullptr, LB_ERR_ARG, "lb_create: 16-bit storage needs nx a multiple of 8, nx >= 8 and ny >= 8");
  if (!(p->rho_ref >= 0.0) || !std::isfinite(p->rho_ref))
    return fail(nullptr, LB_ERR_ARG, "lb_create: rho_ref must be finite and >= 0");
  if (!(p->tau > 0.5)) return fail(nullptr, LB_ERR_ARG, "lb_create: tau must exceed 1/2");
  if (!(p->T > 0.0) || !(p->b >= 0.0) || !std::isfinite(p->a) || !std::isfinite(p->kappa) ||
      !std::isfinite(p->N) || !std::isfinite(p->Q) || !std::isfinite(p->A0) ||
      !(p->lambda >= 0.0) || !std::isfinite(p->u_bot) || !std::isfinite(p->u_top))
    return fail(nullptr, LB_ERR_ARG, "lb_create: non-finite or out-of-range physical parameter");
  if ((double)p->nx * (double)p->ny * 9.0 > 4.0e9)
    return fail(nullptr, LB_ERR_ARG, "lb_create: lattice too large");

  lb_handle *h = new (std::nothrow) lb_handle();
  if (!h) return fail(nullptr, LB_ERR_OOM, "lb_create: host allocation failed");
  h->p = *p;
  h->st = (cudaStream_t)p->stream;
  h->S = (size_t)p->nx * (size_t)p->ny;
  h->elem = fp64(h) ? sizeof(double) : sizeof(float);
  if (dev16(h)) {
    // Reference density of the deviations: the vdW critical density 1/(3b)
    // unless given.
    if (h->p.rho_ref == 0.0) h->p.rho_ref = p->b > 0.0 ? 1.0 / (3.0 * p->b) : 1.0;
    h->ref_ax = (float)(h->p.rho_ref / 9.0);
    h->ref_dg = (float)(h->p.rho_ref / 36.0);
  }
  // The strip-sweep kernel needs x in multiples of its TMA column quantum
  // and at least 8 sites per direction (one ghost band of 4 each).
  h->store = p->precision;
  h->sweep = !fp64(h) && lbk::sweep_supported(h->store, p->nx, p->ny);
  if (h->sweep) {
    h->pitch = ((p->nx + 8 + 31) / 32) * 32;
    h->plane = (long long)h->pitch * (p->ny + 8);
    h->off = 4LL * h->pitch + 4;
    lbk::sweep_plan(h->store, p->nx, p->ny, &h->sweep_nstrips, &h->sweep_base, &h->sweep_extra, &h->sweep_seg,
                    &h->sweep_nseg);
  } else {
    h->pitch = p->nx;
    h->plane = (long long)h->S;
    h->off = 0;
  }
  const size_t buf_bytes = h->sweep ? lbk::sweep_buffer_bytes(h->store, h->plane) : 9 * (size_t)h->plane * h->elem;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->f[0], buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->f[1], buf_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->f[0], 0, buf_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->f[1], 0, buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
  if (e == cudaSuccess && h->sweep) {
    h->cta_bytes = 4 * sizeof(double) * (size_t)h->sweep_nstrips * h->sweep_nseg;
    e = cudaMalloc((void **)&h->d_cta, h->cta_bytes);
    if (e == cudaSuccess) e = lbk::sweep_prepare(h->store, &h->sweep_smem);
    for (int b = 0; b < 2 && e == cudaSuccess; b++)
      e = lbk::sweep_make_maps(h->store, h->f[b], h->pitch, p->ny, h->plane, &h->tmap[b][0], &h->tmap[b][1]);
  }
  if (e == cudaSuccess && dev16(h)) e = cudaMalloc((void **)&h->wide, 9 * (size_t)h->plane * sizeof(float));
  if (e == cudaSuccess && dev16(h)) e = cudaMemset(h->wide, 0, 9 * (size_t)h->plane * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->sinx, (size_t)p->nx * h->elem);
  h->red_blocks = (int)std::min<size_t>((h->S + RED_THREADS - 1) / RED_THREADS, 1024);
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_partials, 3 * (size_t)h->red_blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_out, 5 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_arrive, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(h->d_arrive, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    // sin(2 pi x / lambda), evaluated in FP64 on the host.
    const size_t nb = (size_t)p->nx * h->elem;
    void *tab = malloc(nb);
    if (!tab) e = cudaErrorMemoryAllocation;
    else {
      for (int x = 0; x < p->nx; x++) {
        const double s = (p->lambda != 0.0) ? std::sin((6.283185307179586 * (double)x) / p->lambda) : 0.0;
        if (fp64(h)) ((double *)tab)[x] = s;
        else ((float *)tab)[x] = (float)s;
      }
      e = cudaMemcpy(h->sinx, tab, nb, cudaMemcpyHostToDevice);
      free(tab);
    }
  }
  if (e != cudaSuccess) {
    std::string m = std::string("lb_create: ") + cudaGetErrorString(e);
    int code = (e == cudaErrorMemoryAllocation) ? LB_ERR_OOM : LB_ERR_CUDA;
    lb_destroy(h);
    return fail(nullptr, code, m);
  }
  *out = h;
  return LB_OK;
}

int lb_init(lb_handle *h, int mode, uint64_t seed, double rho_mean, double noise_amp,
            const double *rho0, const double *ux0, const double *uy0) {
  if (!h) return LB_ERR_ARG;
  if (mode != 0 && mode != 1) return fail(h, LB_ERR_ARG, "lb_init: mode must be 0 or 1");
  const double *dr = nullptr, *du = nullptr, *dv = nullptr;
  if (mode == 1) {
    if (!rho0) return fail(h, LB_ERR_ARG, "lb_init: mode 1 needs rho0");
    // Page-locked host fields and fields in this device's memory are read
    // by the init kernel where they are; others are staged first.
    const double *src[3] = {rho0, ux0, uy0};
    const double **dst[3] = {&dr, &du, &dv};
    for (int k = 0; k < 3; ++k) {
      if (!src[k]) continue;
      if (void *m = device_view(src[k])) {
        *dst[k] = (const double *)m;
        continue;
      }
      if (!h->d_fields) LB_CUDA(h, cudaMalloc((void **)&h->d_fields, 3 * h->S * sizeof(double)));
      LB_CUDA(h, cudaMemcpyAsync(h->d_fields + k * h->S, src[k], h->S * sizeof(double), cudaMemcpyDefault, h->st));
      *dst[k] = h->d_fields + k * h->S;
    }
  }
  h->cur = 0;
  // 16-bit storage: the float equilibrium goes through the storage format.
  float *f32 = dev16(h) ? h->wide : (float *)h->f[0];
  cudaError_t e = fp64(h)
                      ? lbk::launch_init((double *)h->f[0], h->p.nx, h->p.ny, h->pitch, h->plane,
                                         h->off, mode, seed, rho_mean, noise_amp, dr, du, dv,
                                         h->p.T, h->st)
                      : lbk::launch_init(f32, h->p.nx, h->p.ny, h->pitch, h->plane,
                                         h->off, mode, seed, rho_mean, noise_amp, dr, du, dv,
                                         h->p.T, h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "lb_init: init kernel");
  if (h->sweep) {
    e = lbk::launch_ghost_fill(f32, 4, 9, h->p.nx, h->p.ny, h->pitch, h->plane, h->off, h->p.walls, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_init: ghost fill");
  }
  if (dev16(h)) {
    e = lbk::launch_narrow(h->store, h->wide, h->f[0], h->plane, h->ref_ax, h->ref_dg, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "lb_init: 16-bit store");
  }
  h->cta_valid = false;
  h->total_valid = false;
  if (mode == 1) LB_CUDA(h, cudaStreamSynchronize(h->st));
  h->step = 0;
  h->initialised = true;
  return LB_OK;
}

int lb_step(lb_handle *h, int64_t nsteps) {
  if (!h) return LB_ERR_ARG;
  if (nsteps < 0) return fail(h, LB_ERR_ARG, "lb_step: nsteps < 0");
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_step: state not initialised");
  if (fp64(h)) {
    const StepArgs<double> A = make_args<double>(h);
    for (int64_t k = 0; k < nsteps; k++) {
      cudaError_t e = lbk::launch_step((const double *)h->f[h->cur], (double *)h->f[h->cur ^ 1], A, h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "lb_step: step kernel");
      h->cur ^= 1;
      h->step++;
    }
  } else if (h->sweep) {
    // Two steps or more: multi-step launches.
    if (nsteps >= 2) {
      const int rc = multi_steps(h, nsteps);
      if (rc != 1) return rc;
    }
    // Per-CTA mass/momentum records only on the last step: lb_reduce reads
    // only the current state's.
    for (int64_t k = 0; k < nsteps; k++) {
      lbk::SweepArgs A = sweep_args(h, (float *)h->f[h->cur ^ 1]);
      // records on the last step, or on every step while monitoring
      A.records = (k == nsteps - 1 || h->mon_cap > 0) ? 1 : 0;
      if (A.records) {  // the last CTA also leaves the global sums in d_out
        A.total = h->d_out;
        A.arrivals = h->d_arrive;
      }
      if (h->mon_cap > 0) {
        const int64_t s = h->step + 1;
        A.monitor = h->mon_ring + 6 * (s % h->mon_cap);
        A.mon_step = (double)s;
      }
      cudaError_t e = lbk::launch_sweep(h->store, h->tmap[h->cur][0], h->tmap[h->cur][1], A, h->sweep_smem, h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "lb_step: sweep kernel");
      h->cur ^= 1;
      h->step++;
      h->cta_valid = true;
      h->total_valid = A.records != 0;
    }
  } else {
    const StepArgs<float> A = make_args<float>(h);
    for (int64_t k = 0; k < nsteps; k++) {
      cudaError_t e = lbk::launch_step((const float *)h->f[h->cur], (float *)h->f[h->cur ^ 1], A, h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "lb_step: step kernel");
      h->cur ^= 1;
      h->step++;
    }
  }
  return LB_OK;
}

int lb_moments(lb_handle *h, void *rho, void *ux, void *uy, int dtype, int on_device) {
  if (!h) return LB_ERR_ARG;
  if (dtype != LB_DTYPE_F64 && dtype != LB_DTYPE_F32) return fail(h, LB_ERR_ARG, "lb_moments: bad dtype");
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_moments: state not initialised");
  const size_t es = dtype == LB_DTYPE_F64 ? sizeof(double) : sizeof(float);
  void *dn = rho, *du = ux, *dv = uy;
  bool staged[3] = {false, false, false};
  if (!on_device) {
    // The kernel writes page-locked host arrays (and this device's memory)
    // directly; pageable ones get a device buffer and a copy.
    void *const host[3] = {rho, ux, uy};
    void **dst[3] = {&dn, &du, &dv};
    for (int k = 0; k < 3; ++k) {
      if (!host[k]) continue;
      if (void *m = device_view(host[k])) {
        *dst[k] = m;
        continue;
      }
      if (!h->d_mom) LB_CUDA(h, cudaMalloc(&h->d_mom, 3 * h->S * sizeof(double)));
      *dst[k] = (char *)h->d_mom + k * h->S * es;
      staged[k] = true;
    }
  }
  cudaError_t e;
  if (fp64(h)) {
    e = lbk::launch_moments((const double *)h->f[h->cur], make_args<double>(h), dn, du, dv, dtype, h->st);
  } else {
    const float *f32 = nullptr;
    e = current_f32(h, &f32);
    if (e == cudaSuccess) e = lbk::launch_moments(f32, make_args<float>(h), dn, du, dv, dtype, h->st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "lb_moments: kernel");
  if (!on_device) {
    const size_t nb = h->S * es;
    if (staged[0]) LB_CUDA(h, cudaMemcpyAsync(rho, dn, nb, cudaMemcpyDefault, h->st));
    if (staged[1]) LB_CUDA(h, cudaMemcpyAsync(ux, du, nb, cudaMemcpyDefault, h->st));
    if (staged[2]) LB_CUDA(h, cudaMemcpyAsync(uy, dv, nb, cudaMemcpyDefault, h->st));
    LB_CUDA(h, cudaStreamSynchronize(h->st));
  }
  return LB_OK;
}

// Enqueue the global sums of the current state into d_out[0..4] (mass,
// momentum x, y, instability flag, wait/layout error flag).
static int enqueue_reduce(lb_handle *h) {
  const double nmax = h->p.b > 0.0 ? 1.0 / h->p.b : INFINITY;
  if (h->sweep && h->total_valid) return LB_OK;  // the last step's kernel left them there
  if (h->sweep && h->cta_valid) {
    // The last sweep step left one record per CTA (site sums in FP32,
    // totals in FP64): only the final pass remains.
    reduce_cta<<<1, RED_THREADS, 0, h->st>>>(h->d_cta, h->sweep_nstrips * h->sweep_nseg, h->d_out, h->d_err);
  } else {
    LB_CUDA(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->st));
    if (fp64(h))
      reduce_pass1<double><<<h->red_blocks, RED_THREADS, 0, h->st>>>(
          (const double *)h->f[h->cur], h->p.nx, h->S, h->pitch, h->plane, h->off, nmax,
          h->d_partials, h->d_flag);
    else {
      const float *f32 = nullptr;
      LB_CUDA(h, current_f32(h, &f32));
      reduce_pass1<float><<<h->red_blocks, RED_THREADS, 0, h->st>>>(
          f32, h->p.nx, h->S, h->pitch, h->plane, h->off, nmax, h->d_partials, h->d_flag);
    }
    LB_CUDA(h, cudaGetLastError());
    reduce_pass2<<<1, RED_THREADS, 0, h->st>>>(h->d_partials, h->red_blocks, h->d_out, h->d_flag, h->d_err);
  }
  LB_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int lb_reduce(lb_handle *h, double *out) {
  if (!h || !out) return h ? fail(h, LB_ERR_ARG, "lb_reduce: null output") : LB_ERR_ARG;
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_reduce: state not initialised");
  const int rc = enqueue_reduce(h);
  if (rc != LB_OK) return rc;
  double r[5];
  LB_CUDA(h, cudaMemcpyAsync(r, h->d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  LB_CUDA(h, cudaStreamSynchronize(h->st));
  out[0] = r[0];
  out[1] = r[1];
  out[2] = r[2];
  if (r[4] != 0.0) return fail(h, LB_ERR_TIMEOUT, "lb_reduce: a device-side wait gave up or a layout check failed during a step");
  if (r[3] != 0.0) {
    char m[128];
    snprintf(m, sizeof m, "lb_reduce: non-finite or out-of-range density at step %lld", (long long)h->step);
    return fail(h, LB_ERR_UNSTABLE, m);
  }
  return LB_OK;
}

int lb_reduce_async(lb_handle *h, double *out) {
  if (!h || !out) return h ? fail(h, LB_ERR_ARG, "lb_reduce_async: null output") : LB_ERR_ARG;
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_reduce_async: state not initialised");
  const int rc = enqueue_reduce(h);
  if (rc != LB_OK) return rc;
  LB_CUDA(h, cudaMemcpyAsync(out, h->d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return LB_OK;
}

int lb_monitor(lb_handle *h, double *host_ring, int32_t capacity) {
  if (!h) return LB_ERR_ARG;
  if (capacity < 0) return fail(h, LB_ERR_ARG, "lb_monitor: capacity < 0");
  if (!host_ring || capacity == 0) {
    h->mon_ring = nullptr;
    h->mon_cap = 0;
    return LB_OK;
  }
  if (!h->sweep || h->in_batch)
    return fail(h, LB_ERR_ARG, "lb_monitor: only for strip-sweep handles outside a batch");
  void *dev = device_view(host_ring, true);
  if (!dev) return fail(h, LB_ERR_ARG, "lb_monitor: the ring is not page-locked memory the device can address");
  // the per-step record slots of the current tiling now, not at the first
  // monitored step (a later, finer tiling grows them at its launch)
  LB_CUDA(h, ensure_mon_slots(h, h->sweep_nstrips * h->sweep_nseg));
  h->mon_ring = static_cast<double *>(dev);
  h->mon_cap = capacity;
  return LB_OK;
}

int lb_get_state(lb_handle *h, void *buf, size_t *bytes) {
  if (!h || !bytes) return h ? fail(h, LB_ERR_ARG, "lb_get_state: null size") : LB_ERR_ARG;
  const size_t need = state_bytes(h);
  if (!buf) {
    *bytes = need;
    return LB_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return fail(h, LB_ERR_ARG, "lb_get_state: buffer too small");
  }
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_get_state: state not initialised");
  if (h->pitch == h->p.nx && h->off == 0 && (size_t)h->plane == h->S) {
    LB_CUDA(h, cudaMemcpyAsync(buf, h->f[h->cur], need, cudaMemcpyDeviceToHost, h->st));
  } else {
    char *dst = (char *)buf;
    for (int q = 0; q < 9; q++) {
      size_t es = 0;
      const char *src = plane_ptr(h, h->cur, q, &es);
      const size_t row = (size_t)h->p.nx * es;
      LB_CUDA(h, cudaMemcpy2DAsync(dst, row, src, (size_t)h->pitch * es, row, h->p.ny,
                                   cudaMemcpyDeviceToHost, h->st));
      dst += h->S * es;
    }
  }
  LB_CUDA(h, cudaStreamSynchronize(h->st));
  *bytes = need;
  return LB_OK;
}

int lb_set_state(lb_handle *h, const void *buf, size_t bytes, int64_t step) {
  if (!h || !buf) return h ? fail(h, LB_ERR_ARG, "lb_set_state: null buffer") : LB_ERR_ARG;
  const size_t need = state_bytes(h);
  if (bytes != need) return fail(h, LB_ERR_ARG, "lb_set_state: size mismatch");
  if (step < 0) return fail(h, LB_ERR_ARG, "lb_set_state: negative step");
  if (h->pitch == h->p.nx && h->off == 0 && (size_t)h->plane == h->S) {
    LB_CUDA(h, cudaMemcpyAsync(h->f[h->cur], buf, need, cudaMemcpyHostToDevice, h->st));
  } else {
    const char *src = (const char *)buf;
    for (int q = 0; q < 9; q++) {
      size_t es = 0;
      char *dst = plane_ptr(h, h->cur, q, &es);
      const size_t row = (size_t)h->p.nx * es;
      LB_CUDA(h, cudaMemcpy2DAsync(dst, (size_t)h->pitch * es, src, row, row, h->p.ny,
                                   cudaMemcpyHostToDevice, h->st));
      src += h->S * es;
    }
    if (dev16(h)) {
      char *base = (char *)h->f[h->cur];
      LB_CUDA(h, lbk::launch_ghost_fill(base, 4, 1, h->p.nx, h->p.ny, h->pitch, h->plane, h->off, h->p.walls,
                                        h->st));
      LB_CUDA(h, lbk::launch_ghost_fill(base + (size_t)h->plane * sizeof(float), 2, 8, h->p.nx, h->p.ny, h->pitch,
                                        h->plane, h->off, h->p.walls, h->st));
    } else {
      LB_CUDA(h, lbk::launch_ghost_fill(h->f[h->cur], 4, 9, h->p.nx, h->p.ny, h->pitch, h->plane, h->off,
                                        h->p.walls, h->st));
    }
  }
  LB_CUDA(h, cudaStreamSynchronize(h->st));
  h->cta_valid = false;
  h->total_valid = false;
  h->step = step;
  h->initialised = true;
  return LB_OK;
}

int lb_autotune(lb_handle *h, int steps, int32_t *seg_h) {
  if (!h) return LB_ERR_ARG;
  if (steps < 1) return fail(h, LB_ERR_ARG, "lb_autotune: steps must be >= 1");
  if (!h->initialised) return fail(h, LB_ERR_STATE, "lb_autotune: state not initialised");
  if (!h->sweep) {
    if (seg_h) *seg_h = 0;
    return LB_OK;  // the tile kernel has no tiling choice
  }
  // Candidate segment heights (rows per CTA): fewer rows give more CTAs per
  // SM and more warm-up rows; the best trade depends on the lattice and on
  // the storage's occupancy.
  const int cand[] = {24, 32, 40, 48, 52, 56, 64, 72, 80, 96, 128, 192, 256};
  const int ny = h->p.ny;
  int max_nseg = h->sweep_nseg;
  for (int c : cand) max_nseg = std::max(max_nseg, (ny + std::min(c, ny) - 1) / std::min(c, ny));
  // Strip counts: the fewest strips, and up to three more while the strips
  // stay at least 64 columns wide.  More, narrower strips cost more halo
  // columns but change how the tiles of the last step fill the GPU (the
  // tail of a multi-step launch); the timing decides.
  const int s_min = lbk::sweep_min_strips(h->store, h->p.nx);
  std::vector<int> strips{s_min};
  for (int sc = s_min + 1; sc <= s_min + 3; ++sc) {
    int bw = 0, ex = 0;
    lbk::sweep_strips(h->store, h->p.nx, sc, &bw, &ex);
    if (bw >= 64) strips.push_back(sc);
  }
  const int strips0 = h->sweep_nstrips, base0 = h->sweep_base, extra0 = h->sweep_extra;
  // Per-CTA records sized for the most strips and the smallest segments
  // (kept afterwards).
  h->sweep_nstrips = strips.back();
  cudaError_t er = ensure_records(h, max_nseg);
  h->sweep_nstrips = strips0;
  LB_CUDA(h, er);
  h->cta_valid = false;
  h->total_valid = false;

  const size_t buf_bytes = lbk::sweep_buffer_bytes(h->store, h->plane);
  const int cur0 = h->cur;
  const int64_t step0 = h->step;
  const int seg0 = h->sweep_seg;
  void *save = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = seg0, best_strips = strips0, rc = LB_OK;
  float best_ms = 3.0e38f;
  cudaError_t e = cudaMalloc(&save, buf_bytes);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(save, h->f[cur0], buf_bytes, cudaMemcpyDeviceToDevice, h->st);
  // One timing of `steps` steps (after a 2-step warm-up) of a tiling, from
  // the saved state, which is restored afterwards; < 0 on failure.
  auto time_tiling = [&](int sc, int sh) -> float {
    h->sweep_nstrips = sc;
    lbk::sweep_strips(h->store, h->p.nx, sc, &h->sweep_base, &h->sweep_extra);
    set_segments(h, sh);
    float ms = -1.f;
    rc = lb_step(h, 2);  // warm-up
    if (rc == LB_OK) e = cudaEventRecord(e0, h->st);
    if (rc == LB_OK && e == cudaSuccess) rc = lb_step(h, steps);
    if (rc == LB_OK && e == cudaSuccess) e = cudaEventRecord(e1, h->st);
    if (rc == LB_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (rc == LB_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    h->cur = cur0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->f[cur0], save, buf_bytes, cudaMemcpyDeviceToDevice, h->st);
    return (rc == LB_OK && e == cudaSuccess) ? ms : -1.f;
  };
  // Every candidate once, then the three fastest twice more: the minimum of
  // three timings decides among them (single timings of close candidates
  // differ by less than their run-to-run spread).
  struct Timed {
    float ms;
    int sc, sh;
  };
  std::vector<Timed> timed;
  for (int sc : strips) {
    int last = -1;
    for (int c : cand) {
      if (e != cudaSuccess || rc != LB_OK) break;
      const int sh = std::min(c, ny);
      if (sh == last) continue;
      last = sh;
      const float ms = time_tiling(sc, sh);
      if (ms >= 0.f) timed.push_back({ms, sc, sh});
    }
  }
  std::sort(timed.begin(), timed.end(), [](const Timed &a, const Timed &b) { return a.ms < b.ms; });
  if (timed.size() > 3) timed.resize(3);
  for (int rep = 0; rep < 2; ++rep)
    for (Timed &t : timed) {
      if (e != cudaSuccess || rc != LB_OK) break;
      const float ms = time_tiling(t.sc, t.sh);
      if (ms >= 0.f) t.ms = std::min(t.ms, ms);
    }
  for (const Timed &t : timed)
    if (t.ms < best_ms) {
      best_ms = t.ms;
      best = t.sh;
      best_strips = t.sc;
    }
  h->cur = cur0;
  h->step = step0;
  const bool tuned = rc == LB_OK && e == cudaSuccess;
  h->sweep_nstrips = tuned ? best_strips : strips0;
  if (tuned)
    lbk::sweep_strips(h->store, h->p.nx, h->sweep_nstrips, &h->sweep_base, &h->sweep_extra);
  else {
    h->sweep_base = base0;
    h->sweep_extra = extra0;
  }
  set_segments(h, tuned ? best : seg0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(save);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, e, "lb_autotune");
  if (rc != LB_OK) return rc;
  if (seg_h) *seg_h = h->sweep_seg;
  return LB_OK;
}

int lb_sweep_dependencies(int32_t precision, int32_t nx, int32_t ny, int32_t walls, int32_t nstrips,
                          int32_t seg_h, int32_t *ofs, int32_t *idx, int64_t cap, int64_t *count) {
  if (!ofs || !count || cap < 0 || (cap > 0 && !idx)) return LB_ERR_ARG;
  if ((precision != LB_FP32 && precision != LB_BF16DEV && precision != LB_FP16DEV) || (walls != 0 && walls != 1))
    return LB_ERR_ARG;
  const int store = precision;  // the storage codes of the sweep are the precision codes
  if (!lbk::sweep_supported(store, nx, ny) || seg_h < 1) return LB_ERR_ARG;
  const int qn = store == lbk::kStoreF32 ? 4 : 8;
  if (nstrips < lbk::sweep_min_strips(store, nx) || nstrips > nx / (2 * qn)) return LB_ERR_ARG;
  int base = 0, extra = 0;
  lbk::sweep_strips(store, nx, nstrips, &base, &extra);
  std::vector<int> o, d;
  lbk::sweep_deps(store, nx, ny, walls, nstrips, base, extra, std::min((int)seg_h, (int)ny), o, d);
  *count = (int64_t)d.size();
  if (cap < *count) return LB_ERR_ARG;
  for (size_t i = 0; i < o.size(); ++i) ofs[i] = o[i];
  for (size_t i = 0; i < d.size(); ++i) idx[i] = d[i];
  return LB_OK;
}

int lb_get_tiling(const lb_handle *h, int32_t *nstrips, int32_t *seg_h) {
  if (!h || !nstrips || !seg_h) return LB_ERR_ARG;
  *nstrips = h->sweep ? h->sweep_nstrips : 0;
  *seg_h = h->sweep ? h->sweep_seg : 0;
  return LB_OK;
}

int lb_set_tiling(lb_handle *h, int32_t nstrips, int32_t seg_h) {
  if (!h) return LB_ERR_ARG;
  if (!h->sweep) return LB_OK;
  const int s_min = lbk::sweep_min_strips(h->store, h->p.nx);
  const int qn = h->store == lbk::kStoreF32 ? 4 : 8;
  if (nstrips < s_min || nstrips > h->p.nx / (2 * qn) || seg_h < 1)
    return fail(h, LB_ERR_ARG, "lb_set_tiling: strip count or segment height out of range");
  const int sh = std::min((int)seg_h, h->p.ny);
  const int old = h->sweep_nstrips;
  h->sweep_nstrips = nstrips;
  const cudaError_t e = ensure_records(h, (h->p.ny + sh - 1) / sh);
  if (e != cudaSuccess) {
    h->sweep_nstrips = old;
    return cuda_fail(h, e, "lb_set_tiling");
  }
  lbk::sweep_strips(h->store, h->p.nx, nstrips, &h->sweep_base, &h->sweep_extra);
  set_segments(h, sh);
  return LB_OK;
}

int lb_set_seg_h(lb_handle *h, int32_t seg_h) {
  if (!h) return LB_ERR_ARG;
  if (seg_h < 1) return fail(h, LB_ERR_ARG, "lb_set_seg_h: seg_h must be >= 1");
  if (!h->sweep) return LB_OK;
  const int sh = std::min((int)seg_h, h->p.ny);
  LB_CUDA(h, ensure_records(h, (h->p.ny + sh - 1) / sh));
  set_segments(h, sh);
  return LB_OK;
}

int lb_get_step(const lb_handle *h, int64_t *step) {
  if (!h || !step) return LB_ERR_ARG;
  *step = h->step;
  return LB_OK;
}

int lb_destroy(lb_handle *h) {
  if (!h) return LB_OK;
  if (h->st || h->initialised) cudaStreamSynchronize(h->st);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->sinx);
  cudaFree(h->d_fields);
  cudaFree(h->d_mom);
  cudaFree(h->d_partials);
  cudaFree(h->d_flag);
  cudaFree(h->d_out);
  cudaFree(h->d_arrive);
  cudaFree(h->d_cta);
  cudaFree(h->d_err);
  cudaFree(h->wide);
  cudaFree(h->d_done);
  cudaFree(h->d_dep);
  cudaFree(h->d_ticket);
  cudaFree(h->d_mon_recs);
  cudaFree(h->d_mon_arr);
  delete h;
  return LB_OK;
}

const char *lb_last_error(const lb_handle *h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

}  // extern "C"

/* ------------------------------------------------------------------------
 * Batched sweep over many independent lattices (one launch per step).
 * ------------------------------------------------------------------------ */

struct lb_batch {
  std::vector<lb_handle *> hs;
  cudaStream_t st = nullptr;
  cudaStream_t cap = nullptr;  // private stream for graph capture
  int store = 0;
  size_t smem = 0;
  lbk::BatchItem *d_items = nullptr;
  lbk::SweepArgs *d_args = nullptr;
  CUtensorMap *d_maps = nullptr;
  int nitems = 0, items_cap = 0;
  std::vector<int> par0;  // input-buffer parity of each instance at kpar = 0
  std::vector<int> gen;   // plan_gen of each instance when the list was built
  int kpar = 0;           // parity of the next batch step
  bool dirty = true;      // device work list out of date
  cudaGraphExec_t graph = nullptr;  // two consecutive steps, kpar 0 then 1
  // Multi-step launches (lb_batch_step with nsteps >= 2): per-item
  // completion counters and dependency lists, rebuilt with the work list.
  int persist_cap = 0;              // resident CTAs of that kernel (0: not queried, < 0: unavailable)
  unsigned *d_done = nullptr;
  int *d_dep = nullptr;             // CSR: nitems + 1 offsets, then indices
  int done_cap = 0, dep_cap = 0;
  unsigned *d_ticket = nullptr;     // ticket counter of a multi-step launch
  unsigned epoch = 0;               // value of every counter between launches
  std::string err;
};

namespace {

int bfail(lb_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  else g_create_err = msg;
  return code;
}

#define LB_BCUDA(b, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

// Rebuild the work list, the per-instance arguments and tensor maps.
int batch_rebuild(lb_batch *b) {
  const int n = (int)b->hs.size();
  std::vector<lbk::BatchItem> items;
  std::vector<lbk::SweepArgs> args(2 * (size_t)n);
  std::vector<CUtensorMap> maps(4 * (size_t)n);
  b->par0.assign(n, 0);
  b->gen.assign(n, 0);
  for (int i = 0; i < n; i++) {
    lb_handle *h = b->hs[i];
    b->par0[i] = h->cur;
    b->gen[i] = h->plan_gen;
    for (int p = 0; p < 2; p++) {
      args[2 * i + p] = sweep_args(h, (float *)h->f[p ^ 1]);
      maps[4 * i + 2 * p + 0] = h->tmap[p][0];
      maps[4 * i + 2 * p + 1] = h->tmap[p][1];
    }
    for (int sg = 0; sg < h->sweep_nseg; sg++)
      for (int sp = 0; sp < h->sweep_nstrips; sp++)
        items.push_back({i, sp, sg, sg * h->sweep_nstrips + sp, h->cur});
  }
  // Longest CTAs first (rows of the segment plus the 7-row warm-up), so the
  // block scheduler fills the tail with the short ones.
  auto rows = [&](const lbk::BatchItem &it) {
    const lb_handle *h = b->hs[it.inst];
    const int ya = it.seg * h->sweep_seg;
    return std::min(h->p.ny, ya + h->sweep_seg) - ya;
  };
  std::stable_sort(items.begin(), items.end(),
                   [&](const lbk::BatchItem &x, const lbk::BatchItem &y) { return rows(x) > rows(y); });
  if ((int)items.size() > b->items_cap) {
    LB_BCUDA(b, cudaStreamSynchronize(b->st));
    cudaFree(b->d_items);
    b->d_items = nullptr;
    LB_BCUDA(b, cudaMalloc((void **)&b->d_items, items.size() * sizeof(lbk::BatchItem)));
    b->items_cap = (int)items.size();
  }
  b->nitems = (int)items.size();
  // Dependency lists of the multi-step kernel, per item: the tiles of the
  // same lattice its tile depends on (lbk::sweep_deps), as item indices.
  std::vector<int> csr(1, 0), dep_idx;
  {
    std::vector<std::vector<int>> item_of(n);
    for (int i = 0; i < n; i++) item_of[i].assign((size_t)b->hs[i]->sweep_nstrips * b->hs[i]->sweep_nseg, -1);
    for (int j = 0; j < (int)items.size(); j++) {
      const lbk::BatchItem &it = items[j];
      item_of[it.inst][(size_t)it.seg * b->hs[it.inst]->sweep_nstrips + it.strip] = j;
    }
    std::vector<std::vector<int>> ofs(n), idx(n);
    for (int i = 0; i < n; i++) {
      const lb_handle *h = b->hs[i];
      lbk::sweep_deps(h->store, h->p.nx, h->p.ny, h->p.walls, h->sweep_nstrips, h->sweep_base, h->sweep_extra,
                      h->sweep_seg, ofs[i], idx[i]);
    }
    for (const lbk::BatchItem &it : items) {
      const size_t tile = (size_t)it.seg * b->hs[it.inst]->sweep_nstrips + it.strip;
      for (int d = ofs[it.inst][tile]; d < ofs[it.inst][tile + 1]; d++) dep_idx.push_back(item_of[it.inst][idx[it.inst][d]]);
      csr.push_back((int)dep_idx.size());
    }
    csr.insert(csr.end(), dep_idx.begin(), dep_idx.end());
  }
  if ((int)items.size() > b->done_cap || (int)csr.size() > b->dep_cap) {
    LB_BCUDA(b, cudaStreamSynchronize(b->st));
    cudaFree(b->d_done);
    cudaFree(b->d_dep);
    b->d_done = nullptr;
    b->d_dep = nullptr;
    b->done_cap = b->dep_cap = 0;
    LB_BCUDA(b, cudaMalloc((void **)&b->d_done, items.size() * sizeof(unsigned)));
    LB_BCUDA(b, cudaMalloc((void **)&b->d_dep, csr.size() * sizeof(int)));
    b->done_cap = (int)items.size();
    b->dep_cap = (int)csr.size();
  }
  LB_BCUDA(b, cudaMemsetAsync(b->d_done, 0, items.size() * sizeof(unsigned), b->st));
  b->epoch = 0;
  LB_BCUDA(b, cudaMemcpyAsync(b->d_dep, csr.data(), csr.size() * sizeof(int), cudaMemcpyHostToDevice, b->st));
  LB_BCUDA(b, cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(lbk::BatchItem),
                              cudaMemcpyHostToDevice, b->st));
  LB_BCUDA(b, cudaMemcpyAsync(b->d_args, args.data(), args.size() * sizeof(lbk::SweepArgs),
                              cudaMemcpyHostToDevice, b->st));
  LB_BCUDA(b, cudaMemcpyAsync(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                              cudaMemcpyHostToDevice, b->st));
  LB_BCUDA(b, cudaStreamSynchronize(b->st));  // host arrays go out of scope
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->kpar = 0;
  b->dirty = false;
  return LB_OK;
}

// Two consecutive batch steps (kpar 0, then 1) as one CUDA graph.
int batch_graph(lb_batch *b) {
  if (b->graph) return LB_OK;
  cudaGraph_t g = nullptr;
  LB_BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = lbk::launch_sweep_batch(b->store, b->d_items, b->nitems, b->d_args, b->d_maps, 0, 0, b->smem, b->cap);
  cudaError_t e2 = lbk::launch_sweep_batch(b->store, b->d_items, b->nitems, b->d_args, b->d_maps, 1, 1, b->smem, b->cap);
  cudaError_t e3 = cudaStreamEndCapture(b->cap, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return bfail(b, LB_ERR_CUDA, "lb_batch_step: graph capture failed");
  }
  cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, LB_ERR_CUDA, std::string("lb_batch_step: graph instantiation: ") + cudaGetErrorString(e));
  }
  return LB_OK;
}

// Whether every instance's buffers are where the device work list expects.
bool batch_in_sync(const lb_batch *b) {
  if (b->dirty) return false;
  for (size_t i = 0; i < b->hs.size(); i++)
    if (b->hs[i]->cur != (b->par0[i] ^ b->kpar) || b->hs[i]->plan_gen != b->gen[i]) return false;
  return true;
}

}  // namespace

extern "C" {

int lb_batch_create(const lb_params *ps, int32_t count, lb_batch **out) {
  if (!ps || !out || count < 1) return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < count; i++) {
    if (ps[i].stream != ps[0].stream)
      return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: all instances must share one stream");
    if (ps[i].precision != ps[0].precision)
      return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: all instances must share one precision");
    if (ps[i].precision == LB_FP64 || !lbk::sweep_supported(ps[i].precision, ps[i].nx, ps[i].ny))
      return bfail(nullptr, LB_ERR_ARG,
                   "lb_batch_create: every instance must run the sweep kernel (FP32 or 16-bit storage, nx a "
                   "multiple of 4 (8 for 16-bit storage), nx, ny >= 8)");
  }
  lb_batch *b = new (std::nothrow) lb_batch();
  if (!b) return bfail(nullptr, LB_ERR_OOM, "lb_batch_create: host allocation failed");
  b->st = (cudaStream_t)ps[0].stream;
  b->store = ps[0].precision;
  for (int i = 0; i < count; i++) {
    lb_handle *h = nullptr;
    int rc = lb_create(&ps[i], &h);
    if (rc != LB_OK) {
      std::string m = std::string("lb_batch_create: instance ") + std::to_string(i) + ": " + g_create_err;
      lb_batch_destroy(b);
      return bfail(nullptr, rc, m);
    }
    h->in_batch = true;
    b->hs.push_back(h);
  }
  cudaError_t e = lbk::sweep_prepare(b->store, &b->smem);
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_args, 2 * (size_t)count * sizeof(lbk::SweepArgs));
  if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_maps, 4 * (size_t)count * sizeof(CUtensorMap));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::string m = std::string("lb_batch_create: ") + cudaGetErrorString(e);
    lb_batch_destroy(b);
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, m);
  }
  *out = b;
  return LB_OK;
}

lb_handle *lb_batch_handle(lb_batch *b, int32_t i) {
  if (!b || i < 0 || i >= (int)b->hs.size()) return nullptr;
  return b->hs[i];  // changes made through it are detected by lb_batch_step
}

int lb_batch_step(lb_batch *b, int64_t nsteps) {
  if (!b) return LB_ERR_ARG;
  if (nsteps < 0) return bfail(b, LB_ERR_ARG, "lb_batch_step: nsteps < 0");
  for (lb_handle *h : b->hs)
    if (!h->initialised) return bfail(b, LB_ERR_STATE, "lb_batch_step: an instance is not initialised");
  if (nsteps == 0) return LB_OK;
  if (!batch_in_sync(b)) {
    int rc = batch_rebuild(b);
    if (rc != LB_OK) return rc;
  }
  if (nsteps >= 2 && b->persist_cap == 0) {
    int cap = 0;
    const cudaError_t e = lbk::persist_capacity(b->store, b->smem, &cap);
    if (e != cudaSuccess) cudaGetLastError();
    b->persist_cap = (e == cudaSuccess && cap > 0) ? cap : -1;
  }
  if (nsteps >= 2 && b->persist_cap > 0) {
    // Every step in multi-step launches (chunks of at most 2^16 steps).
    const int grid = std::min(b->nitems, b->persist_cap);
    if (!b->d_ticket) LB_BCUDA(b, cudaMalloc((void **)&b->d_ticket, sizeof(unsigned)));
    for (int64_t done = 0; done < nsteps;) {
      const int chunk = (int)std::min<int64_t>(nsteps - done, std::max<int64_t>(1, (1LL << 30) / b->nitems));
      lbk::PersistArgs P{};
      P.nitems = b->nitems;
      P.nsteps = chunk;
      P.kpar0 = b->kpar;
      P.epoch = b->epoch;
      P.done = b->d_done;
      P.dep_ofs = b->d_dep;
      P.dep_idx = b->d_dep + b->nitems + 1;
      P.next = b->d_ticket;
      LB_BCUDA(b, cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned), b->st));
      LB_BCUDA(b, lbk::launch_sweep_batch_persist(b->store, b->d_items, b->d_args, b->d_maps, P, grid, b->smem,
                                                  b->st));
      b->kpar = (b->kpar + chunk) & 1;
      b->epoch += (unsigned)chunk;
      done += chunk;
    }
    for (lb_handle *h : b->hs) {
      h->cur ^= (int)(nsteps & 1);
      h->step += nsteps;
      h->cta_valid = true;
      h->total_valid = false;
    }
    return LB_OK;
  }
  int64_t k = 0;
  if (b->kpar == 1) {  // one plain step to reach kpar 0
    LB_BCUDA(b, lbk::launch_sweep_batch(b->store, b->d_items, b->nitems, b->d_args, b->d_maps, 1, 1, b->smem, b->st));
    b->kpar = 0;
    k = 1;
  }
  if (nsteps - k >= 2) {
    int rc = batch_graph(b);
    if (rc != LB_OK) return rc;
    for (; k + 2 <= nsteps; k += 2) LB_BCUDA(b, cudaGraphLaunch(b->graph, b->st));
  }
  if (k < nsteps) {
    LB_BCUDA(b, lbk::launch_sweep_batch(b->store, b->d_items, b->nitems, b->d_args, b->d_maps, 0, 1, b->smem, b->st));
    b->kpar = 1;
    k++;
  }
  for (lb_handle *h : b->hs) {
    h->cur ^= (int)(nsteps & 1);
    h->step += nsteps;
    h->cta_valid = true;
    h->total_valid = false;
  }
  return LB_OK;
}

int lb_batch_autotune(lb_batch *b, int steps, int32_t *seg_h) {
  if (!b) return LB_ERR_ARG;
  if (steps < 1) return bfail(b, LB_ERR_ARG, "lb_batch_autotune: steps must be >= 1");
  const int n = (int)b->hs.size();
  for (lb_handle *h : b->hs)
    if (!h->initialised) return bfail(b, LB_ERR_STATE, "lb_batch_autotune: an instance is not initialised");
  const int cand[] = {24, 32, 40, 48, 56, 64, 80, 96, 128};
  // Lattice classes by height: short, medium, tall.
  auto cls = [](int ny) { return ny <= 96 ? 0 : (ny <= 160 ? 1 : 2); };
  for (lb_handle *h : b->hs) {
    int mx = h->sweep_nseg;
    for (int c : cand) mx = std::max(mx, (h->p.ny + std::min(c, h->p.ny) - 1) / std::min(c, h->p.ny));
    LB_BCUDA(b, ensure_records(h, mx));
  }
  // Save every state; each trial starts from it.
  std::vector<void *> save(n, nullptr);
  std::vector<int> cur0(n), seg0(n);
  std::vector<int64_t> step0(n);
  int rc = LB_OK;
  cudaError_t e = cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  for (int i = 0; i < n && e == cudaSuccess; i++) {
    lb_handle *h = b->hs[i];
    cur0[i] = h->cur;
    seg0[i] = h->sweep_seg;
    step0[i] = h->step;
    const size_t bytes = lbk::sweep_buffer_bytes(h->store, h->plane);
    e = cudaMalloc(&save[i], bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save[i], h->f[h->cur], bytes, cudaMemcpyDeviceToDevice, b->st);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto restore = [&]() -> cudaError_t {
    for (int i = 0; i < n; i++) {
      lb_handle *h = b->hs[i];
      h->cur = cur0[i];
      h->step = step0[i];
      cudaError_t r = cudaMemcpyAsync(h->f[h->cur], save[i], lbk::sweep_buffer_bytes(h->store, h->plane),
                                      cudaMemcpyDeviceToDevice, b->st);
      if (r != cudaSuccess) return r;
    }
    b->dirty = true;
    return cudaSuccess;
  };
  auto trial = [&](float *ms) -> int {
    b->dirty = true;
    int r = lb_batch_step(b, 2);
    if (r == LB_OK) e = cudaEventRecord(e0, b->st);
    if (r == LB_OK && e == cudaSuccess) r = lb_batch_step(b, steps);
    if (r == LB_OK && e == cudaSuccess) e = cudaEventRecord(e1, b->st);
    if (r == LB_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (r == LB_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (r == LB_OK && e == cudaSuccess) e = restore();
    return r;
  };
  // Pass 1: one segment height for all; pass 2: per class, others fixed.
  int best_all = 64;
  float best_ms = 3.0e38f;
  for (int c : cand) {
    if (e != cudaSuccess || rc != LB_OK) break;
    for (lb_handle *h : b->hs) set_segments(h, c);
    float ms = 0.f;
    rc = trial(&ms);
    if (rc == LB_OK && e == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best_all = c;
    }
  }
  int best_cls[3] = {best_all, best_all, best_all};
  for (int k = 0; k < 3; k++) {
    bool any = false;
    for (lb_handle *h : b->hs) any = any || cls(h->p.ny) == k;
    if (!any) continue;
    for (int c : cand) {
      if (e != cudaSuccess || rc != LB_OK) break;
      if (c == best_cls[k]) continue;
      for (lb_handle *h : b->hs) set_segments(h, cls(h->p.ny) == k ? c : best_cls[cls(h->p.ny)]);
      float ms = 0.f;
      rc = trial(&ms);
      if (rc == LB_OK && e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best_cls[k] = c;
      }
    }
  }
  for (int i = 0; i < n; i++) {
    lb_handle *h = b->hs[i];
    set_segments(h, (rc == LB_OK && e == cudaSuccess) ? best_cls[cls(h->p.ny)] : seg0[i]);
    if (seg_h) seg_h[i] = h->sweep_seg;
  }
  if (e == cudaSuccess) e = restore();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  for (void *p : save) cudaFree(p);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->dirty = true;
  if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_autotune: ") + cudaGetErrorString(e));
  if (rc != LB_OK) return bfail(b, rc, "lb_batch_autotune: a trial step failed: " + b->err);
  return LB_OK;
}

int lb_batch_destroy(lb_batch *b) {
  if (!b) return LB_OK;
  if (b->st || !b->hs.empty()) cudaStreamSynchronize(b->st);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (lb_handle *h : b->hs) lb_destroy(h);
  cudaFree(b->d_items);
  cudaFree(b->d_args);
  cudaFree(b->d_maps);
  cudaFree(b->d_done);
  cudaFree(b->d_dep);
  cudaFree(b->d_ticket);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return LB_OK;
}

const char *lb_batch_last_error(const lb_batch *b) {
  if (!b) return g_create_err.c_str();
  return b->err.c_str();
}

}  // extern "C"
