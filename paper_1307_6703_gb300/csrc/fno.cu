// fno.cu -- the learned warm start (include/fno.h): forward and backward
// passes of a small Fourier neural operator, its loss and its Adam update,
// as CUDA kernels of this library.  The truncated Fourier transforms along x
// and the per-site channel mixing are matrix products: in BF16 mode they run
// on the tensor cores through this library's tcgen05 product (gemm_tc.cu:
// BF16 operands with the contracted index contiguous, FP32 accumulation),
// in FP32 mode through its SIMT product; the transforms along y, the
// per-mode complex channel mixing, the lift, the projection, the
// activations, the loss, every reduction of the backward pass and the
// optimizer are the kernels below.  The tensor-core product contracts over
// the contiguous index of both operands, so the kernels that write BF16
// copies also keep, where a product contracts over channels, a site-major
// copy ([b][site][channel]), and the weights and DFT tables have transposed
// BF16 copies.
//
// Activation layout: [batch][channel][ny][nx] (x fastest).  A "row" of the
// x-transform is one (batch, channel, y) line, so the x-transform of all
// channels of all fields is a single GEMM [B*C*ny, nx] x [nx, 2*mx].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fno.h"
#include "gemm_tc.h"

namespace {

constexpr int kMaxLayers = 8;
constexpr int kFeatures = 5;
constexpr int kThreads = 256;

struct Offsets {
  size_t P, p, W[kMaxLayers], w[kMaxLayers], Rr[kMaxLayers], Ri[kMaxLayers], Q1, q1, Q2, q2, total;
};

Offsets make_offsets(const fno_config &c) {
  Offsets o{};
  size_t at = 0;
  const size_t C = c.width, H = c.hidden, M = (size_t)c.modes_x * c.modes_y;
  o.P = at; at += C * kFeatures;
  o.p = at; at += C;
  for (int l = 0; l < c.layers; l++) {
    o.W[l] = at; at += C * C;
    o.w[l] = at; at += C;
    o.Rr[l] = at; at += M * C * C;
    o.Ri[l] = at; at += M * C * C;
  }
  o.Q1 = at; at += H * C;
  o.q1 = at; at += H;
  o.Q2 = at; at += (size_t)c.outputs * H;
  o.q2 = at; at += c.outputs;
  o.total = at;
  return o;
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float gelu(float z) { return z * normcdff(z); }
__device__ __forceinline__ float gelu_grad(float z) {
  return normcdff(z) + z * (0.3989422804014327f * expf(-0.5f * z * z));
}

// Kept y-mode number of mode index k (0..my-1): 0..my/2-1, then -my/2..-1.
__device__ __forceinline__ int ymode(int k, int my) { return k < my / 2 ? k : k - my; }

// Deterministic block sum of one double per thread (blockDim = kThreads).
__device__ double block_sum(double v, double *sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

unsigned blocks_for(long long n) { return (unsigned)std::min<long long>((n + kThreads - 1) / kThreads, 8192); }

// 2D grid: y = rows (one per field and channel), x = enough blocks for S sites
// with a total of about 8192 blocks.
dim3 grid2(long long S, int rows) {
  const long long per_row = std::max<long long>(1, 8192 / std::max(rows, 1));
  return dim3((unsigned)std::min<long long>((S + kThreads - 1) / kThreads, per_row), (unsigned)rows);
}

// ------------------------------------------------------------------ kernels

// Input features of each field from its parameters (U_w, A0, lambda, T_r).
__global__ void features_kernel(const float *__restrict__ prm, int B, int nx, int ny, float *__restrict__ x0) {
  const long long S = (long long)nx * ny, total = (long long)B * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / S);
    const long long s = i - (long long)b * S;
    const int y = (int)(s / nx), x = (int)(s - (long long)y * nx);
    const float uw = prm[4 * b], a0 = prm[4 * b + 1], lam = prm[4 * b + 2], tr = prm[4 * b + 3];
    float sn, cs;
    sincospif(2.0f * (float)x / lam, &sn, &cs);
    const float yy = 2.0f * (float)y / (float)(ny - 1) - 1.0f;
    float *o = x0 + (long long)b * kFeatures * S + s;
    o[0] = (a0 / 1e-3f) * sn;
    o[S] = (a0 / 1e-3f) * cs;
    o[2 * S] = (uw / 0.05f) * yy;
    o[3 * S] = (tr - 0.94f) / 0.02f;
    o[4 * S] = yy;
  }
}

// Elementwise kernels run on 2D grids: y = one (field, channel) row of S
// sites, x = sites, so no per-element index division is needed.
// v0[b, o, s] = sum_c P[o, c] x0[b, c, s] + p[o]
__global__ void lift_kernel(const float *__restrict__ x0, const float *__restrict__ P, const float *__restrict__ pb,
                            int C, long long S, float *__restrict__ v, __nv_bfloat16 *__restrict__ vb) {
  const int row = blockIdx.y, b = row / C, o = row - b * C;
  const float *xb = x0 + (long long)b * kFeatures * S;
  float *vr = v + (long long)row * S;
  __nv_bfloat16 *vbr = vb + (long long)row * S;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
    float acc = pb[o];
#pragma unroll
    for (int c = 0; c < kFeatures; c++) acc += P[o * kFeatures + c] * xb[c * S + s];
    vr[s] = acc;
    vbr[s] = __float2bfloat16_rn(acc);
  }
}

// Spectral kernels.  Rows of the x-transformed lines hold the mx kept
// modes as (real parts, then imaginary parts): X[bc][y][j], j < mx real and
// j >= mx imaginary part of mode j - mx; mode sets are [bc][ky][kx][2].
// Ty[ky][y] = (cos theta, sin theta) with theta = 2 pi ky' y / ny.  Rows are
// processed in chunks of kYChunk staged in shared memory with the chunk's
// twiddles; sums run over y in order.
constexpr int kYChunk = 64;

// y-transform: S[bc][ky][kx] = sum_y (X_r + i X_i)[y][kx] e^{-i theta}.
// One block per line set bc; dynamic shared memory (kYChunk (2 mx + 2 my))
// floats.
__global__ void __launch_bounds__(kThreads)
ydft_kernel(const float *__restrict__ A, const float2 *__restrict__ Ty, int ny, int mx, int my,
            float *__restrict__ Sh) {
  extern __shared__ float ysm[];
  float *xs = ysm;                                              // [kYChunk][2 mx]
  float2 *ts = reinterpret_cast<float2 *>(ysm + kYChunk * 2 * mx);  // [my][kYChunk]
  const int bc = blockIdx.x, t = threadIdx.x, M = my * mx;
  const float *a = A + (long long)bc * ny * 2 * mx;
  float sr[2] = {0.f, 0.f}, si[2] = {0.f, 0.f};  // outputs t and t + kThreads
  for (int y0 = 0; y0 < ny; y0 += kYChunk) {
    const int yc = min(kYChunk, ny - y0);
    __syncthreads();
    for (int e = t; e < yc * 2 * mx; e += kThreads) xs[e] = a[(long long)y0 * 2 * mx + e];
    for (int e = t; e < my * yc; e += kThreads) {
      const int k = e / yc, y = e - k * yc;
      ts[k * kYChunk + y] = Ty[k * ny + y0 + y];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int o = t + q * kThreads;
      if (o < M) {
        const int k = o / mx, kx = o - k * mx;
        float r = sr[q], im = si[q];
        for (int y = 0; y < yc; y++) {
          const float2 tw = ts[k * kYChunk + y];
          const float ar = xs[y * 2 * mx + kx], ai = xs[y * 2 * mx + mx + kx];
          r += ar * tw.x + ai * tw.y;
          im += ai * tw.x - ar * tw.y;
        }
        sr[q] = r;
        si[q] = im;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int o = t + q * kThreads;
    if (o < M) {
      float *d = Sh + ((long long)bc * M + o) * 2;
      d[0] = sr[q];
      d[1] = si[q];
    }
  }
}

// Inverse y-transform (and the adjoint of the y-transform, which has the
// same form): X[bc][y][kx] = sum_ky Y[bc][ky][kx] e^{+i theta}, written as
// (real, imaginary) rows with a BF16 copy.  One block per line set;
// dynamic shared memory (2 my mx + 2 my kYChunk) floats.
__global__ void __launch_bounds__(kThreads)
iy_kernel(const float *__restrict__ Y, const float2 *__restrict__ Ty, int ny, int mx, int my, float *__restrict__ X,
          __nv_bfloat16 *__restrict__ Xb) {
  extern __shared__ float ysm[];
  float *ys = ysm;                                              // [my][mx][2]
  float2 *ts = reinterpret_cast<float2 *>(ysm + 2 * my * mx);   // [my][kYChunk]
  const int bc = blockIdx.x, t = threadIdx.x;
  for (int e = t; e < 2 * my * mx; e += kThreads) ys[e] = Y[(long long)bc * 2 * my * mx + e];
  for (int y0 = 0; y0 < ny; y0 += kYChunk) {
    const int yc = min(kYChunk, ny - y0);
    __syncthreads();
    for (int e = t; e < my * yc; e += kThreads) {
      const int k = e / yc, y = e - k * yc;
      ts[k * kYChunk + y] = Ty[k * ny + y0 + y];
    }
    __syncthreads();
    for (int e = t; e < yc * mx; e += kThreads) {
      const int y = e / mx, kx = e - y * mx;
      float gr = 0.f, gi = 0.f;
      for (int k = 0; k < my; k++) {
        const float2 tw = ts[k * kYChunk + y];
        const float yr = ys[(k * mx + kx) * 2], yi = ys[(k * mx + kx) * 2 + 1];
        gr += yr * tw.x - yi * tw.y;
        gi += yr * tw.y + yi * tw.x;
      }
      const long long g = ((long long)bc * ny + y0 + y) * 2 * mx;
      X[g + kx] = gr;
      X[g + mx + kx] = gi;
      Xb[g + kx] = __float2bfloat16_rn(gr);
      Xb[g + mx + kx] = __float2bfloat16_rn(gi);
    }
  }
}

// Per-mode complex channel mixing: Y[b][o][m] = sum_c S[b][c][m] R[m][c][o]
// (m = ky mx + kx; R as real and imaginary planes [m][c][o]).  One block per
// mode; dynamic shared memory (2 B C + 2 C C) floats.
__global__ void __launch_bounds__(kThreads)
mix_kernel(const float *__restrict__ Sh, const float *__restrict__ Rr, const float *__restrict__ Ri, int B, int C,
           int M, float *__restrict__ Y) {
  extern __shared__ float msm[];
  float2 *ss = reinterpret_cast<float2 *>(msm);          // [B][C]
  float2 *rs = reinterpret_cast<float2 *>(msm + 2 * B * C);  // [C][C]
  const int m = blockIdx.x, t = threadIdx.x;
  const float2 *S2 = reinterpret_cast<const float2 *>(Sh);
  for (int e = t; e < B * C; e += kThreads) ss[e] = S2[(long long)e * M + m];
  for (int e = t; e < C * C; e += kThreads)
    rs[e] = make_float2(Rr[(long long)m * C * C + e], Ri[(long long)m * C * C + e]);
  __syncthreads();
  float2 *Y2 = reinterpret_cast<float2 *>(Y);
  for (int e = t; e < B * C; e += kThreads) {
    const int b = e / C, o = e - b * C;
    float yr = 0.f, yi = 0.f;
    for (int c = 0; c < C; c++) {
      const float2 sv = ss[b * C + c], rv = rs[c * C + o];
      yr += sv.x * rv.x - sv.y * rv.y;
      yi += sv.x * rv.y + sv.y * rv.x;
    }
    Y2[(long long)e * M + m] = make_float2(yr, yi);
  }
}

// z += w (per channel); v' = gelu(z) (or z for the last layer).
__global__ void bias_act_kernel(float *__restrict__ z, const float *__restrict__ w, int C, long long S, int act,
                                float *__restrict__ v, __nv_bfloat16 *__restrict__ vb) {
  const int row = blockIdx.y, o = row % C;
  const float wo = w[o];
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
    const long long i = (long long)row * S + s;
    const float zz = z[i] + wo;
    z[i] = zz;
    const float vv = act ? gelu(zz) : zz;
    v[i] = vv;
    vb[i] = __float2bfloat16_rn(vv);
  }
}

constexpr int kMaxOutputs = 4;

// hp += q1 (kept); out[b, j, s] = sum_h Q2[j, h] gelu(hp[b, h, s]) + q2[j].
__global__ void project_kernel(float *__restrict__ hp, const float *__restrict__ q1, const float *__restrict__ Q2,
                               const float *__restrict__ q2, int H, int O, long long S, float *__restrict__ out,
                               float *__restrict__ out_user) {
  const int b = blockIdx.y;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
    float *h = hp + (long long)b * H * S + s;
    float acc[kMaxOutputs];
#pragma unroll
    for (int j = 0; j < kMaxOutputs; j++) acc[j] = j < O ? q2[j] : 0.f;
    for (int k = 0; k < H; k++) {
      const float z = h[k * S] + q1[k];
      h[k * S] = z;
      const float a = gelu(z);
#pragma unroll
      for (int j = 0; j < kMaxOutputs; j++)
        if (j < O) acc[j] += Q2[j * H + k] * a;
    }
    for (int j = 0; j < O; j++) {
      const long long e = ((long long)b * O + j) * S + s;
      out[e] = acc[j];
      if (out_user) out_user[e] = acc[j];
    }
  }
}

// Loss partial sums and d loss / d out = 2 (out - target) / (B S).
__global__ void loss_kernel(const float *__restrict__ out, const float *__restrict__ tgt, long long total,
                            float *__restrict__ dout, double *__restrict__ partial) {
  __shared__ double sm[kThreads];
  double acc = 0.0;
  const float scale = 2.0f / (float)total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float d = out[i] - tgt[i];
    dout[i] = scale * d;
    acc += (double)d * (double)d;
  }
  const double r = block_sum(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void finish_loss_kernel(const double *__restrict__ partial, int n, long long total, double *__restrict__ loss) {
  __shared__ double sm[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double r = block_sum(acc, sm);
  if (threadIdx.x == 0) *loss = r / (double)total;
}

// Initial fields of the solver from the network output (fno_fields):
// per field b, block j: FP64 sum of the density d = 1 + s0 o0 over the
// block's sites (grid-strided, then the fixed-order block tree).
__global__ void field_mass_kernel(const float *__restrict__ out, int outputs, long long S, double s0,
                                  double *__restrict__ part) {
  __shared__ double sm[kThreads];
  const float *o = out + (size_t)blockIdx.y * outputs * S;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < S; e += (long long)gridDim.x * blockDim.x)
    acc += __dadd_rn(__dmul_rn(s0, (double)o[e]), 1.0);
  const double r = block_sum(acc, sm);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = r;
}

// fields[b] = (d + (rho_mean - mean d), s1 o1, s2 o2); the mean from the
// nblk block sums of field b in a fixed order.
__global__ void fields_kernel(const float *__restrict__ out, int outputs, long long S, double s0, double s1,
                              double s2, double rho_mean, const double *__restrict__ part, int nblk,
                              double *__restrict__ fields) {
  __shared__ double shift;
  const int b = blockIdx.y;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int j = 0; j < nblk; ++j) m += part[(size_t)b * nblk + j];
    shift = rho_mean - m / (double)S;
  }
  __syncthreads();
  const float *o = out + (size_t)b * outputs * S;
  double *f = fields + (size_t)b * 3 * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < S; e += (long long)gridDim.x * blockDim.x) {
    f[e] = __dadd_rn(__dadd_rn(__dmul_rn(s0, (double)o[e]), 1.0), shift);
    f[S + e] = __dmul_rn(s1, (double)o[S + e]);
    f[2 * S + e] = __dmul_rn(s2, (double)o[2 * S + e]);
  }
}

// dhp[b, h, s] = sum_j Q2[j, h] dout[b, j, s] gelu'(hp[b, h, s])
__global__ void project_back_kernel(const float *__restrict__ hp, const float *__restrict__ Q2,
                                    const float *__restrict__ dout, int H, int O, long long S,
                                    float *__restrict__ dhp, __nv_bfloat16 *__restrict__ dhpb) {
  const int row = blockIdx.y, b = row / H, k = row - b * H;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
    const long long i = (long long)row * S + s;
    float acc = 0.f;
    for (int j = 0; j < O; j++) acc += Q2[j * H + k] * dout[((long long)b * O + j) * S + s];
    const float d = acc * gelu_grad(hp[i]);
    dhp[i] = d;
    dhpb[i] = __float2bfloat16_rn(d);
  }
}

// Two-pass per-channel sums over (b, s), deterministic: pass 1 gives each
// of nb blocks per channel a contiguous share of sum a[b, ch, s] (a has C
// channels; FP32 per thread and in the warp trees, the warps' sums added in
// FP64 in order), pass 2 adds the nb partials of a channel in order.
constexpr int kReduceBlocks = 32;
constexpr int kOuterBlocks = 64;  // site shares of outer_pass1_kernel
__global__ void reduce_pass1_kernel(const float *__restrict__ a, int B, int C, long long S, double *__restrict__ part) {
  __shared__ double ws[kThreads / 32];
  const int ch = blockIdx.x, blk = blockIdx.y;
  const long long n = (long long)B * S, per = (n + gridDim.y - 1) / gridDim.y;
  const long long lo = blk * per, hi = min(n, lo + per);
  float acc = 0.f;
  long long i = lo + threadIdx.x;
  int b = (int)(i / S);
  long long s = i - (long long)b * S;
  for (; i < hi; i += blockDim.x) {
    while (s >= S) {  // advance (b, s) without dividing
      s -= S;
      b++;
    }
    acc += a[((long long)b * C + ch) * S + s];
    s += blockDim.x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; w++) r += ws[w];
    part[(long long)ch * gridDim.y + blk] = r;
  }
}

// Weight gradients that are per-site outer products, pass 1 without
// re-reading the operands per channel pair: block (x, y) takes x's contiguous share of the
// (b, s) sites and tile y of NA x NB channel pairs (ca, cb); each thread
// keeps the tile's NA*NB sums of a[b, ca, s] f(o2[b, cb, s]) in FP32 (f =
// gelu or identity, evaluated once per (cb, site) of the tile), then the
// block adds them in a fixed order -- FP32 warp trees (FP64 throughput is
// low on this part), the warps' sums in FP64 -- into
// part[(ca * Cb + cb) * gridDim.x + x], the layout of pass 2.
template <int NA, int NB, bool kGelu>
__global__ void __launch_bounds__(kThreads)
outer_pass1_kernel(const float *__restrict__ a, const float *__restrict__ o2, int B, int Ca, int Cb, long long S,
                   double *__restrict__ part) {
  __shared__ double sm[kThreads / 32][NA * NB];
  const int ntb = (Cb + NB - 1) / NB;
  const int ca0 = (blockIdx.y / ntb) * NA, cb0 = (blockIdx.y % ntb) * NB;
  float acc[NA][NB];
#pragma unroll
  for (int i = 0; i < NA; i++)
#pragma unroll
    for (int j = 0; j < NB; j++) acc[i][j] = 0.f;
  const long long n = (long long)B * S, per = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(n, lo + per);
  long long e = lo + threadIdx.x;
  long long b = e / S, s = e - b * S;  // then advanced without dividing
  for (; e < hi; e += blockDim.x, s += blockDim.x) {
    while (s >= S) {
      s -= S;
      b++;
    }
    float av[NA], bv[NB];
#pragma unroll
    for (int i = 0; i < NA; i++) av[i] = ca0 + i < Ca ? a[(b * Ca + ca0 + i) * S + s] : 0.f;
#pragma unroll
    for (int j = 0; j < NB; j++) {
      const float v = cb0 + j < Cb ? o2[(b * Cb + cb0 + j) * S + s] : 0.f;
      bv[j] = kGelu ? gelu(v) : v;
    }
#pragma unroll
    for (int i = 0; i < NA; i++)
#pragma unroll
      for (int j = 0; j < NB; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NA; i++)
#pragma unroll
    for (int j = 0; j < NB; j++) {
      float v = acc[i][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sm[w][i * NB + j] = (double)v;
    }
  __syncthreads();
  for (int p = threadIdx.x; p < NA * NB; p += blockDim.x) {
    const int i = p / NB, j = p % NB;
    if (ca0 + i >= Ca || cb0 + j >= Cb) continue;
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; k++) t += sm[k][p];
    part[((long long)(ca0 + i) * Cb + cb0 + j) * gridDim.x + blockIdx.x] = t;
  }
}

// Pass 1 of the channel sums when S % 4 == 0: block (ch, b * nsplit + j)
// sums float4s j * 256 + t, (j + nsplit) * 256 + t, ... of field b's channel
// ch, two at a time into two FP32 partials (then a fixed-order warp and
// block tree, FP64 across warps); part[ch][b * nsplit + j].
__global__ void __launch_bounds__(kThreads)
reduce_pass1_v4_kernel(const float *__restrict__ a, int C, long long S, int nsplit, double *__restrict__ part) {
  __shared__ double ws[kThreads / 32];
  const int ch = blockIdx.x, b = blockIdx.y / nsplit, j = blockIdx.y % nsplit;
  const float4 *p = reinterpret_cast<const float4 *>(a + ((long long)b * C + ch) * S);
  const long long S4 = S / 4, step = (long long)nsplit * blockDim.x;
  float acc0 = 0.f, acc1 = 0.f;
  long long i = (long long)j * blockDim.x + threadIdx.x;
  for (; i + step < S4; i += 2 * step) {
    const float4 u = p[i], v = p[i + step];
    acc0 += (u.x + u.y) + (u.z + u.w);
    acc1 += (v.x + v.y) + (v.z + v.w);
  }
  if (i < S4) {
    const float4 u = p[i];
    acc0 += (u.x + u.y) + (u.z + u.w);
  }
  float acc = acc0 + acc1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; w++) r += ws[w];
    part[(long long)ch * gridDim.y + blockIdx.y] = r;
  }
}

// Pass 2: one warp per output; lane l adds partials l, l + 32, ... in order,
// then a fixed-order shuffle tree.
__global__ void __launch_bounds__(kThreads)
reduce_pass2_kernel(const double *__restrict__ part, int nch, int nb, float *__restrict__ out) {
  const int ch = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (ch >= nch) return;
  double acc = 0.0;
  for (int i = lane; i < nb; i += 32) acc += part[(long long)ch * nb + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[ch] = (float)acc;
}

// out[i] = sum_b part[b][i] (weight gradients of the per-field GEMMs):
// block k takes outputs 32k .. 32k + 31; its eight warps sum the parts
// w, w + 8, ... in order, then warp 0 adds the eight partials in order.
__global__ void __launch_bounds__(kThreads)
sum_fields_kernel(const float *__restrict__ part, int B, int n, float *__restrict__ out) {
  __shared__ float ws[kThreads / 32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float acc = 0.f;
  if (i < n) {
    for (int b = w; b < B; b += kThreads / 32) acc += part[(long long)b * n + i];
  }
  ws[w][lane] = acc;
  __syncthreads();
  if (w == 0 && i < n) {
    float r = ws[0][lane];
#pragma unroll
    for (int q = 1; q < kThreads / 32; q++) r += ws[q][lane];
    out[i] = r;
  }
}

// dz = dv * gelu'(z) (or dv for the last layer), with a BF16 copy.
__global__ void act_back_kernel(const float *__restrict__ dv, const float *__restrict__ z, long long total, int act,
                                float *__restrict__ dz, __nv_bfloat16 *__restrict__ dzb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float d = act ? dv[i] * gelu_grad(z[i]) : dv[i];
    dz[i] = d;
    dzb[i] = __float2bfloat16_rn(d);
  }
}

// Adjoint of the mode mixing and the spectral weights' gradient, per mode m:
// dS[b][c][m] = sum_o dY[b][o][m] conj(R[m][c][o]) and
// dR[m][c][o] = sum_b conj(S[b][c][m]) dY[b][o][m] (real and imaginary
// planes).  One block per mode; dynamic shared memory (4 B C + 2 C C) floats.
__global__ void __launch_bounds__(kThreads)
mix_back_kernel(const float *__restrict__ dY, const float *__restrict__ Sh, const float *__restrict__ Rr,
                const float *__restrict__ Ri, int B, int C, int M, float *__restrict__ dS, float *__restrict__ dRr,
                float *__restrict__ dRi) {
  extern __shared__ float msm[];
  float2 *ds = reinterpret_cast<float2 *>(msm);               // dY [B][C]
  float2 *ss = reinterpret_cast<float2 *>(msm + 2 * B * C);   // S [B][C]
  float2 *rs = reinterpret_cast<float2 *>(msm + 4 * B * C);   // R [C][C]
  const int m = blockIdx.x, t = threadIdx.x;
  const float2 *D2 = reinterpret_cast<const float2 *>(dY), *S2 = reinterpret_cast<const float2 *>(Sh);
  for (int e = t; e < B * C; e += kThreads) {
    ds[e] = D2[(long long)e * M + m];
    ss[e] = S2[(long long)e * M + m];
  }
  for (int e = t; e < C * C; e += kThreads)
    rs[e] = make_float2(Rr[(long long)m * C * C + e], Ri[(long long)m * C * C + e]);
  __syncthreads();
  float2 *dS2 = reinterpret_cast<float2 *>(dS);
  for (int e = t; e < B * C; e += kThreads) {
    const int b = e / C, c = e - b * C;
    float sr = 0.f, si = 0.f;
    for (int o = 0; o < C; o++) {
      const float2 yv = ds[b * C + o], rv = rs[c * C + o];
      sr += yv.x * rv.x + yv.y * rv.y;
      si += -yv.x * rv.y + yv.y * rv.x;
    }
    dS2[(long long)e * M + m] = make_float2(sr, si);
  }
  for (int e = t; e < C * C; e += kThreads) {
    const int c = e / C, o = e - c * C;
    float ar = 0.f, ai = 0.f;
    for (int b = 0; b < B; b++) {
      const float2 sv = ss[b * C + c], dv = ds[b * C + o];
      ar += sv.x * dv.x + sv.y * dv.y;
      ai += -sv.y * dv.x + sv.x * dv.y;
    }
    dRr[(long long)m * C * C + e] = ar;
    dRi[(long long)m * C * C + e] = ai;
  }
}

// Truncated DFT matrices for nx: Fx[x][j] (forward, e^{-i phi}) and
// Fxi[j][x] (real inverse with c_kx and 1/(nx ny)).
__global__ void dft_tables_kernel(int nx, int ny, int mx, int my, float *Fx, float *Fxi, __nv_bfloat16 *Fxb,
                                  __nv_bfloat16 *Fxib, __nv_bfloat16 *FxTb, __nv_bfloat16 *FxiTb, float2 *Ty) {
  // y twiddles: Ty[k][y] = (cos, sin)(2 pi ky y / ny), argument reduced mod ny
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < my * ny; i += gridDim.x * blockDim.x) {
    const int k = i / ny, y = i - k * ny;
    const int r = ((ymode(k, my) * y) % ny + ny) % ny;
    float sn, cs;
    sincospif(2.0f * (float)r / (float)ny, &sn, &cs);
    Ty[i] = make_float2(cs, sn);
  }
  const int n = nx * mx;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int x = i / mx, k = i - x * mx;
    float sn, cs;
    sincospif(2.0f * (float)((long long)k * x % nx) / (float)nx, &sn, &cs);
    Fx[x * 2 * mx + k] = cs;
    Fx[x * 2 * mx + mx + k] = -sn;
    const float sc = (k == 0 ? 1.0f : 2.0f) / ((float)nx * (float)ny);
    Fxi[k * nx + x] = sc * cs;
    Fxi[(mx + k) * nx + x] = -sc * sn;
    Fxb[x * 2 * mx + k] = __float2bfloat16_rn(cs);
    Fxb[x * 2 * mx + mx + k] = __float2bfloat16_rn(-sn);
    Fxib[k * nx + x] = __float2bfloat16_rn(sc * cs);
    Fxib[(mx + k) * nx + x] = __float2bfloat16_rn(-sc * sn);
    // transposed copies: FxT[j][x] = Fx[x][j], FxiT[x][j] = Fxi[j][x]
    FxTb[k * nx + x] = __float2bfloat16_rn(cs);
    FxTb[(mx + k) * nx + x] = __float2bfloat16_rn(-sn);
    FxiTb[x * 2 * mx + k] = __float2bfloat16_rn(sc * cs);
    FxiTb[x * 2 * mx + mx + k] = __float2bfloat16_rn(-sc * sn);
  }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16 *__restrict__ pb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

// out[b][c][r] = in[b][r][c] for batch b (R x Cc BF16 matrices, R and Cc
// even), through 32 x 64 shared-memory tiles; both sides move bf16 pairs,
// so a warp reads 128 contiguous bytes of a row of `in` and writes 128
// contiguous bytes of `out` (two rows of 32 when R = 32).
__global__ void __launch_bounds__(256)
transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, long long R, long long Cc,
                      __nv_bfloat16 *__restrict__ out) {
  __shared__ __nv_bfloat16 tile[32][64 + 2];
  const long long r0 = (long long)blockIdx.x * 32, c0 = (long long)blockIdx.y * 64;
  const int b = blockIdx.z;
  in += (long long)b * R * Cc;
  out += (long long)b * R * Cc;
  for (int i = threadIdx.x; i < 32 * 32; i += blockDim.x) {
    const int rr = i / 32, cp = i % 32;
    const long long r = r0 + rr, c = c0 + 2 * cp;
    if (r < R && c < Cc) {
      const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(in + r * Cc + c);
      tile[rr][2 * cp] = v.x;
      tile[rr][2 * cp + 1] = v.y;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) {
    const int cc = i / 16, rp = i % 16;
    const long long c = c0 + cc, r = r0 + 2 * rp;
    if (c < Cc && r < R) {
      __nv_bfloat162 v;
      v.x = tile[2 * rp][cc];
      v.y = tile[2 * rp + 1][cc];
      *reinterpret_cast<__nv_bfloat162 *>(out + c * R + r) = v;
    }
  }
}

// The same transpose with 16-byte accesses, for R % 32 == 0 and S % 8 == 0:
// block (i, j, b) moves rows 32i .. 32i + 31 by sites 64j .. 64j + 63; each
// thread reads eight sites of one row and writes eight rows of one site.
__global__ void __launch_bounds__(256)
transpose_bf16_v8_kernel(const __nv_bfloat16 *__restrict__ in, long long R, long long S,
                         __nv_bfloat16 *__restrict__ out) {
  __shared__ __align__(16) __nv_bfloat16 tile[32][64 + 8];
  const long long r0 = (long long)blockIdx.x * 32, s0 = (long long)blockIdx.y * 64;
  const int b = blockIdx.z, t = threadIdx.x;
  in += (long long)b * R * S;
  out += (long long)b * R * S;
  {
    const int rr = t >> 3, sc = (t & 7) * 8;
    if (s0 + sc < S)
      *reinterpret_cast<uint4 *>(&tile[rr][sc]) = *reinterpret_cast<const uint4 *>(in + (r0 + rr) * S + s0 + sc);
  }
  __syncthreads();
  {
    const int ss = t >> 2, rc = (t & 3) * 8;
    if (s0 + ss < S) {
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = tile[rc + q][ss];
      *reinterpret_cast<uint4 *>(out + (s0 + ss) * R + r0 + rc) = *reinterpret_cast<const uint4 *>(v);
    }
  }
}

// Transposed BF16 weights for the tensor-core products: WT_l[c][o] =
// W_l[o][c] (layer l at l C C), then Q1T[c][h] = Q1[h][c].
__global__ void weights_t_kernel(const __nv_bfloat16 *__restrict__ prmb, Offsets o, int C, int H, int L,
                                 __nv_bfloat16 *__restrict__ wt) {
  const int n = L * C * C + C * H;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < L * C * C) {
      const int l = i / (C * C), r = i - l * C * C, c = r / C, oo = r - c * C;
      wt[i] = prmb[o.W[l] + (size_t)oo * C + c];
    } else {
      const int r = i - L * C * C, c = r / H, hh = r - c * H;
      wt[i] = prmb[o.Q1 + (size_t)hh * C + c];
    }
  }
}

__global__ void to_bf16_kernel(const float *__restrict__ a, long long n, __nv_bfloat16 *__restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace

// ------------------------------------------------------------------ handle

struct fno_handle {
  fno_config c{};
  cudaStream_t st = nullptr;
  Offsets o{};
  float *prm = nullptr, *grd = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16 *prmb = nullptr;
  long long cap_bcs = 0, cap_bs = 0, cap_bhs = 0, cap_line = 0, cap_modes = 0;  // workspace sizes (elements)
  float *x0 = nullptr, *V[kMaxLayers + 1] = {}, *Z[kMaxLayers] = {}, *Sh[kMaxLayers] = {};
  __nv_bfloat16 *Vb[kMaxLayers + 1] = {};
  float *A = nullptr, *G = nullptr, *hp = nullptr, *out = nullptr;
  __nv_bfloat16 *Gb = nullptr;
  float *dout = nullptr, *dhp = nullptr, *dV = nullptr, *dZ = nullptr, *dG = nullptr, *dA = nullptr, *dY = nullptr,
        *dS = nullptr;
  __nv_bfloat16 *dhpb = nullptr, *dZb = nullptr, *dAb = nullptr;
  double *partial = nullptr, *loss = nullptr, *rpart = nullptr;
  int rpart_fields = 0;  // FP64 partials per channel that rpart holds
  float *wpart = nullptr;  // per-field weight gradients [B][max(C, H) * C]
  float *Fx = nullptr, *Fxi = nullptr;
  __nv_bfloat16 *Fxb = nullptr, *Fxib = nullptr, *FxTb = nullptr, *FxiTb = nullptr;
  // site-major BF16 copies ([b][site][channel]) for the products that
  // contract over channels; transposed BF16 weights (W_l^T per layer, Q1^T)
  __nv_bfloat16 *VbT[kMaxLayers + 1] = {}, *dZT = nullptr, *dhpT = nullptr, *wTb = nullptr;
  int *gerr = nullptr;  // set by a tensor-core product whose bounded wait gave up
  float2 *Ty = nullptr;
  int tab_nx = 0, tab_ny = 0;
  int B = 0, nx = 0, ny = 0;  // shape of the last forward pass
  bool have_forward = false;
  std::string err;
};

namespace {

thread_local std::string g_err;

int ffail(fno_handle *h, int code, const std::string &m) {
  if (h) h->err = m;
  else g_err = m;
  return code;
}

#define FNO_CUDA(h, call)                                                                                      \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess)                                                                                     \
      return ffail(h, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,                              \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                        \
  } while (0)

#define FNO_GEMM(h, call)                                                                                      \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess) return ffail(h, LB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

// K-split of the weight-gradient products (K = sites): the split partial
// products land in separate slices of wpart, summed with the fields.
constexpr int kWSplit = 8;

// Tensor-core product (BF16 mode): C(m, n) = sum_k X(m, k) Y(n, k), see
// gemm_tc.h for the argument layout.
cudaError_t tcg(fno_handle *h, const __nv_bfloat16 *X, int ldx, long long sX, const __nv_bfloat16 *Y, int ldy,
                long long sY, float *C, long long cm, long long cn, long long sC, int M, int N, int K, int batch,
                int ksplit, float beta) {
  return tc::gemm_tn_bf16(X, ldx, sX, Y, ldy, sY, C, cm, cn, sC, M, N, K, batch, ksplit, beta, h->gerr, h->st);
}

// SIMT product (FP32 mode): C(m, n) = sum_k A(m, k) B(k, n), general strides.
cudaError_t sg(fno_handle *h, const float *A, long long am, long long ak, long long sA, const float *B, long long bk,
               long long bn, long long sB, float *C, long long cm, long long cn, long long sC, int M, int N, int K,
               int batch, float beta) {
  return tc::gemm_f32(A, am, ak, sA, B, bk, bn, sB, C, cm, cn, sC, M, N, K, batch, beta, h->st);
}

// Site-major copy of a [B][rows][S] BF16 activation: out[b][s][row].
// Dynamic shared memory of the spectral kernels (bytes).
size_t ydft_smem(int mx, int my) { return (size_t)kYChunk * (2 * mx + 2 * my) * sizeof(float); }
size_t iy_smem(int mx, int my) { return (size_t)(2 * my * mx + 2 * my * kYChunk) * sizeof(float); }
size_t mix_smem(int B, int C, bool back) { return (size_t)((back ? 4 : 2) * B * C + 2 * C * C) * sizeof(float); }

void site_major(fno_handle *h, const __nv_bfloat16 *in, int B, int rows, long long S, __nv_bfloat16 *out) {
  const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((S + 63) / 64), (unsigned)B);
  if (rows % 32 == 0 && S % 8 == 0)
    transpose_bf16_v8_kernel<<<grid, 256, 0, h->st>>>(in, rows, S, out);
  else
    transpose_bf16_kernel<<<grid, 256, 0, h->st>>>(in, rows, S, out);
}

// out[ch] = sum over (b, s) of a[b, ch, s] for the C channels of a.
void chan_reduce(fno_handle *h, const float *a, int B, int C, long long S, float *out) {
  if (S % 4 == 0 && B * kReduceBlocks <= h->rpart_fields) {
    // float4 loads; about 2048 blocks, at most 32 shares of a field
    const int nsplit = std::max(1, std::min(kReduceBlocks, (2048 + C * B - 1) / (C * B)));
    reduce_pass1_v4_kernel<<<dim3(C, B * nsplit), kThreads, 0, h->st>>>(a, C, S, nsplit, h->rpart);
    reduce_pass2_kernel<<<(C + 7) / 8, kThreads, 0, h->st>>>(h->rpart, C, B * nsplit, out);
    return;
  }
  reduce_pass1_kernel<<<dim3(C, kReduceBlocks), kThreads, 0, h->st>>>(a, B, C, S, h->rpart);
  reduce_pass2_kernel<<<(C + 7) / 8, kThreads, 0, h->st>>>(h->rpart, C, kReduceBlocks, out);
}

// out[ca * Cb + cb] = sum over (b, s) of a[b, ca, s] f(o2[b, cb, s]) (f = gelu
// for the projection's Q2, identity for the lift's P), in the order of
// outer_pass1_kernel and reduce_pass2_kernel.
template <int NA, int NB, bool kGelu>
void outer_reduce(fno_handle *h, const float *a, const float *o2, int B, int Ca, int Cb, long long S, float *out) {
  const int tiles = ((Ca + NA - 1) / NA) * ((Cb + NB - 1) / NB);
  outer_pass1_kernel<NA, NB, kGelu><<<dim3(kOuterBlocks, tiles), kThreads, 0, h->st>>>(a, o2, B, Ca, Cb, S, h->rpart);
  reduce_pass2_kernel<<<(Ca * Cb + 7) / 8, kThreads, 0, h->st>>>(h->rpart, Ca * Cb, kOuterBlocks,
                                                                                   out);
}

template <typename T>
cudaError_t alloc(T **p, long long n) {
  return cudaMalloc((void **)p, (size_t)std::max<long long>(n, 1) * sizeof(T));
}

void free_workspace(fno_handle *h) {
  void *ps[] = {h->x0, h->A, h->G, h->Gb, h->hp, h->out, h->dout, h->dhp, h->dhpb, h->dV, h->dZ, h->dZb, h->dG,
                h->dA, h->dAb, h->dY, h->dS, h->partial, h->loss, h->Fx, h->Fxi, h->Fxb, h->Fxib, h->rpart, h->wpart, h->Ty,
                h->FxTb, h->FxiTb, h->dZT, h->dhpT, h->wTb, h->gerr};
  for (void *p : ps) cudaFree(p);
  for (int l = 0; l <= kMaxLayers; l++) {
    cudaFree(h->V[l]);
    cudaFree(h->Vb[l]);
    cudaFree(h->VbT[l]);
    h->V[l] = nullptr;
    h->Vb[l] = nullptr;
    h->VbT[l] = nullptr;
  }
  for (int l = 0; l < kMaxLayers; l++) {
    cudaFree(h->Z[l]);
    cudaFree(h->Sh[l]);
    h->Z[l] = nullptr;
    h->Sh[l] = nullptr;
  }
}

cudaError_t alloc_workspace(fno_handle *h) {
  const fno_config &c = h->c;
  const long long S = (long long)c.nx_max * c.ny_max, B = c.batch_max;
  h->cap_bcs = B * c.width * S;
  h->cap_bs = B * c.outputs * S;
  h->cap_bhs = B * c.hidden * S;
  h->cap_line = B * c.width * (long long)c.ny_max * 2 * c.modes_x;
  h->cap_modes = B * c.width * (long long)c.modes_x * c.modes_y * 2;
  cudaError_t e = alloc(&h->x0, B * kFeatures * S);
  for (int l = 0; l <= c.layers && e == cudaSuccess; l++) {
    e = alloc(&h->V[l], h->cap_bcs);
    if (e == cudaSuccess) e = alloc(&h->Vb[l], h->cap_bcs);
    if (e == cudaSuccess && c.gemm_bf16) e = alloc(&h->VbT[l], h->cap_bcs);
  }
  if (e == cudaSuccess && c.gemm_bf16) e = alloc(&h->dZT, h->cap_bcs);
  if (e == cudaSuccess && c.gemm_bf16) e = alloc(&h->dhpT, h->cap_bhs);
  if (e == cudaSuccess) e = alloc(&h->wTb, (long long)c.layers * c.width * c.width + (long long)c.width * c.hidden);
  if (e == cudaSuccess) e = alloc(&h->gerr, 1);
  if (e == cudaSuccess) e = cudaMemset(h->gerr, 0, sizeof(int));
  for (int l = 0; l < c.layers && e == cudaSuccess; l++) {
    e = alloc(&h->Z[l], h->cap_bcs);
    if (e == cudaSuccess) e = alloc(&h->Sh[l], h->cap_modes);
  }
  if (e == cudaSuccess) e = alloc(&h->A, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->G, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->Gb, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->hp, h->cap_bhs);
  if (e == cudaSuccess) e = alloc(&h->out, h->cap_bs);
  if (e == cudaSuccess) e = alloc(&h->dout, h->cap_bs);
  if (e == cudaSuccess) e = alloc(&h->dhp, h->cap_bhs);
  if (e == cudaSuccess) e = alloc(&h->dhpb, h->cap_bhs);
  if (e == cudaSuccess) e = alloc(&h->dV, h->cap_bcs);
  if (e == cudaSuccess) e = alloc(&h->dZ, h->cap_bcs);
  if (e == cudaSuccess) e = alloc(&h->dZb, h->cap_bcs);
  if (e == cudaSuccess) e = alloc(&h->dG, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->dA, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->dAb, h->cap_line);
  if (e == cudaSuccess) e = alloc(&h->dY, h->cap_modes);
  if (e == cudaSuccess) e = alloc(&h->dS, h->cap_modes);
  if (e == cudaSuccess) e = alloc(&h->partial, 8192);
  const long long max_ch = std::max(std::max(c.width, c.hidden), c.outputs);
  h->rpart_fields = (int)(B * kReduceBlocks);  // channel sums: at most 32 shares of each field
  if (e == cudaSuccess)
    e = alloc(&h->rpart, std::max((long long)std::max(c.width * kFeatures, c.hidden * c.outputs) * kOuterBlocks,
                                  max_ch * h->rpart_fields));
  if (e == cudaSuccess) e = alloc(&h->wpart, B * kWSplit * (long long)std::max(c.width, c.hidden) * c.width);
  if (e == cudaSuccess) e = alloc(&h->loss, 1);
  if (e == cudaSuccess) e = alloc(&h->Fx, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->Fxi, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->Fxb, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->Fxib, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->FxTb, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->FxiTb, (long long)c.nx_max * 2 * c.modes_x);
  if (e == cudaSuccess) e = alloc(&h->Ty, (long long)c.ny_max * c.modes_y);
  return e;
}

}  // namespace

extern "C" {

int fno_create(const fno_config *cfg, fno_handle **out) {
  if (!cfg || !out) return ffail(nullptr, LB_ERR_ARG, "fno_create: null argument");
  *out = nullptr;
  const fno_config &c = *cfg;
  if (c.width < 1 || c.hidden < 1 || c.layers < 1 || c.layers > kMaxLayers || c.modes_x < 1 || c.modes_y < 2 ||
      c.modes_y % 2 != 0 || c.batch_max < 1 || c.nx_max < 2 || c.ny_max < 2 || 2 * c.modes_x > c.nx_max ||
      c.modes_y > c.ny_max || c.outputs < 1 || c.outputs > kMaxOutputs ||
      c.modes_x * c.modes_y > 2 * kThreads ||  // ydft_kernel: two modes per thread
      std::max(ydft_smem(c.modes_x, c.modes_y), std::max(iy_smem(c.modes_x, c.modes_y),
                                                            mix_smem(c.batch_max, c.width, true))) > 48 * 1024)
    return ffail(nullptr, LB_ERR_ARG, "fno_create: bad sizes");
  if (c.gemm_bf16 && (c.width % 8 || c.hidden % 8 || (2 * c.modes_x) % 8))
    return ffail(nullptr, LB_ERR_ARG, "fno_create: BF16 tensor-core products need width, hidden and 2 modes_x "
                                      "divisible by 8");
  fno_handle *h = new (std::nothrow) fno_handle();
  if (!h) return ffail(nullptr, LB_ERR_OOM, "fno_create: host allocation failed");
  h->c = c;
  h->st = (cudaStream_t)c.stream;
  h->o = make_offsets(c);
  const long long np = (long long)h->o.total;
  cudaError_t e = alloc(&h->prm, np);
  if (e == cudaSuccess) e = alloc(&h->grd, np);
  if (e == cudaSuccess) e = alloc(&h->m1, np);
  if (e == cudaSuccess) e = alloc(&h->m2, np);
  if (e == cudaSuccess) e = alloc(&h->prmb, np);
  if (e == cudaSuccess) e = cudaMemset(h->prm, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->grd, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->m1, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->m2, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(h->prmb, 0, np * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = alloc_workspace(h);
  if (e != cudaSuccess) {
    std::string m = std::string("fno_create: ") + cudaGetErrorString(e);
    fno_destroy(h);
    return ffail(nullptr, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA, m);
  }
  *out = h;
  return LB_OK;
}

int64_t fno_param_count(const fno_handle *h) { return h ? (int64_t)h->o.total : 0; }

int fno_set_params(fno_handle *h, const float *host) {
  if (!h || !host) return ffail(h, LB_ERR_ARG, "fno_set_params: null argument");
  const long long np = (long long)h->o.total;
  FNO_CUDA(h, cudaMemcpyAsync(h->prm, host, np * sizeof(float), cudaMemcpyHostToDevice, h->st));
  to_bf16_kernel<<<blocks_for(np), kThreads, 0, h->st>>>(h->prm, np, h->prmb);
  weights_t_kernel<<<blocks_for(np), kThreads, 0, h->st>>>(h->prmb, h->o, h->c.width, h->c.hidden, h->c.layers,
                                                           h->wTb);
  FNO_CUDA(h, cudaGetLastError());
  FNO_CUDA(h, cudaStreamSynchronize(h->st));
  return LB_OK;
}

int fno_get_params(fno_handle *h, float *host) {
  if (!h || !host) return ffail(h, LB_ERR_ARG, "fno_get_params: null argument");
  FNO_CUDA(h, cudaMemcpyAsync(host, h->prm, h->o.total * sizeof(float), cudaMemcpyDeviceToHost, h->st));
  FNO_CUDA(h, cudaStreamSynchronize(h->st));
  return LB_OK;
}

int fno_get_grads(fno_handle *h, float *host) {
  if (!h || !host) return ffail(h, LB_ERR_ARG, "fno_get_grads: null argument");
  FNO_CUDA(h, cudaMemcpyAsync(host, h->grd, h->o.total * sizeof(float), cudaMemcpyDeviceToHost, h->st));
  FNO_CUDA(h, cudaStreamSynchronize(h->st));
  return LB_OK;
}

int fno_forward(fno_handle *h, int32_t B, int32_t nx, int32_t ny, const float *params_dev, float *out) {
  if (!h || !params_dev) return ffail(h, LB_ERR_ARG, "fno_forward: null argument");
  const fno_config &c = h->c;
  if (B < 1 || B > c.batch_max || nx > c.nx_max || ny > c.ny_max || nx < 2 * c.modes_x || ny < c.modes_y)
    return ffail(h, LB_ERR_ARG, "fno_forward: batch or lattice outside the workspace bounds");
  if (c.gemm_bf16 && nx % 8) return ffail(h, LB_ERR_ARG, "fno_forward: BF16 products need nx divisible by 8");
  const int C = c.width, H = c.hidden, L = c.layers, mx = c.modes_x, my = c.modes_y;
  const long long S = (long long)nx * ny;
  const int R = B * C * ny;
  cudaStream_t st = h->st;
  if (h->tab_nx != nx || h->tab_ny != ny) {
    dft_tables_kernel<<<blocks_for((long long)std::max(nx * mx, ny * my)), kThreads, 0, st>>>(
        nx, ny, mx, my, h->Fx, h->Fxi, h->Fxb, h->Fxib, h->FxTb, h->FxiTb, h->Ty);
    FNO_CUDA(h, cudaGetLastError());
    h->tab_nx = nx;
    h->tab_ny = ny;
  }
  const float *P = h->prm;
  features_kernel<<<blocks_for((long long)B * S), kThreads, 0, st>>>(params_dev, B, nx, ny, h->x0);
  lift_kernel<<<grid2(S, B * C), kThreads, 0, st>>>(h->x0, P + h->o.P, P + h->o.p, C, S, h->V[0], h->Vb[0]);
  FNO_CUDA(h, cudaGetLastError());
  const bool bf = c.gemm_bf16 != 0;
  if (bf) site_major(h, h->Vb[0], B, C, S, h->VbT[0]);
  const long long CS = (long long)C * S;
  for (int l = 0; l < L; l++) {
    // x-transform of every line: A[R, 2mx] = V[R, nx] Fx[nx, 2mx]
    if (bf)
      FNO_GEMM(h, tcg(h, h->Vb[l], nx, 0, h->FxTb, nx, 0, h->A, 2 * mx, 1, 0, R, 2 * mx, nx, 1, 1, 0.f));
    else
      FNO_GEMM(h, sg(h, h->V[l], nx, 1, 0, h->Fx, 2 * mx, 1, 0, h->A, 2 * mx, 1, 0, R, 2 * mx, nx, 1, 0.f));
    // y-transform, per-mode mixing (into the dY scratch), inverse y-transform
    ydft_kernel<<<B * C, kThreads, ydft_smem(mx, my), st>>>(h->A, h->Ty, ny, mx, my, h->Sh[l]);
    mix_kernel<<<my * mx, kThreads, mix_smem(B, C, false), st>>>(h->Sh[l], P + h->o.Rr[l], P + h->o.Ri[l], B, C,
                                                                   my * mx, h->dY);
    iy_kernel<<<B * C, kThreads, iy_smem(mx, my), st>>>(h->dY, h->Ty, ny, mx, my, h->G, h->Gb);
    FNO_CUDA(h, cudaGetLastError());
    // inverse x-transform into z: Z[R, nx] = G[R, 2mx] Fxi[2mx, nx]
    if (bf)
      FNO_GEMM(h, tcg(h, h->Gb, 2 * mx, 0, h->FxiTb, 2 * mx, 0, h->Z[l], nx, 1, 0, R, nx, 2 * mx, 1, 1, 0.f));
    else
      FNO_GEMM(h, sg(h, h->G, 2 * mx, 1, 0, h->Fxi, nx, 1, 0, h->Z[l], nx, 1, 0, R, nx, 2 * mx, 1, 0.f));
    // z[b][o][s] += sum_c W[o][c] v[b][c][s]  (tensor cores: sites as rows,
    // the site-major copy of v against W, written transposed)
    if (bf)
      FNO_GEMM(h, tcg(h, h->VbT[l], C, CS, h->prmb + h->o.W[l], C, 0, h->Z[l], 1, S, CS, (int)S, C, C, B, 1, 1.f));
    else
      FNO_GEMM(h, sg(h, P + h->o.W[l], C, 1, 0, h->V[l], S, 1, CS, h->Z[l], S, 1, CS, C, (int)S, C, B, 1.f));
    bias_act_kernel<<<grid2(S, B * C), kThreads, 0, st>>>(h->Z[l], P + h->o.w[l], C, S, l < L - 1 ? 1 : 0,
                                                           h->V[l + 1], h->Vb[l + 1]);
    FNO_CUDA(h, cudaGetLastError());
    if (bf) site_major(h, h->Vb[l + 1], B, C, S, h->VbT[l + 1]);
  }
  // projection: hp[b][h][s] = sum_c Q1[h][c] v_L[b][c][s]; out = Q2 gelu(hp + q1) + q2
  if (bf)
    FNO_GEMM(h, tcg(h, h->VbT[L], C, CS, h->prmb + h->o.Q1, C, 0, h->hp, 1, S, (long long)H * S, (int)S, H, C, B, 1,
                    0.f));
  else
    FNO_GEMM(h, sg(h, P + h->o.Q1, C, 1, 0, h->V[L], S, 1, CS, h->hp, S, 1, (long long)H * S, H, (int)S, C, B, 0.f));
  project_kernel<<<grid2(S, B), kThreads, 0, st>>>(h->hp, P + h->o.q1, P + h->o.Q2, P + h->o.q2, H,
                                                                     c.outputs, S, h->out, out);
  FNO_CUDA(h, cudaGetLastError());
  h->B = B;
  h->nx = nx;
  h->ny = ny;
  h->have_forward = true;
  return LB_OK;
}

int fno_backward(fno_handle *h, const float *target, double *loss) {
  if (!h || !target) return ffail(h, LB_ERR_ARG, "fno_backward: null argument");
  if (!h->have_forward) return ffail(h, LB_ERR_STATE, "fno_backward: no forward pass");
  const fno_config &c = h->c;
  const int B = h->B, nx = h->nx, ny = h->ny, C = c.width, H = c.hidden, L = c.layers, mx = c.modes_x, my = c.modes_y;
  const int O = c.outputs;
  const long long S = (long long)nx * ny, BCS = (long long)B * C * S, BS = (long long)B * O * S;
  const int R = B * C * ny;
  cudaStream_t st = h->st;
  const float *P = h->prm;
  const Offsets &o = h->o;
  float *g = h->grd;
  const unsigned lb = blocks_for(BS);
  loss_kernel<<<lb, kThreads, 0, st>>>(h->out, target, BS, h->dout, h->partial);
  finish_loss_kernel<<<1, kThreads, 0, st>>>(h->partial, (int)lb, BS, h->loss);
  // projection: dq2, dQ2, dhp, dq1, dQ1, dV = Q1^T dhp
  chan_reduce(h, h->dout, B, O, S, g + o.q2);
  outer_reduce<kMaxOutputs, 8, true>(h, h->dout, h->hp, B, O, H, S, g + o.Q2);
  project_back_kernel<<<grid2(S, B * H), kThreads, 0, st>>>(h->hp, P + o.Q2, h->dout, H, O, S, h->dhp, h->dhpb);
  chan_reduce(h, h->dhp, B, H, S, g + o.q1);
  FNO_CUDA(h, cudaGetLastError());
  const bool bf = c.gemm_bf16 != 0;
  const long long CS = (long long)C * S, HS = (long long)H * S;
  // dQ1 = sum_b dhp[b] v_L[b]^T: per-field (and K-split) parts, then their sum
  int parts = B;
  if (bf) {
    parts = B * kWSplit;
    FNO_GEMM(h, tcg(h, h->dhpb, (int)S, HS, h->Vb[L], (int)S, CS, h->wpart, C, 1, (long long)H * C, H, C, (int)S, B,
                    kWSplit, 0.f));
  } else {
    FNO_GEMM(h, sg(h, h->dhp, S, 1, HS, h->V[L], 1, S, CS, h->wpart, C, 1, (long long)H * C, H, C, (int)S, B, 0.f));
  }
  sum_fields_kernel<<<(H * C + 31) / 32, kThreads, 0, st>>>(h->wpart, parts, H * C, g + o.Q1);
  // dv[b][c][s] = sum_h Q1[h][c] dhp[b][h][s]
  if (bf) {
    site_major(h, h->dhpb, B, H, S, h->dhpT);
    FNO_GEMM(h, tcg(h, h->dhpT, H, HS, h->wTb + (size_t)L * C * C, H, 0, h->dV, 1, S, CS, (int)S, C, H, B, 1, 0.f));
  } else {
    FNO_GEMM(h, sg(h, P + o.Q1, 1, C, 0, h->dhp, S, 1, HS, h->dV, S, 1, CS, C, (int)S, H, B, 0.f));
  }
  for (int l = L - 1; l >= 0; l--) {
    act_back_kernel<<<blocks_for(BCS), kThreads, 0, st>>>(h->dV, h->Z[l], BCS, l < L - 1 ? 1 : 0, h->dZ, h->dZb);
    chan_reduce(h, h->dZ, B, C, S, g + o.w[l]);
    FNO_CUDA(h, cudaGetLastError());
    // dW = sum_b dz[b] v[b]^T
    if (bf)
      FNO_GEMM(h, tcg(h, h->dZb, (int)S, CS, h->Vb[l], (int)S, CS, h->wpart, C, 1, (long long)C * C, C, C, (int)S, B,
                      kWSplit, 0.f));
    else
      FNO_GEMM(h, sg(h, h->dZ, S, 1, CS, h->V[l], 1, S, CS, h->wpart, C, 1, (long long)C * C, C, C, (int)S, B, 0.f));
    sum_fields_kernel<<<(C * C + 31) / 32, kThreads, 0, st>>>(h->wpart, parts, C * C, g + o.W[l]);
    // spectral path: dG = dz Fxi^T, then the adjoints of the mixing and of the y-transform
    if (bf)
      FNO_GEMM(h, tcg(h, h->dZb, nx, 0, h->Fxib, nx, 0, h->dG, 2 * mx, 1, 0, R, 2 * mx, nx, 1, 1, 0.f));
    else
      FNO_GEMM(h, sg(h, h->dZ, nx, 1, 0, h->Fxi, 1, nx, 0, h->dG, 2 * mx, 1, 0, R, 2 * mx, nx, 1, 0.f));
    // adjoints: of the inverse y-transform (a y-transform), of the mixing
    // (with the weights' gradient), of the y-transform (an inverse one)
    ydft_kernel<<<B * C, kThreads, ydft_smem(mx, my), st>>>(h->dG, h->Ty, ny, mx, my, h->dY);
    mix_back_kernel<<<my * mx, kThreads, mix_smem(B, C, true), st>>>(h->dY, h->Sh[l], P + o.Rr[l], P + o.Ri[l], B, C,
                                                                       my * mx, h->dS, g + o.Rr[l], g + o.Ri[l]);
    iy_kernel<<<B * C, kThreads, iy_smem(mx, my), st>>>(h->dS, h->Ty, ny, mx, my, h->dA, h->dAb);
    FNO_CUDA(h, cudaGetLastError());
    // dv = W^T dz (pointwise path) + dA Fx^T (spectral path)
    if (bf) {
      site_major(h, h->dZb, B, C, S, h->dZT);
      FNO_GEMM(h, tcg(h, h->dZT, C, CS, h->wTb + (size_t)l * C * C, C, 0, h->dV, 1, S, CS, (int)S, C, C, B, 1, 0.f));
      FNO_GEMM(h, tcg(h, h->dAb, 2 * mx, 0, h->Fxb, 2 * mx, 0, h->dV, nx, 1, 0, R, nx, 2 * mx, 1, 1, 1.f));
    } else {
      FNO_GEMM(h, sg(h, P + o.W[l], 1, C, 0, h->dZ, S, 1, CS, h->dV, S, 1, CS, C, (int)S, C, B, 0.f));
      FNO_GEMM(h, sg(h, h->dA, 2 * mx, 1, 0, h->Fx, 1, 2 * mx, 0, h->dV, nx, 1, 0, R, nx, 2 * mx, 1, 1.f));
    }
  }
  // lift: dp = sum dv0, dP[o, c] = sum dv0[b, o, s] x0[b, c, s]
  chan_reduce(h, h->dV, B, C, S, g + o.p);
  outer_reduce<8, kFeatures, false>(h, h->dV, h->x0, B, C, kFeatures, S, g + o.P);
  FNO_CUDA(h, cudaGetLastError());
  if (loss) {
    int gerr = 0;
    FNO_CUDA(h, cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    FNO_CUDA(h, cudaMemcpyAsync(&gerr, h->gerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    FNO_CUDA(h, cudaStreamSynchronize(st));
    if (gerr) return ffail(h, LB_ERR_TIMEOUT, "fno_backward: a tensor-core product's bounded wait gave up");
  }
  return LB_OK;
}

int fno_fields(fno_handle *h, const float *out, int32_t batch, int32_t nx, int32_t ny, const double *scales,
               double rho_mean, double *fields) {
  if (!h || !out || !scales || !fields) return ffail(h, LB_ERR_ARG, "fno_fields: null argument");
  // (the block sums of every field share the 8192-double loss partials)
  if (batch < 1 || batch > 8192 || nx < 1 || ny < 1 || h->c.outputs < 3)
    return ffail(h, LB_ERR_ARG, "fno_fields: batch, lattice or output channels out of range");
  const long long S = (long long)nx * ny;
  // block sums in the loss partials (8192 doubles, batch * nblk of them; the
  // same stream orders their uses)
  const int nblk = (int)std::max<long long>(1, std::min<long long>({256, 8192 / batch, (S + kThreads - 1) / kThreads}));
  field_mass_kernel<<<dim3(nblk, batch), kThreads, 0, h->st>>>(out, h->c.outputs, S, scales[0], h->partial);
  fields_kernel<<<dim3(nblk, batch), kThreads, 0, h->st>>>(out, h->c.outputs, S, scales[0], scales[1], scales[2],
                                                           rho_mean, h->partial, nblk, fields);
  FNO_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int fno_adam(fno_handle *h, float lr, float beta1, float beta2, float eps, int32_t t) {
  if (!h || t < 1) return ffail(h, LB_ERR_ARG, "fno_adam: bad arguments");
  const long long np = (long long)h->o.total;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  adam_kernel<<<blocks_for(np), kThreads, 0, h->st>>>(h->prm, h->grd, h->m1, h->m2, np, lr, beta1, beta2, eps, c1, c2,
                                                       h->prmb);
  weights_t_kernel<<<blocks_for(np), kThreads, 0, h->st>>>(h->prmb, h->o, h->c.width, h->c.hidden, h->c.layers,
                                                           h->wTb);
  FNO_CUDA(h, cudaGetLastError());
  return LB_OK;
}

int fno_destroy(fno_handle *h) {
  if (!h) return LB_OK;
  cudaStreamSynchronize(h->st);
  free_workspace(h);
  cudaFree(h->prm);
  cudaFree(h->grd);
  cudaFree(h->m1);
  cudaFree(h->m2);
  cudaFree(h->prmb);
  delete h;
  return LB_OK;
}

const char *fno_last_error(const fno_handle *h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"
