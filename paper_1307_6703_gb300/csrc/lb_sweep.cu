// lb_sweep.cu -- FP32 strip-sweep kernel: one fused time step of the vdW
// lattice Boltzmann scheme (arXiv:1307.6703, Sec. II) streamed through
// shared memory by TMA.
//
// Work decomposition.  The lattice is cut into column strips of W <= 120
// interior columns and row segments of up to SEG rows.  One CTA (128
// threads, one thread per column of a 128-column window x0-4 .. x0+123)
// sweeps its segment upwards, one row per iteration.  Every row of the
// previous state is read from HBM once by the TMA engine: a 3D tensor copy
// brings the 128-column row of all nine population planes into a ring of
// RING rows in shared memory (mbarrier-tracked), RING-7 rows ahead of use.
//
// Per iteration r four stages run, separated by CTA barriers:
//   A  row r    : propagated populations (pull), density n (n-hat on walls),
//                 raw momentum sum_i f_i c_i                 -> ring n[5]
//   B  row r-1  : P = p^i - p^w (Eq. eqstate) and L = lap n   -> ring P,L[3]
//   C  row r-2  : F = dP + kappa n dL + F_ext (Eq. force2), n u* (Eq. newvel),
//                 wall rule on wall rows                       -> ring J[3]
//   D  row r-3  : grad n, div(n u*), equilibrium (Eq. eqfunc), forcing
//                 (Eqs. forceterm, coeff), BGK collision; store f* to HBM.
// Column halos (3, 2, 1 sites for n, P/L, F/J) are computed by the edge
// threads of the window; row halos come from the sweep itself, so apart from
// the 7-row warm-up of each segment nothing is recomputed.
//
// Walls: rows -1 and ny of n, P, L and n u* are read from their mirror rows
// 1 and ny-2 (even reflection; y part of n u* odd), mathematically the ghost
// rows of the scheme.  Periodic directions: the state buffers carry 4 ghost
// columns (and, without walls, 4 ghost rows) on each side, refreshed by the
// kernel when it stores boundary sites, so every TMA box is one plain copy.
//
// The collision uses the algebraically equivalent "moment" form
//   f*_i = (1 - omega) f_i + w_i E_i,
//   E_i = omega n [A_i + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2] + 3 c.B + 9/2 C:cc - 3/2 tr C,
// with A_i the rest factor 1 + (T - T0)(c.c - 2 T0) / (2 T0^2), T0 = 1/3;
// the rest population is taken as n minus the other eight, which is the same
// value in exact arithmetic and keeps the site mass exact in FP32.
//
// Every CTA also writes FP64 partial sums of mass and momentum of the state
// it stored, and a flag for non-finite or out-of-range sites, so that the
// global reduction of the new state costs one tiny kernel.
#include <cuda.h>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbk {

namespace {

constexpr int kThreads = 128;
constexpr int kCols = 128;
constexpr int kRing = 10;
constexpr unsigned kRowBytes = 9u * kCols * sizeof(float);
constexpr uint32_t kWaitLimit = 1u << 22;

struct __align__(128) SweepSmem {
  float pops[kRing][9][kCols];
  float n[5][kCols];
  float P[3][kCols];
  float L[3][kCols];
  float Jx[3][kCols];
  float Jy[3][kCols];
  unsigned long long full[kRing];
  double red[4][kThreads / 32];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// Wait for phase `parity` of an mbarrier; gives up after a bounded number
// of polls and reports it (the data are then meaningless but every address
// the kernel touches stays in bounds).
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, int *err) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return;
  }
  atomicOr(err, 1);
}

// One row (all nine planes, 128 columns) of the padded state into a ring slot.
__device__ __forceinline__ void tma_row(const CUtensorMap *map, uint32_t dst, uint32_t bar, int xpad,
                                        int ypad) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kRowBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(xpad), "r"(ypad), "r"(0), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int mirror_row(int y, int ny, int walls) {
  if (!walls) return y;
  if (y < 0) return -y;
  if (y > ny - 1) return 2 * (ny - 1) - y;
  return y;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 4)
sweep_step_kernel(const __grid_constant__ CUtensorMap tin, const SweepArgs A) {
  extern __shared__ unsigned char smem_raw[];
  SweepSmem &S = *reinterpret_cast<SweepSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));

  const int t = threadIdx.x;
  const int strip = blockIdx.x, seg = blockIdx.y;
  const int x0 = strip * A.base_w + 4 * min(strip, A.extra);
  const int W = A.base_w + (strip < A.extra ? 4 : 0);
  const int ya = seg * A.seg_h;
  const int yb = min(A.ny, ya + A.seg_h);
  const int nx = A.nx, ny = A.ny;
  const bool walls = A.walls != 0;
  const int x = x0 - 4 + t;  // interior column of this thread (may be a halo column)
  const int xw = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  const bool actA = t >= 1 && t <= W + 6;
  const bool actB = t >= 2 && t <= W + 5;
  const bool actC = t >= 3 && t <= W + 4;
  const bool actD = t >= 4 && t <= W + 3;
  const int nload = (yb - ya) + 8;  // rows ya-4 .. yb+3
  const float sinx = actC ? A.sinx[xw] : 0.f;  // x in [x0-1, x0+W] for stage C

  if (t == 0) {
    for (int s = 0; s < kRing; ++s) mbar_init(smem_u32(&S.full[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int L = 0; L < min(kRing, nload); ++L)
      tma_row(&tin, smem_u32(&S.pops[L][0][0]), smem_u32(&S.full[L]), x0, ya + L);
  }
  __syncthreads();
  mbar_wait(smem_u32(&S.full[0]), 0, A.err);
  mbar_wait(smem_u32(&S.full[1]), 0, A.err);

  // ring slots (all row arguments are >= ya - 4)
  auto pslot = [&](int y) { return (y - ya + 4) % kRing; };
  auto nslot = [&](int y) { return (y - ya + 10) % 5; };
  auto tslot = [&](int y) { return (y - ya + 12) % 3; };

  float sx0 = 0.f, sy0 = 0.f, sx1 = 0.f, sy1 = 0.f, sx2 = 0.f, sy2 = 0.f;
  float Fx_cur = 0.f, Fy_cur = 0.f, Fx_prev = 0.f, Fy_prev = 0.f;
  float acc_m = 0.f, acc_x = 0.f, acc_y = 0.f;
  int bad = 0;

  for (int r = ya - 3; r <= yb + 2; ++r) {
    const int i = r - (ya - 3);
    {
      const int Lw = i + 2;  // newest row needed by this iteration
      mbar_wait(smem_u32(&S.full[Lw % kRing]), (Lw / kRing) & 1, A.err);
    }
    const int rA = r, rB = r - 1, rC = r - 2, rD = r - 3;

    // ------------------------------------------------ A: density, raw momentum
    sx2 = sx1; sy2 = sy1; sx1 = sx0; sy1 = sy0;
    if (actA && (!walls || (rA >= 0 && rA <= ny - 1))) {
      const float(*pm)[kCols] = S.pops[pslot(rA - 1)];
      const float(*p0)[kCols] = S.pops[pslot(rA)];
      const float(*pp)[kCols] = S.pops[pslot(rA + 1)];
      const float f0 = p0[0][t], f1 = p0[1][t - 1], f3 = p0[3][t + 1];
      const float f2 = pm[2][t], f5 = pm[5][t - 1], f6 = pm[6][t + 1];
      const float f4 = pp[4][t], f7 = pp[7][t + 1], f8 = pp[8][t - 1];
      float n;
      if (walls && rA == 0) {
        n = p0[0][t] + p0[4][t] + p0[7][t] + p0[8][t] + f1 + f3 + f4 + f7 + f8;
      } else if (walls && rA == ny - 1) {
        n = p0[0][t] + p0[2][t] + p0[6][t] + p0[5][t] + f1 + f3 + f2 + f6 + f5;
      } else {
        n = (((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7))) + f8;
        sx0 = ((f1 - f3) + (f5 - f6)) + (f8 - f7);
        sy0 = ((f2 - f4) + (f5 + f6)) - (f7 + f8);
      }
      S.n[nslot(rA)][t] = n;
    }
    __syncthreads();
    // The slot of row L = i - 4 is free now (last used by iteration i - 1).
    if (t == 0 && i >= 4 && i - 4 + kRing < nload) {
      const int L = i - 4 + kRing;
      tma_row(&tin, smem_u32(&S.pops[L % kRing][0][0]), smem_u32(&S.full[L % kRing]), x0, ya + L);
    }

    // ------------------------------------------------ B: P and lap n
    if (actB && rB >= ya - 2 && (!walls || (rB >= 0 && rB <= ny - 1))) {
      const float *nm = S.n[nslot(mirror_row(rB - 1, ny, A.walls))];
      const float *n0 = S.n[nslot(rB)];
      const float *np = S.n[nslot(mirror_row(rB + 1, ny, A.walls))];
      const float c = n0[t];
      const float lap = A.Q * ((n0[t + 1] + n0[t - 1]) + (np[t] + nm[t])) +
                        A.R * ((np[t + 1] + np[t - 1]) + (nm[t + 1] + nm[t - 1])) - A.four_QR * c;
      const float nT = c * A.T;
      const float pw = nT * __frcp_rn(1.0f - A.b * c) - A.a * c * c;
      S.P[tslot(rB)][t] = nT - pw;
      S.L[tslot(rB)][t] = lap;
    }
    __syncthreads();

    // ------------------------------------------------ C: force and n u*
    Fx_prev = Fx_cur;
    Fy_prev = Fy_cur;
    if (actC && rC >= ya - 1 && (!walls || (rC >= 0 && rC <= ny - 1))) {
      const int sm = tslot(mirror_row(rC - 1, ny, A.walls));
      const int s0 = tslot(rC);
      const int sp = tslot(mirror_row(rC + 1, ny, A.walls));
      const float *Pm = S.P[sm], *P0 = S.P[s0], *Pp = S.P[sp];
      const float *Lm = S.L[sm], *L0 = S.L[s0], *Lp = S.L[sp];
      const float dPx = A.N * (P0[t + 1] - P0[t - 1]) + A.M * ((Pp[t + 1] - Pp[t - 1]) + (Pm[t + 1] - Pm[t - 1]));
      const float dPy = A.N * (Pp[t] - Pm[t]) + A.M * ((Pp[t + 1] - Pm[t + 1]) + (Pp[t - 1] - Pm[t - 1]));
      const float dLx = A.N * (L0[t + 1] - L0[t - 1]) + A.M * ((Lp[t + 1] - Lp[t - 1]) + (Lm[t + 1] - Lm[t - 1]));
      const float dLy = A.N * (Lp[t] - Lm[t]) + A.M * ((Lp[t + 1] - Lm[t + 1]) + (Lp[t - 1] - Lm[t - 1]));
      const float n = S.n[nslot(rC)][t];
      const float kn = A.kappa * n;
      Fx_cur = (dPx + kn * dLx) + A.A0 * sinx;
      Fy_cur = dPy + kn * dLy;
      float sx = sx2, sy = sy2;
      if (walls && (rC == 0 || rC == ny - 1)) {
        const float(*pm)[kCols] = S.pops[pslot(rC - 1)];
        const float(*p0)[kCols] = S.pops[pslot(rC)];
        const float(*pp)[kCols] = S.pops[pslot(rC + 1)];
        float f[9];
        f[0] = p0[0][t]; f[1] = p0[1][t - 1]; f[3] = p0[3][t + 1];
        f[2] = pm[2][t]; f[5] = pm[5][t - 1]; f[6] = pm[6][t + 1];
        f[4] = pp[4][t]; f[7] = pp[7][t + 1]; f[8] = pp[8][t - 1];
        const bool top = rC != 0;
        wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx_cur, Fy_cur, n, f);
        sx = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
        sy = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
      }
      S.Jx[s0][t] = sx + 0.5f * Fx_cur;
      S.Jy[s0][t] = sy + 0.5f * Fy_cur;
    }
    __syncthreads();

    // ------------------------------------------------ D: collide and store
    if (actD && rD >= ya) {
      const bool bot_wall = walls && rD == 0, top_wall = walls && rD == ny - 1;
      const int mrm = mirror_row(rD - 1, ny, A.walls), mrp = mirror_row(rD + 1, ny, A.walls);
      const float *nm = S.n[nslot(mrm)], *n0 = S.n[nslot(rD)], *np = S.n[nslot(mrp)];
      const float n = n0[t];
      const float dnx = A.N * (n0[t + 1] - n0[t - 1]) + A.M * ((np[t + 1] - np[t - 1]) + (nm[t + 1] - nm[t - 1]));
      const float dny = A.N * (np[t] - nm[t]) + A.M * ((np[t + 1] - nm[t + 1]) + (np[t - 1] - nm[t - 1]));
      const int jm = tslot(mrm), j0 = tslot(rD), jp = tslot(mrp);
      const float sgm = (walls && rD == 0) ? -1.f : 1.f;       // J_y is odd across a wall
      const float sgp = (walls && rD == ny - 1) ? -1.f : 1.f;
      const float *Xm = S.Jx[jm], *X0 = S.Jx[j0], *Xp = S.Jx[jp];
      const float *Ym = S.Jy[jm], *Y0 = S.Jy[j0], *Yp = S.Jy[jp];
      const float dJx = A.N * (X0[t + 1] - X0[t - 1]) + A.M * ((Xp[t + 1] - Xp[t - 1]) + (Xm[t + 1] - Xm[t - 1]));
      const float dJy = A.N * (sgp * Yp[t] - sgm * Ym[t]) +
                        A.M * ((sgp * Yp[t + 1] - sgm * Ym[t + 1]) + (sgp * Yp[t - 1] - sgm * Ym[t - 1]));
      const float divJ = dJx + dJy;
      const float Jx = X0[t], Jy = Y0[t];
      const float Fx = Fx_prev, Fy = Fy_prev;

      const float(*pm)[kCols] = S.pops[pslot(rD - 1)];
      const float(*p0)[kCols] = S.pops[pslot(rD)];
      const float(*pp)[kCols] = S.pops[pslot(rD + 1)];
      float f[9];
      f[0] = p0[0][t]; f[1] = p0[1][t - 1]; f[3] = p0[3][t + 1];
      f[2] = pm[2][t]; f[5] = pm[5][t - 1]; f[6] = pm[6][t + 1];
      f[4] = pp[4][t]; f[7] = pp[7][t + 1]; f[8] = pp[8][t - 1];
      if (bot_wall || top_wall) wall_fill<float>(top_wall, top_wall ? A.u_top : A.u_bot, Fx, Fy, n, f);

      const float rn = __frcp_rn(n);
      const float ux = Jx * rn, uy = Jy * rn;
      // Guo coefficients B = g F, C (Eq. coeff with (T0 - T))
      const float Bx = A.g * Fx, By = A.g * Fy;
      const float Cxx = A.g * (2.f * ux * Fx + A.th * (2.f * ux * dnx + divJ));
      const float Cyy = A.g * (2.f * uy * Fy + A.th * (2.f * uy * dny + divJ));
      const float Cxy = A.g * ((ux * Fy + Fx * uy) + A.th * (ux * dny + uy * dnx));
      const float trC = Cxx + Cyy;
      const float on = A.omega * n;
      const float base = -1.5f * (on * (ux * ux + uy * uy) + trC);
      const float e_ax = on * A.A_ax + base, e_dg = on * A.A_diag + base;
      const float symx = 4.5f * (on * ux * ux + Cxx), antx = 3.f * (on * ux + Bx);
      const float symy = 4.5f * (on * uy * uy + Cyy), anty = 3.f * (on * uy + By);
      const float vp = ux + uy, vm = uy - ux;
      const float sym5 = 4.5f * (on * vp * vp + trC + 2.f * Cxy), ant5 = 3.f * (on * vp + (Bx + By));
      const float sym6 = 4.5f * (on * vm * vm + trC - 2.f * Cxy), ant6 = 3.f * (on * vm + (By - Bx));
      const float om1 = A.one_minus_omega;
      constexpr float w1 = 1.f / 9.f, w5 = 1.f / 36.f;
      float fs[9];
      fs[1] = om1 * f[1] + w1 * (e_ax + symx + antx);
      fs[3] = om1 * f[3] + w1 * (e_ax + symx - antx);
      fs[2] = om1 * f[2] + w1 * (e_ax + symy + anty);
      fs[4] = om1 * f[4] + w1 * (e_ax + symy - anty);
      fs[5] = om1 * f[5] + w5 * (e_dg + sym5 + ant5);
      fs[7] = om1 * f[7] + w5 * (e_dg + sym5 - ant5);
      fs[6] = om1 * f[6] + w5 * (e_dg + sym6 + ant6);
      fs[8] = om1 * f[8] + w5 * (e_dg + sym6 - ant6);
      // Collision conserves the site's mass exactly (A = 0 in Eq. forceterm,
      // sum f^eq = n): take the rest population as the remainder, so that
      // rounded weights cannot bias the total mass step after step.
      fs[0] = n - (((fs[1] + fs[3]) + (fs[2] + fs[4])) + ((fs[5] + fs[7]) + (fs[6] + fs[8])));

      const long long idx = A.off + (long long)rD * A.pitch + x;
#pragma unroll
      for (int q = 0; q < 9; ++q) A.fout[q * A.plane + idx] = fs[q];
      // periodic images in the ghost band
      const int gx = (x < 4) ? nx : ((x >= nx - 4) ? -nx : 0);
      const int gy = walls ? 0 : ((rD < 4) ? ny : ((rD >= ny - 4) ? -ny : 0));
      if (gx != 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) A.fout[q * A.plane + idx + gx] = fs[q];
      }
      if (gy != 0) {
        const long long iy = idx + (long long)gy * A.pitch;
#pragma unroll
        for (int q = 0; q < 9; ++q) A.fout[q * A.plane + iy] = fs[q];
        if (gx != 0) {
#pragma unroll
          for (int q = 0; q < 9; ++q) A.fout[q * A.plane + iy + gx] = fs[q];
        }
      }
      const float m = (((fs[0] + fs[1]) + (fs[2] + fs[3])) + ((fs[4] + fs[5]) + (fs[6] + fs[7]))) + fs[8];
      const float jx = ((fs[1] - fs[3]) + (fs[5] - fs[6])) + (fs[8] - fs[7]);
      const float jy = ((fs[2] - fs[4]) + (fs[5] + fs[6])) - (fs[7] + fs[8]);
      if (!(m > 0.f && m < A.nmax) || !isfinite(jx) || !isfinite(jy)) bad = 1;
      acc_m += m;
      acc_x += jx;
      acc_y += jy;
    }
  }

  // CTA partial sums of the stored state (FP64, fixed order).
  double v[4] = {(double)acc_m, (double)acc_x, (double)acc_y, (double)bad};
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if ((t & 31) == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) S.red[c][t >> 5] = v[c];
  __syncthreads();
  if (t == 0) {
    double *out = A.partials + 4 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) s += S.red[c][w];
      out[c] = s;
    }
  }
}

// Copy the periodic images into the ghost band of a padded buffer.
__global__ void ghost_fill_kernel(float *f, int nx, int ny, int pitch, long long plane, long long off,
                                  int walls) {
  const int rows = ny + 8;
  const long long total = 9LL * rows * pitch;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(k / ((long long)rows * pitch));
    const long long rem = k - (long long)q * rows * pitch;
    const int py = (int)(rem / pitch), px = (int)(rem % pitch);
    const int y = py - 4, x = px - 4;
    if (x >= nx + 4) continue;
    const bool gxb = (x < 0 || x >= nx), gyb = (y < 0 || y >= ny);
    if (!gxb && !gyb) continue;
    if (gyb && walls) continue;
    const int sx = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    const int sy = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    f[q * plane + off + (long long)y * pitch + x] = f[q * plane + off + (long long)sy * pitch + sx];
  }
}

cudaError_t sweep_prepare(size_t *smem_bytes) {
  *smem_bytes = sizeof(SweepSmem) + 128;
  return cudaFuncSetAttribute(sweep_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)*smem_bytes);
}

cudaError_t launch_sweep(const CUtensorMap &tin, const SweepArgs &A, size_t smem, cudaStream_t st) {
  dim3 grid((unsigned)A.nstrips, (unsigned)A.nseg);
  sweep_step_kernel<<<grid, kThreads, smem, st>>>(tin, A);
  return cudaGetLastError();
}

cudaError_t launch_ghost_fill(float *f, int nx, int ny, int pitch, long long plane, long long off,
                              int walls, cudaStream_t st) {
  const long long total = 9LL * (ny + 8) * pitch;
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 4096);
  ghost_fill_kernel<<<blocks, 256, 0, st>>>(f, nx, ny, pitch, plane, off, walls);
  return cudaGetLastError();
}

}  // namespace lbk
