// lb_sweep.cu -- FP32 strip-sweep kernel: one fused time step of the vdW
// lattice Boltzmann scheme (arXiv:1307.6703, Sec. II) streamed through
// shared memory by TMA.
//
// Work decomposition.  The lattice is cut into column strips of W <= 120
// interior columns and row segments of up to SEG rows.  One CTA (256
// threads: two warp groups, one per row of a row pair, each with one thread
// per column of a 128-column window x0-4 .. x0+123) sweeps its segment
// upwards, two rows per iteration.  Every row of the previous state is read
// from HBM once by the TMA engine: a 3D tensor copy brings a pair of
// 128-column rows of all nine population planes into a ring of six pairs in
// shared memory (mbarrier-tracked), two pairs ahead of use.
//
// Iteration k (a = ya - 3 + 2k) runs four stages, separated by CTA barriers,
// each on two rows:
//   A  rows a, a+1     : propagated populations (pull), density n (n-hat on
//                        walls), raw momentum sum_i f_i c_i      -> n ring
//   B  rows a-1, a     : P = p^i - p^w (Eq. eqstate), L = lap n  -> P/L ring
//   C  rows a-2, a-1   : F = dP + kappa n dL + F_ext (Eq. force2), n u*
//                        (Eq. newvel), wall rule on wall rows   -> J/F ring
//   D  rows a-3, a-2   : grad n, div(n u*), equilibrium (Eq. eqfunc), forcing
//                        (Eqs. forceterm, coeff), BGK collision; store f*.
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

constexpr int kCols = 128;                 // TMA box width (columns x0-4 .. x0+123)
constexpr int kPairs = 6;                  // population ring, in pairs of rows
constexpr int kThreads = 256;              // warps 0-3: first row of a pair, 4-7: second
constexpr int kPairFloats = 9 * 2 * kCols;  // one pair of rows of all nine planes
constexpr unsigned kPairBytes = kPairFloats * sizeof(float);
constexpr uint32_t kWaitLimit = 1u << 22;

// Rings of row pairs.  A row y belongs to pair (y - y0) / 2 of a ring with
// origin y0: populations y0 = ya - 4, density ya - 3, P/L ya - 4, n u* and
// force ya - 5, chosen so that iteration k writes pair k of every ring.
struct __align__(128) SweepSmem {
  float pops[kPairs][9][2][kCols];
  float n[3][2][kCols];
  float P[2][2][kCols];
  float L[2][2][kCols];
  float Jx[2][2][kCols];
  float Jy[2][2][kCols];
  float Fx[2][2][kCols];
  float Fy[2][2][kCols];
  unsigned long long full[kPairs];
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

// Two rows (all nine planes, 128 columns) of the padded state into a ring slot.
__device__ __forceinline__ void tma_pair(const CUtensorMap *map, uint32_t dst, uint32_t bar, int xpad,
                                         int ypad) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kPairBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(xpad), "r"(ypad), "r"(0), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int dec(int s, int n) { return s == 0 ? n - 1 : s - 1; }
__device__ __forceinline__ int inc(int s, int n) { return s == n - 1 ? 0 : s + 1; }

// Row j (0, 1, 2 = r-1, r, r+1) of the three rows centred on this thread's
// row, in a ring of pairs whose pairs `lo` and `hi` hold them.
__device__ __forceinline__ const float *row_in(const float *ring, int pair_floats, int row_floats,
                                               int lo, int hi, int g, int j) {
  const int q = g + j;
  return ring + (q >> 1 ? hi : lo) * pair_floats + (q & 1) * row_floats;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 3)
sweep_step_kernel(const __grid_constant__ CUtensorMap tin, const SweepArgs A) {
  extern __shared__ unsigned char smem_raw[];
  SweepSmem &S = *reinterpret_cast<SweepSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));

  const int t = threadIdx.x & (kCols - 1);
  const int g = threadIdx.x >> 7;  // row within the pair
  const int strip = blockIdx.x, seg = blockIdx.y;
  const int x0 = strip * A.base_w + 4 * min(strip, A.extra);
  const int W = A.base_w + (strip < A.extra ? 4 : 0);
  const int ya = seg * A.seg_h;
  const int yb = min(A.ny, ya + A.seg_h);
  const int nx = A.nx, ny = A.ny;
  const bool walls = A.walls != 0;
  const int x = x0 - 4 + t;  // interior column of this thread (may be a halo column)
  const bool actA = t >= 1 && t <= W + 6;
  const bool actB = t >= 2 && t <= W + 5;
  const bool actC = t >= 3 && t <= W + 4;
  const bool actD = t >= 4 && t <= W + 3;
  const int kmax = (yb - ya + 5) >> 1;  // last iteration
  const int npairs = kmax + 2;          // rows ya-4 .. ya+2*kmax+3
  float sinx = 0.f;
  if (actC) sinx = A.sinx[x < 0 ? x + nx : (x >= nx ? x - nx : x)];

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPairs; ++s) mbar_init(smem_u32(&S.full[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int P = 0; P < min(kPairs, npairs); ++P)
      tma_pair(&tin, smem_u32(&S.pops[P][0][0][0]), smem_u32(&S.full[P]), x0, ya + 2 * P);
  }
  __syncthreads();
  mbar_wait(smem_u32(&S.full[0]), 0, A.err);

  const float *pops = &S.pops[0][0][0][0];
  constexpr int PF = kPairFloats, PR = 2 * kCols;  // pair / plane strides in pops
  float sx_prev = 0.f, sy_prev = 0.f;
  float acc_m = 0.f, acc_x = 0.f, acc_y = 0.f;
  int bad = 0;
  // ring slots of pair k (and neighbours) for the rings of 6, 3 and 2 pairs
  int s6 = 0, s3 = 0;

  for (int k = 0; k <= kmax; ++k) {
    const int s6m1 = dec(s6, kPairs), s6m2 = dec(s6m1, kPairs), s6p1 = inc(s6, kPairs);
    const int s3m1 = dec(s3, 3), s3m2 = dec(s3m1, 3);
    const int s2 = k & 1, s2m1 = s2 ^ 1;
    {
      const int P = k + 1;  // newest pair needed by this iteration
      mbar_wait(smem_u32(&S.full[s6p1]), (P / kPairs) & 1, A.err);
    }
    const int a = ya - 3 + 2 * k;
    const int rA = a + g, rB = a - 1 + g, rC = a - 2 + g, rD = a - 3 + g;

    // ------------------------------------------------ A: density, raw momentum
    float sx_new = 0.f, sy_new = 0.f;
    if (actA && (!walls || (rA >= 0 && rA <= ny - 1))) {
      const float *pm = row_in(pops, PF, kCols, s6, s6p1, g, 0);
      const float *p0 = row_in(pops, PF, kCols, s6, s6p1, g, 1);
      const float *pp = row_in(pops, PF, kCols, s6, s6p1, g, 2);
      const float f0 = p0[0 * PR + t], f1 = p0[1 * PR + t - 1], f3 = p0[3 * PR + t + 1];
      const float f2 = pm[2 * PR + t], f5 = pm[5 * PR + t - 1], f6 = pm[6 * PR + t + 1];
      const float f4 = pp[4 * PR + t], f7 = pp[7 * PR + t + 1], f8 = pp[8 * PR + t - 1];
      float n;
      if (walls && rA == 0) {
        n = p0[0 * PR + t] + p0[4 * PR + t] + p0[7 * PR + t] + p0[8 * PR + t] + f1 + f3 + f4 + f7 + f8;
      } else if (walls && rA == ny - 1) {
        n = p0[0 * PR + t] + p0[2 * PR + t] + p0[6 * PR + t] + p0[5 * PR + t] + f1 + f3 + f2 + f6 + f5;
      } else {
        n = (((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7))) + f8;
        sx_new = ((f1 - f3) + (f5 - f6)) + (f8 - f7);
        sy_new = ((f2 - f4) + (f5 + f6)) - (f7 + f8);
      }
      S.n[s3][g][t] = n;
    }
    __syncthreads();
    // The slot of pair k-3 is free (last used by iteration k-1): refill it.
    if (threadIdx.x == 0 && k >= 3 && k + 3 < npairs) {
      const int P = k + 3;  // slot (k+3) % 6 == (k-3) % 6
      tma_pair(&tin, smem_u32(pops + dec(s6m2, kPairs) * PF), smem_u32(&S.full[dec(s6m2, kPairs)]), x0,
               ya + 2 * P);
    }

    // ------------------------------------------------ B: P = p^i - p^w, L = lap n
    if (actB && rB >= ya - 2 && (!walls || (rB >= 0 && rB <= ny - 1))) {
      const float *nr = &S.n[0][0][0];
      const float *nm = row_in(nr, 2 * kCols, kCols, s3m1, s3, g, 0);
      const float *n0 = row_in(nr, 2 * kCols, kCols, s3m1, s3, g, 1);
      const float *np = row_in(nr, 2 * kCols, kCols, s3m1, s3, g, 2);
      if (walls && rB == 0) nm = np;
      if (walls && rB == ny - 1) np = nm;
      const float c = n0[t];
      const float lap = A.Q * ((n0[t + 1] + n0[t - 1]) + (np[t] + nm[t])) +
                        A.R * ((np[t + 1] + np[t - 1]) + (nm[t + 1] + nm[t - 1])) - A.four_QR * c;
      const float nT = c * A.T;
      const float pw = nT * __frcp_rn(1.0f - A.b * c) - A.a * c * c;
      S.P[s2][g][t] = nT - pw;
      S.L[s2][g][t] = lap;
    }
    __syncthreads();

    // ------------------------------------------------ C: force and n u*
    if (actC && rC >= ya - 1 && (!walls || (rC >= 0 && rC <= ny - 1))) {
      const float *Pr = &S.P[0][0][0], *Lr = &S.L[0][0][0];
      const float *Pm = row_in(Pr, 2 * kCols, kCols, s2m1, s2, g, 0);
      const float *P0 = row_in(Pr, 2 * kCols, kCols, s2m1, s2, g, 1);
      const float *Pp = row_in(Pr, 2 * kCols, kCols, s2m1, s2, g, 2);
      const float *Lm = row_in(Lr, 2 * kCols, kCols, s2m1, s2, g, 0);
      const float *L0 = row_in(Lr, 2 * kCols, kCols, s2m1, s2, g, 1);
      const float *Lp = row_in(Lr, 2 * kCols, kCols, s2m1, s2, g, 2);
      if (walls && rC == 0) { Pm = Pp; Lm = Lp; }
      if (walls && rC == ny - 1) { Pp = Pm; Lp = Lm; }
      const float dPx = A.N * (P0[t + 1] - P0[t - 1]) + A.M * ((Pp[t + 1] - Pp[t - 1]) + (Pm[t + 1] - Pm[t - 1]));
      const float dPy = A.N * (Pp[t] - Pm[t]) + A.M * ((Pp[t + 1] - Pm[t + 1]) + (Pp[t - 1] - Pm[t - 1]));
      const float dLx = A.N * (L0[t + 1] - L0[t - 1]) + A.M * ((Lp[t + 1] - Lp[t - 1]) + (Lm[t + 1] - Lm[t - 1]));
      const float dLy = A.N * (Lp[t] - Lm[t]) + A.M * ((Lp[t + 1] - Lm[t + 1]) + (Lp[t - 1] - Lm[t - 1]));
      // density of row rC: pair k-1 (+g) of the density ring
      const float n = S.n[s3m1][g][t];  // row rC: pair k-1, row g of the density ring
      const float kn = A.kappa * n;
      const float Fx = (dPx + kn * dLx) + A.A0 * sinx;
      const float Fy = dPy + kn * dLy;
      float sx = sx_prev, sy = sy_prev;
      if (walls && (rC == 0 || rC == ny - 1)) {
        const float *pm = row_in(pops, PF, kCols, s6m1, s6, g, 0);
        const float *p0 = row_in(pops, PF, kCols, s6m1, s6, g, 1);
        const float *pp = row_in(pops, PF, kCols, s6m1, s6, g, 2);
        float f[9];
        f[0] = p0[0 * PR + t]; f[1] = p0[1 * PR + t - 1]; f[3] = p0[3 * PR + t + 1];
        f[2] = pm[2 * PR + t]; f[5] = pm[5 * PR + t - 1]; f[6] = pm[6 * PR + t + 1];
        f[4] = pp[4 * PR + t]; f[7] = pp[7 * PR + t + 1]; f[8] = pp[8 * PR + t - 1];
        const bool top = rC != 0;
        wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
        sx = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
        sy = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
      }
      S.Jx[s2][g][t] = sx + 0.5f * Fx;
      S.Jy[s2][g][t] = sy + 0.5f * Fy;
      S.Fx[s2][g][t] = Fx;
      S.Fy[s2][g][t] = Fy;
    }
    sx_prev = sx_new;
    sy_prev = sy_new;
    __syncthreads();

    // ------------------------------------------------ D: collide and store
    if (actD && rD >= ya && rD < yb) {
      const bool bot_wall = walls && rD == 0, top_wall = walls && rD == ny - 1;
      const float *nr = &S.n[0][0][0];
      const float *nm = row_in(nr, 2 * kCols, kCols, s3m2, s3m1, g, 0);
      const float *n0 = row_in(nr, 2 * kCols, kCols, s3m2, s3m1, g, 1);
      const float *np = row_in(nr, 2 * kCols, kCols, s3m2, s3m1, g, 2);
      const float *Xr = &S.Jx[0][0][0], *Yr = &S.Jy[0][0][0];
      const float *Xm = row_in(Xr, 2 * kCols, kCols, s2m1, s2, g, 0);
      const float *X0 = row_in(Xr, 2 * kCols, kCols, s2m1, s2, g, 1);
      const float *Xp = row_in(Xr, 2 * kCols, kCols, s2m1, s2, g, 2);
      const float *Ym = row_in(Yr, 2 * kCols, kCols, s2m1, s2, g, 0);
      const float *Y0 = row_in(Yr, 2 * kCols, kCols, s2m1, s2, g, 1);
      const float *Yp = row_in(Yr, 2 * kCols, kCols, s2m1, s2, g, 2);
      float sgm = 1.f, sgp = 1.f;  // J_y is odd across a wall
      if (bot_wall) { nm = np; Xm = Xp; Ym = Yp; sgm = -1.f; }
      if (top_wall) { np = nm; Xp = Xm; Yp = Ym; sgp = -1.f; }
      const float n = n0[t];
      const float dnx = A.N * (n0[t + 1] - n0[t - 1]) + A.M * ((np[t + 1] - np[t - 1]) + (nm[t + 1] - nm[t - 1]));
      const float dny = A.N * (np[t] - nm[t]) + A.M * ((np[t + 1] - nm[t + 1]) + (np[t - 1] - nm[t - 1]));
      const float dJx = A.N * (X0[t + 1] - X0[t - 1]) + A.M * ((Xp[t + 1] - Xp[t - 1]) + (Xm[t + 1] - Xm[t - 1]));
      const float dJy = A.N * (sgp * Yp[t] - sgm * Ym[t]) +
                        A.M * ((sgp * Yp[t + 1] - sgm * Ym[t + 1]) + (sgp * Yp[t - 1] - sgm * Ym[t - 1]));
      const float divJ = dJx + dJy;
      const float Jx = X0[t], Jy = Y0[t];
      const float Fx = S.Fx[g ? s2 : s2m1][g ? 0 : 1][t];
      const float Fy = S.Fy[g ? s2 : s2m1][g ? 0 : 1][t];

      // rows rD-1 .. rD+1 lie one row above the pair grid of the population
      // ring: pairs (k-2, k-1) for the first row of a pair, (k-1, k) for the
      // second, entered at the opposite row.
      const int dlo = g ? s6m1 : s6m2, dhi = g ? s6 : s6m1;
      const float *pm = row_in(pops, PF, kCols, dlo, dhi, 1 - g, 0);
      const float *p0 = row_in(pops, PF, kCols, dlo, dhi, 1 - g, 1);
      const float *pp = row_in(pops, PF, kCols, dlo, dhi, 1 - g, 2);
      float f[9];
      f[0] = p0[0 * PR + t]; f[1] = p0[1 * PR + t - 1]; f[3] = p0[3 * PR + t + 1];
      f[2] = pm[2 * PR + t]; f[5] = pm[5 * PR + t - 1]; f[6] = pm[6 * PR + t + 1];
      f[4] = pp[4 * PR + t]; f[7] = pp[7 * PR + t + 1]; f[8] = pp[8 * PR + t - 1];
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
    s6 = s6p1;
    s3 = inc(s3, 3);
  }

  // CTA partial sums of the stored state (FP64, fixed order).
  double v[4] = {(double)acc_m, (double)acc_x, (double)acc_y, (double)bad};
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 4; ++c) S.red[c][threadIdx.x >> 5] = v[c];
  __syncthreads();
  if (threadIdx.x == 0) {
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

// cuTensorMapEncodeTiled through the runtime's driver entry point.
typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t sweep_make_map(void *base, int pitch, int ny, long long plane, CUtensorMap *map) {
  static encode_tiled_fn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (encode_tiled_fn)fn;
  }
  // 3D view (column, padded row, plane).  One box = the ring slot: kCols
  // columns x 2 rows x 9 planes, kPairBytes in all.
  const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)(ny + 8), 9};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)plane * 4};
  const cuuint32_t box[3] = {kCols, 2, 9};
  static_assert(kCols * 2 * 9 * sizeof(float) == kPairBytes, "TMA box must fill one ring slot");
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
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
