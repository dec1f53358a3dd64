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
#include <cstddef>

#include <cuda.h>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbk {

namespace {

constexpr int kCols = 124;                  // TMA box width (columns x0-4 .. x0+119)
constexpr int kMaxW = kCols - 8;            // interior columns per strip
constexpr int kPairs = 5;                   // population ring, in pairs of rows
constexpr int kThreads = kCols;             // one thread per window column
constexpr int kSeg = 64;                    // rows per segment
constexpr int kPairFloats = 9 * 2 * kCols;  // one pair of rows of all nine planes
constexpr unsigned kPairBytes = kPairFloats * sizeof(float);
// Ring slots start on 128-byte boundaries (TMA destination alignment).
constexpr int kSlotFloats = ((kPairFloats * 4 + 127) / 128) * 128 / 4;
constexpr uint32_t kWaitLimit = 1u << 22;

// Rings of row pairs.  A row y belongs to pair (y - y0) / 2 of a ring with
// origin y0: populations y0 = ya - 4, density ya - 3, P/L ya - 4, n u*
// ya - 5, chosen so that iteration k writes pair k of every ring.  Each
// ring is long enough that no stage overwrites a slot another thread may
// still read without a barrier in between.
struct __align__(128) SweepSmem {
  float pops[kPairs][kSlotFloats];  // [slot][plane][row of pair][column] + padding
  // four pairs: stage A of iteration k+1 writes pair k+1 while stage D of
  // iteration k (no barrier in between) may still read pairs k-2 and k-1
  float n[4][2][kCols];
  float P[2][2][kCols];
  float L[2][2][kCols];
  float Jx[2][2][kCols];
  float Jy[2][2][kCols];
  unsigned long long full[kPairs];
};
static_assert(sizeof(float) * kPairs * kSlotFloats >= sizeof(double) * 4 * kThreads,
              "the end-of-kernel reduction reuses the population ring");
static_assert((kSlotFloats * sizeof(float)) % 128 == 0, "TMA destinations must be 128-byte aligned");
static_assert(offsetof(SweepSmem, pops) == 0, "the ring starts the (128-byte aligned) block");

// Row r (0 or 1) of a ring slot; plane q of that row starts q * 2 * kCols later.
__device__ __forceinline__ const float *pop_row(const SweepSmem &S, int slot, int r) {
  return &S.pops[slot][r * kCols];
}

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

// Two rows (all nine planes, kCols columns) of the padded state into a slot.
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

// x-derivative, y-derivative and Laplacian stencils of Eqs. (xstencil,
// laplstencil) at column t of row r1, rows r0 = y-1 and r2 = y+1.
struct Sten {
  float N, M, Q, R, four_QR;
};
__device__ __forceinline__ float sdx(const Sten &s, const float *r0, const float *r1, const float *r2, int t) {
  return s.N * (r1[t + 1] - r1[t - 1]) + s.M * ((r2[t + 1] - r2[t - 1]) + (r0[t + 1] - r0[t - 1]));
}
__device__ __forceinline__ float sdy(const Sten &s, const float *r0, const float *r2, int t) {
  return s.N * (r2[t] - r0[t]) + s.M * ((r2[t + 1] - r0[t + 1]) + (r2[t - 1] - r0[t - 1]));
}
__device__ __forceinline__ float slap(const Sten &s, const float *r0, const float *r1, const float *r2, int t) {
  return s.Q * ((r1[t + 1] + r1[t - 1]) + (r2[t] + r0[t])) +
         s.R * ((r2[t + 1] + r2[t - 1]) + (r0[t + 1] + r0[t - 1])) - s.four_QR * r1[t];
}

// Propagated populations of the site in column t of row r1 (pull).
__device__ __forceinline__ void pull(const float *r0, const float *r1, const float *r2, int t, float *f) {
  constexpr int PR = 2 * kCols;  // plane stride inside a ring slot
  f[0] = r1[0 * PR + t]; f[1] = r1[1 * PR + t - 1]; f[3] = r1[3 * PR + t + 1];
  f[2] = r0[2 * PR + t]; f[5] = r0[5 * PR + t - 1]; f[6] = r0[6 * PR + t + 1];
  f[4] = r2[4 * PR + t]; f[7] = r2[7 * PR + t + 1]; f[8] = r2[8 * PR + t - 1];
}

// One collision (Eqs. evoleq, eqfunc, forceterm, coeff) in the moment form
//   f*_i = (1 - omega) f_i + w_i E_i,
//   E_i = omega n [A_i + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2] + 3 c.B + 9/2 C:cc - 3/2 tr C,
// with the rest population taken as n minus the other eight.
__device__ __forceinline__ void collide(const SweepArgs &A, const float *f, float n, float Jx, float Jy,
                                        float Fx, float Fy, float dnx, float dny, float divJ, float *fs) {
  const float rn = __fdividef(1.0f, n);
  const float ux = Jx * rn, uy = Jy * rn;
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
  fs[1] = om1 * f[1] + w1 * (e_ax + symx + antx);
  fs[3] = om1 * f[3] + w1 * (e_ax + symx - antx);
  fs[2] = om1 * f[2] + w1 * (e_ax + symy + anty);
  fs[4] = om1 * f[4] + w1 * (e_ax + symy - anty);
  fs[5] = om1 * f[5] + w5 * (e_dg + sym5 + ant5);
  fs[7] = om1 * f[7] + w5 * (e_dg + sym5 - ant5);
  fs[6] = om1 * f[6] + w5 * (e_dg + sym6 + ant6);
  fs[8] = om1 * f[8] + w5 * (e_dg + sym6 - ant6);
  // Collision conserves the site's mass exactly (A = 0, sum f^eq = n); the
  // remainder form keeps rounded weights from biasing the mass.
  fs[0] = n - (((fs[1] + fs[3]) + (fs[2] + fs[4])) + ((fs[5] + fs[7]) + (fs[6] + fs[8])));
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 4)
sweep_step_kernel(const __grid_constant__ CUtensorMap tin, const SweepArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SweepSmem &S = *reinterpret_cast<SweepSmem *>(smem_raw);

  const int t = threadIdx.x;
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
  const Sten st{A.N, A.M, A.Q, A.R, A.four_QR};
  float sinx = 0.f;
  if (actC) sinx = A.sinx[x < 0 ? x + nx : (x >= nx ? x - nx : x)];
  float *col = A.fout + A.off + x;  // f* of this column at interior row 0
  const int pitch = A.pitch, plane = (int)A.plane;
  const int gx = (x < 4) ? nx : ((x >= nx - 4) ? -nx : 0);  // periodic image column

  // TMA writes need 128-byte aligned destinations: refuse to run otherwise.
  if (smem_u32(&S.pops[0][0]) & 127u) {
    if (t == 0) atomicOr(A.err, 2);
    return;
  }
  if (t == 0) {
    for (int s = 0; s < kPairs; ++s) mbar_init(smem_u32(&S.full[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int P = 0; P < min(kPairs, npairs); ++P)
      tma_pair(&tin, smem_u32(pop_row(S, P, 0)), smem_u32(&S.full[P]), x0, ya + 2 * P);
  }
  __syncthreads();
  mbar_wait(smem_u32(&S.full[0]), 0, A.err);

  float sxa[2] = {0.f, 0.f}, sya[2] = {0.f, 0.f};  // raw momentum of rows a-2, a-1 (from last A)
  float Fx_prev = 0.f, Fy_prev = 0.f;              // force of row a-3 (from last C)
  float acc_m = 0.f, acc_x = 0.f, acc_y = 0.f;
  int bad = 0;
  int s5 = 0, s3 = 0;
  uint32_t par = 0;  // phase parity of pair k+1

  for (int k = 0; k <= kmax; ++k) {
    const int s5m1 = dec(s5, kPairs), s5m2 = dec(s5m1, kPairs), s5p1 = inc(s5, kPairs);
    const int s3m1 = (s3 + 3) & 3, s3m2 = (s3 + 2) & 3;  // density ring: 4 pairs
    const int s2 = k & 1, s2m1 = s2 ^ 1;
    mbar_wait(smem_u32(&S.full[s5p1]), par, A.err);  // newest pair needed: k+1
    if (s5p1 == kPairs - 1) par ^= 1u;
    const int a = ya - 3 + 2 * k;

    // ---------------------------------------- A: rows a, a+1 -- n, raw momentum
    {
      const float *q0 = pop_row(S, s5, 0), *q1 = pop_row(S, s5, 1);    // rows a-1, a
      const float *q2 = pop_row(S, s5p1, 0), *q3 = pop_row(S, s5p1, 1);  // rows a+1, a+2
      float sx_new[2] = {0.f, 0.f}, sy_new[2] = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int y = a + j;
        const float *r0 = j ? q1 : q0, *r1 = j ? q2 : q1, *r2 = j ? q3 : q2;
        if (actA && (!walls || (y >= 0 && y <= ny - 1))) {
          float f[9];
          pull(r0, r1, r2, t, f);
          float n;
          constexpr int PR = 2 * kCols;
          if (walls && y == 0) {
            n = r1[0 * PR + t] + r1[4 * PR + t] + r1[7 * PR + t] + r1[8 * PR + t] + f[1] + f[3] + f[4] + f[7] + f[8];
          } else if (walls && y == ny - 1) {
            n = r1[0 * PR + t] + r1[2 * PR + t] + r1[6 * PR + t] + r1[5 * PR + t] + f[1] + f[3] + f[2] + f[6] + f[5];
          } else {
            n = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
            sx_new[j] = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
            sy_new[j] = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
          }
          S.n[s3][j][t] = n;
        }
      }
      __syncthreads();
      // The slot of pair k-3 is free (last used by iteration k-1): refill it
      // with pair k+2.
      if (t == 0 && k >= 3 && k + 2 < npairs) {
        const int slot = dec(s5m2, kPairs);
        tma_pair(&tin, smem_u32(pop_row(S, slot, 0)), smem_u32(&S.full[slot]), x0, ya + 2 * (k + 2));
      }

      // -------------------------------------- B: rows a-1, a -- P, lap n
      {
        const float *n0 = S.n[s3m1][0], *n1 = S.n[s3m1][1];  // rows a-2, a-1
        const float *n2 = S.n[s3][0], *n3 = S.n[s3][1];      // rows a, a+1
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int y = a - 1 + j;
          const float *r0 = j ? n1 : n0, *r1 = j ? n2 : n1, *r2 = j ? n3 : n2;
          if (actB && y >= ya - 2 && (!walls || (y >= 0 && y <= ny - 1))) {
            if (walls && y == 0) r0 = r2;
            if (walls && y == ny - 1) r2 = r0;
            const float c = r1[t];
            const float nT = c * A.T;
            const float pw = nT * __fdividef(1.0f, 1.0f - A.b * c) - A.a * c * c;
            S.P[s2][j][t] = nT - pw;
            S.L[s2][j][t] = slap(st, r0, r1, r2, t);
          }
        }
      }
      __syncthreads();

      // -------------------------------------- C: rows a-2, a-1 -- F, n u*
      float Fx_cur[2] = {0.f, 0.f}, Fy_cur[2] = {0.f, 0.f};
      {
        const float *P0 = S.P[s2m1][0], *P1 = S.P[s2m1][1], *P2 = S.P[s2][0], *P3 = S.P[s2][1];
        const float *L0 = S.L[s2m1][0], *L1 = S.L[s2m1][1], *L2 = S.L[s2][0], *L3 = S.L[s2][1];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int y = a - 2 + j;
          if (!(actC && y >= ya - 1 && (!walls || (y >= 0 && y <= ny - 1)))) continue;
          const float *p0 = j ? P1 : P0, *p1 = j ? P2 : P1, *p2 = j ? P3 : P2;
          const float *l0 = j ? L1 : L0, *l1 = j ? L2 : L1, *l2 = j ? L3 : L2;
          if (walls && y == 0) { p0 = p2; l0 = l2; }
          if (walls && y == ny - 1) { p2 = p0; l2 = l0; }
          const float n = S.n[s3m1][j][t];
          const float kn = A.kappa * n;
          const float Fx = (sdx(st, p0, p1, p2, t) + kn * sdx(st, l0, l1, l2, t)) + A.A0 * sinx;
          const float Fy = sdy(st, p0, p2, t) + kn * sdy(st, l0, l2, t);
          float sx = sxa[j], sy = sya[j];
          if (walls && (y == 0 || y == ny - 1)) {
            // populations of rows y-1 .. y+1: pairs k-1 and k of the ring
            const float *w0 = pop_row(S, s5m1, 0), *w1 = pop_row(S, s5m1, 1);
            const float *w2 = pop_row(S, s5, 0), *w3 = pop_row(S, s5, 1);
            float f[9];
            pull(j ? w1 : w0, j ? w2 : w1, j ? w3 : w2, t, f);
            const bool top = y != 0;
            wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
            sx = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
            sy = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
          }
          S.Jx[s2][j][t] = sx + 0.5f * Fx;
          S.Jy[s2][j][t] = sy + 0.5f * Fy;
          Fx_cur[j] = Fx;
          Fy_cur[j] = Fy;
        }
      }
      sxa[0] = sx_new[0]; sxa[1] = sx_new[1];
      sya[0] = sy_new[0]; sya[1] = sy_new[1];
      __syncthreads();

      // -------------------------------------- D: rows a-3, a-2 -- collide, store
      {
        const float *n0 = S.n[s3m2][0], *n1 = S.n[s3m2][1], *n2 = S.n[s3m1][0], *n3 = S.n[s3m1][1];
        const float *X0 = S.Jx[s2m1][0], *X1 = S.Jx[s2m1][1], *X2 = S.Jx[s2][0], *X3 = S.Jx[s2][1];
        const float *Y0 = S.Jy[s2m1][0], *Y1 = S.Jy[s2m1][1], *Y2 = S.Jy[s2][0], *Y3 = S.Jy[s2][1];
        // population rows a-4 .. a-1: pair k-2 row 1, pair k-1 rows 0, 1, pair k row 0
        const float *q0p = pop_row(S, s5m2, 1), *q1p = pop_row(S, s5m1, 0);
        const float *q2p = pop_row(S, s5m1, 1), *q3p = pop_row(S, s5, 0);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int y = a - 3 + j;
          if (!(actD && y >= ya && y < yb)) continue;
          const float *m0 = j ? n1 : n0, *m1 = j ? n2 : n1, *m2 = j ? n3 : n2;
          const float *x0p = j ? X1 : X0, *x1p = j ? X2 : X1, *x2p = j ? X3 : X2;
          const float *y0p = j ? Y1 : Y0, *y1p = j ? Y2 : Y1, *y2p = j ? Y3 : Y2;
          const float Fx = j ? Fx_cur[0] : Fx_prev, Fy = j ? Fy_cur[0] : Fy_prev;
          const bool bot = walls && y == 0, top = walls && y == ny - 1;
          float dJy;
          if (bot || top) {
            // mirror rows across the wall: n and J_x even, J_y odd
            float sgm = 1.f, sgp = 1.f;
            if (bot) { m0 = m2; x0p = x2p; y0p = y2p; sgm = -1.f; }
            if (top) { m2 = m0; x2p = x0p; y2p = y0p; sgp = -1.f; }
            dJy = st.N * (sgp * y2p[t] - sgm * y0p[t]) +
                  st.M * ((sgp * y2p[t + 1] - sgm * y0p[t + 1]) + (sgp * y2p[t - 1] - sgm * y0p[t - 1]));
          } else {
            dJy = sdy(st, y0p, y2p, t);
          }
          const float n = m1[t];
          const float dnx = sdx(st, m0, m1, m2, t), dny = sdy(st, m0, m2, t);
          const float divJ = sdx(st, x0p, x1p, x2p, t) + dJy;
          const float Jx = x1p[t], Jy = y1p[t];
          float f[9], fs[9];
          pull(j ? q1p : q0p, j ? q2p : q1p, j ? q3p : q2p, t, f);
          if (bot || top) wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
          collide(A, f, n, Jx, Jy, Fx, Fy, dnx, dny, divJ, fs);

          float *o = col + (long long)y * pitch;
#pragma unroll
          for (int q = 0; q < 9; ++q) o[q * plane] = fs[q];
          const int gy = walls ? 0 : ((y < 4) ? ny : ((y >= ny - 4) ? -ny : 0));
          if (gx != 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) o[q * plane + gx] = fs[q];
          }
          if (gy != 0) {
            float *oy = o + (long long)gy * pitch;
#pragma unroll
            for (int q = 0; q < 9; ++q) oy[q * plane] = fs[q];
            if (gx != 0) {
#pragma unroll
              for (int q = 0; q < 9; ++q) oy[q * plane + gx] = fs[q];
            }
          }
          // Mass and momentum of the stored site: sum f* = n (by
          // construction), sum f* c = n u* + F/2 (identity of the collision).
          if (!(n > 0.f && n < A.nmax && fabsf(Jx) + fabsf(Jy) < 3.0e38f)) bad = 1;
          acc_m += n;
          acc_x += Jx + 0.5f * Fx;
          acc_y += Jy + 0.5f * Fy;
        }
      }
      Fx_prev = Fx_cur[1];
      Fy_prev = Fy_cur[1];
    }
    s5 = s5p1;
    s3 = (s3 + 1) & 3;
  }

  // CTA partial sums of the stored state (FP64, fixed order).  Every TMA
  // copy has been waited for, so the population ring is free for them.
  double *red = reinterpret_cast<double *>(&S.pops[0][0]);
  __syncthreads();
  red[0 * kThreads + t] = (double)acc_m;
  red[1 * kThreads + t] = (double)acc_x;
  red[2 * kThreads + t] = (double)acc_y;
  red[3 * kThreads + t] = (double)bad;
  __syncthreads();
  if (t == 0) {
    double *out = A.partials + 4 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    for (int q = 0; q < 4; ++q) {
      double sum = 0.0;
      for (int i = 0; i < kThreads; ++i) sum += red[q * kThreads + i];
      out[q] = sum;
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

void sweep_plan(int nx, int ny, int *nstrips, int *base_w, int *extra, int *seg_h, int *nseg) {
  *nstrips = (nx + kMaxW - 1) / kMaxW;
  *base_w = 4 * (nx / (4 * *nstrips));
  *extra = (nx - *base_w * *nstrips) / 4;
  *seg_h = ny < kSeg ? ny : kSeg;
  *nseg = (ny + *seg_h - 1) / *seg_h;
}

cudaError_t sweep_prepare(size_t *smem_bytes) {
  *smem_bytes = sizeof(SweepSmem);
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
