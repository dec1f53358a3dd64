// lb_device.cuh -- per-site physics of the vdW lattice Boltzmann step
// (arXiv:1307.6703, Sec. II) as device functions, and the tile kernel that
// fuses one whole time step.
//
// The formulas are evaluated in a fixed order (left to right as written, no
// reassociation).  Built with --fmad=false in FP64 this order makes the FP64
// path reproduce an independent IEEE implementation of the same formulas
// bit for bit; in FP32 the compiler may fuse multiply-adds.
//
// Units: lattice units, c_i in {0,+-1}^2, T0 = 1/3 (see include/lb.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbk {

// D2Q9 links: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

template <typename real_t>
struct Consts {
  static constexpr real_t T0 = real_t(1.0) / real_t(3.0);
  __host__ __device__ static constexpr real_t w(int i) {
    return i == 0 ? real_t(4.0) / real_t(9.0)
                  : (i < 5 ? real_t(1.0) / real_t(9.0) : real_t(1.0) / real_t(36.0));
  }
};

// Per-launch parameters (all derived quantities computed on the host).
template <typename real_t>
struct StepArgs {
  int nx, ny, walls;
  size_t plane;         // element stride between population planes
  int pitch;            // element stride between rows
  long long off;        // element offset of site (0, 0) within a plane
  real_t T, a, b, kappa, omega /* 1/tau */, g /* 1 - 1/(2 tau) */, th /* T0 - T */;
  real_t A0, u_bot, u_top;
  real_t N, M, Q, R, four_QR /* 4 (Q + R) */;
  const real_t *sinx;   // sin(2 pi x / lambda), device, [nx]
};

// ------------------------------------------------------------ site physics

// Eq. (eqfunc) with general T0.
template <typename real_t>
__device__ __forceinline__ void feq9(real_t n, real_t ux, real_t uy, real_t T, real_t *fe) {
  constexpr real_t T0 = Consts<real_t>::T0;
  const real_t uu = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const real_t cu = real_t(cx(i)) * ux + real_t(cy(i)) * uy;
    const real_t cc = real_t(cx(i) * cx(i) + cy(i) * cy(i));
    const real_t t1 = cu / T0;
    const real_t t2 = (cu * cu - T0 * uu) / (real_t(2.0) * T0 * T0);
    const real_t t3 = (T - T0) * (cc - real_t(2.0) * T0) / (real_t(2.0) * T0 * T0);
    fe[i] = Consts<real_t>::w(i) * n * (((real_t(1.0) + t1) + t2) + t3);
  }
}

// Eqs. (forceterm, coeff), A = 0.
template <typename real_t>
__device__ __forceinline__ void forcing9(real_t g, real_t th, real_t ux, real_t uy, real_t Fx,
                                         real_t Fy, real_t dnx, real_t dny, real_t divJ,
                                         real_t *Fi) {
  constexpr real_t T0 = Consts<real_t>::T0;
  const real_t u[2] = {ux, uy}, F[2] = {Fx, Fy}, dn[2] = {dnx, dny};
  real_t B[2], C[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++) {
    B[a] = g * F[a];
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const real_t delta = (a == b) ? real_t(1.0) : real_t(0.0);
      C[a][b] = g * ((u[a] * F[b] + F[a] * u[b]) + th * ((u[a] * dn[b] + u[b] * dn[a]) + delta * divJ));
    }
  }
  const real_t trC = C[0][0] + C[1][1];
#pragma unroll
  for (int i = 0; i < 9; i++) {
    const real_t c0 = real_t(cx(i)), c1 = real_t(cy(i));
    const real_t cB = c0 * B[0] + c1 * B[1];
    const real_t Ccc = ((C[0][0] * c0 * c0 + C[0][1] * c0 * c1) + C[1][0] * c1 * c0) + C[1][1] * c1 * c1;
    const real_t A = real_t(0.0);
    Fi[i] = Consts<real_t>::w(i) * ((A + cB / T0) + (Ccc - T0 * trC) / (real_t(2.0) * T0 * T0));
  }
}

// p^i - p^w, Eqs. (eqstate, force2).
template <typename real_t>
__device__ __forceinline__ real_t pdiff(real_t a, real_t b, real_t T, real_t n) {
  const real_t pw = (n * T) / (real_t(1.0) - b * n) - a * n * n;
  return n * T - pw;
}

// Eqs. (xstencil, laplstencil) on a 3x3 neighbourhood given in link order.
template <typename real_t>
__device__ __forceinline__ void grad9(const StepArgs<real_t> &A, const real_t *p, real_t &dx,
                                      real_t &dy) {
  dx = A.N * (p[1] - p[3]) + A.M * ((p[5] - p[6]) + (p[8] - p[7]));
  dy = A.N * (p[2] - p[4]) + A.M * ((p[5] - p[8]) + (p[6] - p[7]));
}
template <typename real_t>
__device__ __forceinline__ real_t lap9(const StepArgs<real_t> &A, const real_t *p) {
  return (A.Q * (((p[1] + p[2]) + p[3]) + p[4]) + A.R * (((p[5] + p[6]) + p[7]) + p[8])) -
         A.four_QR * p[0];
}

// Moving-wall rule of Sec. II for one wall node; f holds the propagated
// populations (unknown links are overwritten), g the node's own
// post-collision populations of the previous step.  Returns n-hat.
template <typename real_t>
__device__ __forceinline__ real_t nhat_of(bool top, const real_t *f, const real_t *g) {
  return top ? g[0] + g[2] + g[6] + g[5] + f[1] + f[3] + f[2] + f[6] + f[5]
             : g[0] + g[4] + g[7] + g[8] + f[1] + f[3] + f[4] + f[7] + f[8];
}
template <typename real_t>
__device__ __forceinline__ void wall_fill(bool top, real_t U, real_t Fx, real_t Fy, real_t nh,
                                          real_t *f) {
  const real_t h = real_t(0.5), q = real_t(0.25), two = real_t(2.0);
  if (!top) {
    f[0] = ((nh - (f[1] + f[3])) - two * ((f[4] + f[7]) + f[8])) + h * Fy;
    f[5] = ((f[7] - h * (f[1] - f[3])) - q * (Fx + Fy)) + h * nh * U;
    f[6] = ((f[8] + h * (f[1] - f[3])) + q * (Fx - Fy)) - h * nh * U;
    f[2] = f[4];
  } else {
    f[0] = ((nh - (f[1] + f[3])) - two * ((f[2] + f[6]) + f[5])) - h * Fy;
    f[8] = ((f[6] - h * (f[1] - f[3])) - q * (Fx - Fy)) + h * nh * U;
    f[7] = ((f[5] + h * (f[1] - f[3])) + q * (Fx + Fy)) - h * nh * U;
    f[4] = f[2];
  }
}

__device__ __forceinline__ int wrapi(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Propagation (pull): f_i(x, y) = f*_i(x - cx_i, y - cy_i).  Links coming
// from outside a wall are set to zero (the wall rule rebuilds them).  g
// receives the node's own stored populations (needed on wall rows).
template <typename real_t>
__device__ __forceinline__ void pull9(const real_t *__restrict__ fin, const StepArgs<real_t> &A,
                                      int x, int y, real_t *f, real_t *g) {
  const int xm = (x == 0) ? A.nx - 1 : x - 1;
  const int xp = (x == A.nx - 1) ? 0 : x + 1;
  const bool wl = A.walls != 0;
  const int ym = (y == 0) ? (wl ? -1 : A.ny - 1) : y - 1;
  const int yp = (y == A.ny - 1) ? (wl ? -1 : 0) : y + 1;
  const size_t P = A.plane;
  const size_t r0 = (size_t)(A.off + (long long)y * A.pitch);
  f[0] = fin[0 * P + r0 + x];
  f[1] = fin[1 * P + r0 + xm];
  f[3] = fin[3 * P + r0 + xp];
  if (ym >= 0) {
    const size_t rm = (size_t)(A.off + (long long)ym * A.pitch);
    f[2] = fin[2 * P + rm + x];
    f[5] = fin[5 * P + rm + xm];
    f[6] = fin[6 * P + rm + xp];
  } else {
    f[2] = f[5] = f[6] = real_t(0);
  }
  if (yp >= 0) {
    const size_t rp = (size_t)(A.off + (long long)yp * A.pitch);
    f[4] = fin[4 * P + rp + x];
    f[7] = fin[7 * P + rp + xp];
    f[8] = fin[8 * P + rp + xm];
  } else {
    f[4] = f[7] = f[8] = real_t(0);
  }
  if (wl && (y == 0 || y == A.ny - 1)) {
#pragma unroll
    for (int i = 0; i < 9; i++) g[i] = fin[i * P + r0 + x];
  }
}

// Density of the propagated state: sum_i f_i in bulk, n-hat on wall rows.
template <typename real_t>
__device__ __forceinline__ real_t density_at(const real_t *__restrict__ fin,
                                             const StepArgs<real_t> &A, int x, int y) {
  real_t f[9], g[9];
  pull9(fin, A, x, y, f, g);
  if (A.walls && (y == 0 || y == A.ny - 1)) return nhat_of(y != 0, f, g);
  return (((((((f[0] + f[1]) + f[2]) + f[3]) + f[4]) + f[5]) + f[6]) + f[7]) + f[8];
}

// Row read for a ghost row: even reflection about the wall rows (neutral
// wetting), clamped into range (clamped rows are never used), or periodic.
__device__ __forceinline__ int ghost_row(int y, int ny, int walls) {
  if (!walls) return wrapi(y, ny);
  if (y < 0) y = -y;
  if (y > ny - 1) y = 2 * (ny - 1) - y;
  return y < 0 ? 0 : (y > ny - 1 ? ny - 1 : y);
}

// ------------------------------------------------ the tile kernel (one step)
//
// One CTA owns a TX x TY tile of sites.  Shared memory holds the density on
// the tile plus a 3-site ring, p^i - p^w and lap n on a 2-site ring, and the
// force and n u* on a 1-site ring; populations are pulled straight from the
// previous state (L1/L2 serve the halo re-reads).
//
// MODE 0: full step, writes fout.  MODE 1: moments only (n, u*) into mom.

constexpr int TX = 32, TY = 8, TTHREADS = TX * TY;
constexpr int NXR3 = TX + 6, NYR3 = TY + 6;
constexpr int NXR2 = TX + 4, NYR2 = TY + 4;
constexpr int NXR1 = TX + 2, NYR1 = TY + 2;

template <typename real_t, int MODE, typename mom_t>
__global__ void __launch_bounds__(TTHREADS)
tile_step_kernel(const real_t *__restrict__ fin, real_t *__restrict__ fout,
                 mom_t *__restrict__ mom_n, mom_t *__restrict__ mom_ux,
                 mom_t *__restrict__ mom_uy, const StepArgs<real_t> A) {
  __shared__ real_t s_n[NYR3 * NXR3];
  __shared__ real_t s_P[NYR2 * NXR2], s_L[NYR2 * NXR2];
  __shared__ real_t s_Fx[NYR1 * NXR1], s_Fy[NYR1 * NXR1];
  __shared__ real_t s_Jx[NYR1 * NXR1], s_Jy[NYR1 * NXR1];

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = A.nx, ny = A.ny;
  const bool walls = A.walls != 0;

  // 1. density on tile + 3 (ghost rows: reflection or periodic image).
  for (int k = tid; k < NYR3 * NXR3; k += TTHREADS) {
    const int lx = k % NXR3, ly = k / NXR3;
    const int gx = wrapi(x0 + lx - 3, nx);
    const int gy = ghost_row(y0 + ly - 3, ny, A.walls);
    s_n[k] = density_at(fin, A, gx, gy);
  }
  __syncthreads();

  // 2. P = p^i - p^w and L = lap n on tile + 2.
  for (int k = tid; k < NYR2 * NXR2; k += TTHREADS) {
    const int lx = k % NXR2 + 1, ly = k / NXR2 + 1;  // centre in s_n coords
    real_t p[9];
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_n[(ly + cy(i)) * NXR3 + lx + cx(i)];
    s_L[k] = lap9(A, p);
    s_P[k] = pdiff(A.a, A.b, A.T, p[0]);
  }
  __syncthreads();

  // 3. F and n u* on tile + 1 (real rows; ghost rows by reflection below).
  for (int k = tid; k < NYR1 * NXR1; k += TTHREADS) {
    const int lx = k % NXR1 + 1, ly = k / NXR1 + 1;  // centre in s_P coords
    const int gy_raw = y0 + ly - 2;
    if (walls && (gy_raw < 0 || gy_raw > ny - 1)) continue;
    const int gx = wrapi(x0 + lx - 2, nx);
    const int gy = walls ? gy_raw : wrapi(gy_raw, ny);
    real_t p[9], dPx, dPy, dLx, dLy;
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_P[(ly + cy(i)) * NXR2 + lx + cx(i)];
    grad9(A, p, dPx, dPy);
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_L[(ly + cy(i)) * NXR2 + lx + cx(i)];
    grad9(A, p, dLx, dLy);
    const real_t n = s_n[(ly + 1) * NXR3 + lx + 1];
    const real_t Fx = (dPx + A.kappa * n * dLx) + A.A0 * A.sinx[gx];
    const real_t Fy = dPy + A.kappa * n * dLy;
    real_t f[9], g[9];
    pull9(fin, A, gx, gy, f, g);
    if (walls && (gy == 0 || gy == ny - 1)) {
      const bool top = (gy != 0);
      wall_fill(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
    }
    const real_t sx = ((((f[1] - f[3]) + f[5]) - f[6]) - f[7]) + f[8];
    const real_t sy = ((((f[2] - f[4]) + f[5]) + f[6]) - f[7]) - f[8];
    s_Fx[k] = Fx;
    s_Fy[k] = Fy;
    s_Jx[k] = sx + real_t(0.5) * Fx;
    s_Jy[k] = sy + real_t(0.5) * Fy;
  }
  __syncthreads();
  if (walls) {
    for (int k = tid; k < NYR1 * NXR1; k += TTHREADS) {
      const int lx = k % NXR1, ly = k / NXR1;
      const int gy = y0 + ly - 1;
      int src = -1;
      if (gy < 0) src = 2 * (0 - y0 + 1) - ly;                  // row -gy
      if (gy > ny - 1) src = 2 * ((ny - 1) - y0 + 1) - ly;      // mirror
      if (src >= 0 && src < NYR1) {
        s_Jx[k] = s_Jx[src * NXR1 + lx];
        s_Jy[k] = -s_Jy[src * NXR1 + lx];
      }
    }
    __syncthreads();
  }

  // 4. interior: gradients, u*, equilibrium, forcing, collision.
  {
    const int lx = tid % TX, ly = tid / TX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) return;
    const int c1 = (ly + 1) * NXR1 + lx + 1;   // in ring-1 arrays
    const real_t n = s_n[(ly + 3) * NXR3 + lx + 3];
    const real_t Jx = s_Jx[c1], Jy = s_Jy[c1];
    const real_t ux = Jx / n, uy = Jy / n;
    if constexpr (MODE == 1) {
      const size_t s = (size_t)gy * nx + gx;
      if (mom_n) mom_n[s] = (mom_t)n;
      if (mom_ux) mom_ux[s] = (mom_t)ux;
      if (mom_uy) mom_uy[s] = (mom_t)uy;
    } else {
    real_t p[9], dnx, dny, dJx, dJy, tmp;
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_n[(ly + 3 + cy(i)) * NXR3 + lx + 3 + cx(i)];
    grad9(A, p, dnx, dny);
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_Jx[(ly + 1 + cy(i)) * NXR1 + lx + 1 + cx(i)];
    grad9(A, p, dJx, tmp);
#pragma unroll
    for (int i = 0; i < 9; i++) p[i] = s_Jy[(ly + 1 + cy(i)) * NXR1 + lx + 1 + cx(i)];
    grad9(A, p, tmp, dJy);
    const real_t divJ = dJx + dJy;
    real_t f[9], g[9];
    pull9(fin, A, gx, gy, f, g);
    const real_t Fx = s_Fx[c1], Fy = s_Fy[c1];
    if (walls && (gy == 0 || gy == ny - 1)) {
      const bool top = (gy != 0);
      wall_fill(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
    }
    real_t fe[9], Fi[9];
    feq9(n, ux, uy, A.T, fe);
    forcing9(A.g, A.th, ux, uy, Fx, Fy, dnx, dny, divJ, Fi);
    const size_t s = (size_t)(A.off + (long long)gy * A.pitch + gx);
#pragma unroll
    for (int i = 0; i < 9; i++) fout[i * A.plane + s] = (f[i] - A.omega * (f[i] - fe[i])) + Fi[i];
    }
  }
}

// ------------------------------------------------------------------ init

// Counter-based SplitMix64 (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// f*_i = f_i^eq(n0, u0) evaluated in FP64, stored as real_t.  Threads run
// along x, blocks stride over rows (blockIdx.y); site s = y * nx + x is the
// noise counter and the index into the host fields.  With zero velocity
// (noise, or a density field alone) t1 = +-0 and t2 = +0 in feq9, so
// f^eq_i = (w_i n) (1 + t3_i) with the same roundings: the three isotropic
// factors 1 + t3 (rest, axes, diagonals) are evaluated once per thread by
// the same expression and each site costs two FP64 products per link
// class instead of feq9's divisions.
template <typename real_t>
__global__ void init_kernel(real_t *__restrict__ f, int nx, int ny, int pitch, long long plane,
                            long long off, int mode, uint64_t seed, double rho_mean, double amp,
                            const double *__restrict__ rho0, const double *__restrict__ ux0,
                            const double *__restrict__ uy0, double T) {
  constexpr double T0 = Consts<double>::T0;
  const bool at_rest = mode == 0 || (ux0 == nullptr && uy0 == nullptr);
  double iso[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double t3 = (T - T0) * (double(c) - 2.0 * T0) / (2.0 * T0 * T0);
    iso[c] = 1.0 + t3;
  }
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
      const size_t s = (size_t)y * nx + x;
      double n0, u = 0.0, v = 0.0;
      if (mode == 0) {
        const double U = (double)(splitmix64_at(seed, (uint64_t)s) >> 11) * 0x1.0p-53;
        n0 = rho_mean + amp * (2.0 * U - 1.0);
      } else {
        n0 = rho0[s];
        if (ux0) u = ux0[s];
        if (uy0) v = uy0[s];
      }
      double fe[9];
      if (at_rest) {
#pragma unroll
        for (int i = 0; i < 9; i++) fe[i] = Consts<double>::w(i) * n0 * iso[cx(i) * cx(i) + cy(i) * cy(i)];
      } else {
        feq9<double>(n0, u, v, T, fe);
      }
      const long long e = off + (long long)y * pitch + x;
#pragma unroll
      for (int i = 0; i < 9; i++) f[i * plane + e] = (real_t)fe[i];
    }
  }
}

// Grid of init_kernel: 256-thread blocks along x; up to 256 row blocks, so
// that a thread sets several rows.
inline dim3 init_grid(int nx, int ny) {
  const unsigned bx = (unsigned)((nx + 255) / 256);
  return dim3(bx < 64u ? bx : 64u, (unsigned)(ny < 256 ? ny : 256));
}

}  // namespace lbk
