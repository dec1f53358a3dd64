/*
 * lb_oracle.c -- plain FP64 CPU oracle of the lattice Boltzmann time step of
 * Coclite, Gonnella & Lamura, "Pattern formation in liquid-vapor systems
 * under periodic potential and shear" (arXiv:1307.6703).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; the
 * GPU product path never calls it.
 *
 * What it computes, in the paper's order (Sec. II):
 *   Eq. (evoleq)   f_i(r+c_i, t+1) - f_i(r,t) = -(1/tau)[f_i - f_i^eq] + F_i
 *   Eq. (eqfunc)   Hermite 2nd-order equilibrium with the (T - T0) term
 *   Eq. (newvel)   n u* = sum_i f_i c_i + F/2
 *   Eq. (periodicforce)  F_ext = (A0 sin(2 pi x / lambda), 0)
 *   Eqs. (forceterm, coeff)  F_i = w_i [A + B.c/T0 + C:(cc - T0 I)/(2 T0^2)]
 *                  A = 0, B = g F, C = g{uF + Fu + (T0-T)[u dn + dn u + I div(n u)]}
 *                  g = 1 - 1/(2 tau)
 *   Eq. (eqstate)  p^w = n T / (1 - b n) - a n^2  (vdW; the paper's 3nT/(3-n)
 *                  - 9/8 n^2 is b = 1/3, a = 9/8 in its own units)
 *   Eq. (force2)   F_int = d(p^i - p^w) + kappa n d(lap n),  p^i = n T
 *   Eqs. (xstencil, laplstencil)  isotropic 3x3 stencils (N, M), (Q, R)
 *                  with 2N + 4M = 1 and Q + 2R = 1
 *   Sec. II, moving walls: unknown links after propagation, the independent
 *                  rest population f0 and the wall density n-hat.
 *
 * Units (readings of the paper, listed in the design notes):
 *   lattice units, dx = dt = 1, c_i in {0, +-1}^2, reference temperature
 *   T0 = 1/3.  The paper's own units (dt = sqrt(3)/3, |e| = sqrt(3), T0 = 1)
 *   map onto these by T -> T/3, a -> a/3, kappa -> kappa/3, with b, n, tau
 *   (in steps), lengths and A0, shear rate, velocities (in dx/dt) unchanged.
 *   The (1 - T) factor of C becomes (T0 - T).
 *
 * State convention: the stored populations are the post-collision,
 * not-yet-propagated values f*(r, t-1).  One step pulls them along the links
 * (periodic in x; periodic in y unless walls are on), rebuilds the wall links,
 * collides and stores f*(r, t).  The wall density n-hat uses the wall node's
 * own post-collision f*_0, f*_4, f*_7, f*_8 (bottom) or f*_0, f*_2, f*_6, f*_5
 * (top) of the previous step, which are exactly the stored values.
 *
 * Floating point: every formula below is evaluated left to right exactly as
 * written (C evaluation order, no reassociation, built with
 * -ffp-contract=off so that no multiply-add is fused).  The order is part of
 * the specification of the FP64 parity mode.
 *
 * Parallelism: the site loops may run under OpenMP; every site is computed
 * independently, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t nx, ny;      /* columns (periodic x), rows                        */
  int32_t walls;       /* 1: moving walls on rows 0 and ny-1; 0: periodic y */
  int32_t nthreads;    /* OpenMP threads (<= 0: library default)             */
  double a, b;         /* vdW constants in lattice units                     */
  double T;            /* temperature (lattice units, T0 = 1/3)              */
  double kappa;        /* interface (square-gradient) coefficient            */
  double tau;          /* relaxation time in steps                           */
  double A0, lambda;   /* periodic force amplitude and wavelength            */
  double u_bot, u_top; /* wall x-velocities                                  */
  double N, Q;         /* stencil parameters; M = (1-2N)/4, R = (1-Q)/2      */
} orc_params;

/* D2Q9 links: 0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE (Sec. II). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#define T0 (1.0 / 3.0)

static double weight(int i) {
  if (i == 0) return 4.0 / 9.0;
  if (i < 5) return 1.0 / 9.0;
  return 1.0 / 36.0;
}

static int wrap(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

/* ---------------------------------------------------------------- pieces */

/* Eq. (eqfunc), general T0:
 * f_i^eq = w_i n [1 + c.u/T0 + ((c.u)^2 - T0 u.u)/(2 T0^2)
 *                 + (T - T0)(c.c - 2 T0)/(2 T0^2)]                          */
void orc_feq(double n, double ux, double uy, double T, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < 9; i++) {
    double cu = CX[i] * ux + CY[i] * uy;
    double cc = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
    double t1 = cu / T0;
    double t2 = (cu * cu - T0 * uu) / (2.0 * T0 * T0);
    double t3 = (T - T0) * (cc - 2.0 * T0) / (2.0 * T0 * T0);
    feq[i] = weight(i) * n * (((1.0 + t1) + t2) + t3);
  }
}

/* Eqs. (forceterm, coeff), A = 0:
 * B = g F,  C_ab = g{u_a F_b + F_a u_b + (T0 - T)[u_a dn_b + u_b dn_a
 *                                                  + delta_ab div(n u*)]}
 * F_i = w_i [A + c.B/T0 + (C:cc - T0 tr C)/(2 T0^2)]                        */
void orc_forcing(double tau, double T, double ux, double uy, double Fx,
                 double Fy, double dnx, double dny, double divJ, double *Fi) {
  double g = 1.0 - 1.0 / (2.0 * tau);
  double th = T0 - T;
  double u[2] = {ux, uy}, F[2] = {Fx, Fy}, dn[2] = {dnx, dny};
  double B[2], C[2][2];
  for (int a = 0; a < 2; a++) {
    B[a] = g * F[a];
    for (int b = 0; b < 2; b++) {
      double delta = (a == b) ? 1.0 : 0.0;
      C[a][b] = g * ((u[a] * F[b] + F[a] * u[b]) +
                     th * ((u[a] * dn[b] + u[b] * dn[a]) + delta * divJ));
    }
  }
  double trC = C[0][0] + C[1][1];
  for (int i = 0; i < 9; i++) {
    double c[2] = {(double)CX[i], (double)CY[i]};
    double cB = c[0] * B[0] + c[1] * B[1];
    double Ccc = ((C[0][0] * c[0] * c[0] + C[0][1] * c[0] * c[1]) +
                  C[1][0] * c[1] * c[0]) + C[1][1] * c[1] * c[1];
    double A = 0.0;
    Fi[i] = weight(i) * ((A + cB / T0) + (Ccc - T0 * trC) / (2.0 * T0 * T0));
  }
}

/* Eq. (eqstate) and the ideal pressure: P = p^i - p^w. */
double orc_pressure_diff(double a, double b, double T, double n) {
  double pw = (n * T) / (1.0 - b * n) - a * n * n;
  return n * T - pw;
}

/* Eqs. (xstencil, laplstencil) on the 3x3 neighbourhood phi[9] given in link
 * order (phi[0] centre, phi[i] at r + c_i).  The y derivative is the
 * transposed x stencil, oriented so that d_y(y) = +1.                       */
void orc_stencils(double N, double Q, const double *phi, double *dx,
                  double *dy, double *lap) {
  double M = (1.0 - 2.0 * N) / 4.0;
  double R = (1.0 - Q) / 2.0;
  *dx = N * (phi[1] - phi[3]) + M * ((phi[5] - phi[6]) + (phi[8] - phi[7]));
  *dy = N * (phi[2] - phi[4]) + M * ((phi[5] - phi[8]) + (phi[6] - phi[7]));
  *lap = (Q * (((phi[1] + phi[2]) + phi[3]) + phi[4]) +
          R * (((phi[5] + phi[6]) + phi[7]) + phi[8])) -
         (4.0 * (Q + R)) * phi[0];
}

/* Moving-wall rule of Sec. II for one wall node (general wall velocity U;
 * the paper's -n gammadot L_y / 4 is + n U / 2 with U = -gammadot L_y / 2).
 * f[9] holds the propagated populations (unknown links ignored), g[9] the
 * node's own post-collision populations of the previous step.  On return
 * f[] holds the completed populations and *nhat the wall density.
 * top = 0: lower wall (unknown 2, 5, 6); top = 1: upper wall, the mirror
 * image y -> -y (unknown 4, 8, 7).                                          */
void orc_wall(int top, double U, double Fx, double Fy, double *f,
              const double *g, double *nhat) {
  double nh;
  if (!top) {
    nh = g[0] + g[4] + g[7] + g[8] + f[1] + f[3] + f[4] + f[7] + f[8];
    f[0] = ((nh - (f[1] + f[3])) - 2.0 * ((f[4] + f[7]) + f[8])) + 0.5 * Fy;
    f[5] = ((f[7] - 0.5 * (f[1] - f[3])) - 0.25 * (Fx + Fy)) + 0.5 * nh * U;
    f[6] = ((f[8] + 0.5 * (f[1] - f[3])) + 0.25 * (Fx - Fy)) - 0.5 * nh * U;
    f[2] = f[4];
  } else {
    nh = g[0] + g[2] + g[6] + g[5] + f[1] + f[3] + f[2] + f[6] + f[5];
    f[0] = ((nh - (f[1] + f[3])) - 2.0 * ((f[2] + f[6]) + f[5])) - 0.5 * Fy;
    f[8] = ((f[6] - 0.5 * (f[1] - f[3])) - 0.25 * (Fx - Fy)) + 0.5 * nh * U;
    f[7] = ((f[5] + 0.5 * (f[1] - f[3])) + 0.25 * (Fx + Fy)) - 0.5 * nh * U;
    f[4] = f[2];
  }
  *nhat = nh;
}

/* Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output k of
 * the stream seeded with s is mix(s + (k+1) * 0x9E3779B97F4A7C15).         */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Noisy uniform density: n0 = rho_mean + amp (2U - 1), U in [0, 1) from the
 * top 53 bits of output k = y*nx + x.                                       */
void orc_noise_field(int nx, int ny, uint64_t seed, double rho_mean,
                     double amp, double *n0) {
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      uint64_t k = (uint64_t)y * (uint64_t)nx + (uint64_t)x;
      double U = (double)(splitmix64_at(seed, k) >> 11) * 0x1.0p-53;
      n0[(size_t)y * nx + x] = rho_mean + amp * (2.0 * U - 1.0);
    }
}

/* Initial state: f*_i = f_i^eq(n0, u0) with no force correction.  ux0, uy0
 * may be NULL (fluid at rest).                                              */
void orc_init(const orc_params *p, const double *n0, const double *ux0,
              const double *uy0, double *f) {
  size_t S = (size_t)p->nx * p->ny;
  for (size_t s = 0; s < S; s++) {
    double feq[9];
    orc_feq(n0[s], ux0 ? ux0[s] : 0.0, uy0 ? uy0[s] : 0.0, p->T, feq);
    for (int i = 0; i < 9; i++) f[i * S + s] = feq[i];
  }
}

/* --------------------------------------------------------- the full step */

typedef struct {
  int nx, ny;
  double *fp;          /* propagated + wall-completed populations [9][ny][nx] */
  double *n;           /* density, rows -2 .. ny+1   [(ny+4)][nx]             */
  double *P, *L;       /* p^i - p^w and lap n, rows -1 .. ny  [(ny+2)][nx]    */
  double *Fx, *Fy;     /* total force, rows 0 .. ny-1                         */
  double *Jx, *Jy;     /* n u*, rows -1 .. ny  [(ny+2)][nx]                   */
  double *sinx;        /* sin(2 pi x / lambda)                                */
} work_t;

static int work_alloc(work_t *w, int nx, int ny) {
  size_t S = (size_t)nx * ny;
  w->nx = nx;
  w->ny = ny;
  w->fp = malloc(9 * S * sizeof(double));
  w->n = malloc((size_t)(ny + 4) * nx * sizeof(double));
  w->P = malloc((size_t)(ny + 2) * nx * sizeof(double));
  w->L = malloc((size_t)(ny + 2) * nx * sizeof(double));
  w->Fx = malloc(S * sizeof(double));
  w->Fy = malloc(S * sizeof(double));
  w->Jx = malloc((size_t)(ny + 2) * nx * sizeof(double));
  w->Jy = malloc((size_t)(ny + 2) * nx * sizeof(double));
  w->sinx = malloc((size_t)nx * sizeof(double));
  return w->fp && w->n && w->P && w->L && w->Fx && w->Fy && w->Jx && w->Jy &&
         w->sinx;
}

static void work_free(work_t *w) {
  free(w->fp); free(w->n); free(w->P); free(w->L); free(w->Fx);
  free(w->Fy); free(w->Jx); free(w->Jy); free(w->sinx);
}

/* Extended-row accessors (row y may lie outside 0 .. ny-1). */
#define NEXT(w, x, y) ((w)->n[(size_t)((y) + 2) * (w)->nx + (x)])
#define PEXT(w, x, y) ((w)->P[(size_t)((y) + 1) * (w)->nx + (x)])
#define LEXT(w, x, y) ((w)->L[(size_t)((y) + 1) * (w)->nx + (x)])
#define JXE(w, x, y) ((w)->Jx[(size_t)((y) + 1) * (w)->nx + (x)])
#define JYE(w, x, y) ((w)->Jy[(size_t)((y) + 1) * (w)->nx + (x)])

/* Gather the 3x3 neighbourhood of (x, y) of an extended field in link
 * order; x wraps, y must lie inside the stored rows.                        */
static void gather(const double *base, int nx, int row0, int x, int y,
                   double *phi) {
  for (int i = 0; i < 9; i++) {
    int xx = wrap(x + CX[i], nx);
    int yy = y + CY[i] + row0;
    phi[i] = base[(size_t)yy * nx + xx];
  }
}

/* Steps 1-8 of one update: propagate, density (n-hat on walls), P and L,
 * forces, wall rule, n u*.  Fills w from the stored state f.               */
static void prepare(const orc_params *p, const double *f, work_t *w) {
  const int nx = p->nx, ny = p->ny;
  const size_t S = (size_t)nx * ny;
  const int walls = p->walls;
  const double kappa = p->kappa;
  int nt = p->nthreads;
#ifdef _OPENMP
  if (nt <= 0) nt = omp_get_max_threads();
#else
  (void)nt;
#endif

  for (int x = 0; x < nx; x++)
    w->sinx[x] = (p->lambda != 0.0)
                     ? sin((6.283185307179586 * (double)x) / p->lambda)
                     : 0.0;

  /* 1. propagation: f_i(r) = f*_i(r - c_i); links from outside a wall are
   *    left as NaN and completed by the wall rule.  2. density.             */
#pragma omp parallel for num_threads(nt) if (nt > 1)
  for (int y = 0; y < ny; y++) {
    for (int x = 0; x < nx; x++) {
      double fl[9], g[9];
      size_t s = (size_t)y * nx + x;
      for (int i = 0; i < 9; i++) {
        int xs = wrap(x - CX[i], nx);
        int ys = y - CY[i];
        if (walls && (ys < 0 || ys >= ny)) {
          fl[i] = NAN;
        } else {
          ys = wrap(ys, ny);
          fl[i] = f[i * S + (size_t)ys * nx + xs];
        }
        g[i] = f[i * S + s];
      }
      double n;
      if (walls && (y == 0 || y == ny - 1)) {
        /* n-hat of the wall rule; the completed links come later, once F
         * is known.                                                         */
        if (y == 0)
          n = g[0] + g[4] + g[7] + g[8] + fl[1] + fl[3] + fl[4] + fl[7] + fl[8];
        else
          n = g[0] + g[2] + g[6] + g[5] + fl[1] + fl[3] + fl[2] + fl[6] + fl[5];
      } else {
        n = 0.0;
        for (int i = 0; i < 9; i++) n = n + fl[i];
        /* 0.0 + f0 == f0 exactly, so this is ((f0 + f1) + f2) + ... */
      }
      for (int i = 0; i < 9; i++) w->fp[i * S + s] = fl[i];
      NEXT(w, x, y) = n;
    }
  }

  /* 3. density on the ghost rows -2, -1, ny, ny+1: even reflection about
   *    the wall rows (neutral wetting, a . grad n = 0), else periodic.     */
  for (int k = 1; k <= 2; k++)
    for (int x = 0; x < nx; x++) {
      if (walls) {
        NEXT(w, x, -k) = NEXT(w, x, k);
        NEXT(w, x, ny - 1 + k) = NEXT(w, x, ny - 1 - k);
      } else {
        NEXT(w, x, -k) = NEXT(w, x, wrap(-k, ny));
        NEXT(w, x, ny - 1 + k) = NEXT(w, x, wrap(ny - 1 + k, ny));
      }
    }

  /* 4. P = p^i - p^w and L = lap n on rows -1 .. ny. */
#pragma omp parallel for num_threads(nt) if (nt > 1)
  for (int y = -1; y <= ny; y++)
    for (int x = 0; x < nx; x++) {
      double phi[9], dx, dy, lap;
      gather(w->n, nx, 2, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &dx, &dy, &lap);
      PEXT(w, x, y) = orc_pressure_diff(p->a, p->b, p->T, NEXT(w, x, y));
      LEXT(w, x, y) = lap;
    }

  /* 5. F = d(p^i - p^w) + kappa n d(lap n) + F_ext on rows 0 .. ny-1;
   * 6./7. wall rule; 8. n u* = sum f c + F/2.                               */
#pragma omp parallel for num_threads(nt) if (nt > 1)
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t s = (size_t)y * nx + x;
      double phi[9], dPx, dPy, dLx, dLy, tmp;
      gather(w->P, nx, 1, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &dPx, &dPy, &tmp);
      gather(w->L, nx, 1, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &dLx, &dLy, &tmp);
      double n = NEXT(w, x, y);
      double Fx = (dPx + kappa * n * dLx) + p->A0 * w->sinx[x];
      double Fy = dPy + kappa * n * dLy;
      w->Fx[s] = Fx;
      w->Fy[s] = Fy;

      double fl[9];
      for (int i = 0; i < 9; i++) fl[i] = w->fp[i * S + s];
      if (walls && (y == 0 || y == ny - 1)) {
        double g[9], nh;
        for (int i = 0; i < 9; i++) g[i] = f[i * S + s];
        int top = (y == ny - 1);
        orc_wall(top, top ? p->u_top : p->u_bot, Fx, Fy, fl, g, &nh);
        for (int i = 0; i < 9; i++) w->fp[i * S + s] = fl[i];
      }
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < 9; i++) {
        sx = sx + CX[i] * fl[i];
        sy = sy + CY[i] * fl[i];
      }
      JXE(w, x, y) = sx + 0.5 * Fx;
      JYE(w, x, y) = sy + 0.5 * Fy;
    }

  /* n u* on the ghost rows -1 and ny: mirror image about the wall (x part
   * even, y part odd), else periodic.                                       */
  for (int x = 0; x < nx; x++) {
    if (walls) {
      JXE(w, x, -1) = JXE(w, x, 1);
      JYE(w, x, -1) = -JYE(w, x, 1);
      JXE(w, x, ny) = JXE(w, x, ny - 2);
      JYE(w, x, ny) = -JYE(w, x, ny - 2);
    } else {
      JXE(w, x, -1) = JXE(w, x, ny - 1);
      JYE(w, x, -1) = JYE(w, x, ny - 1);
      JXE(w, x, ny) = JXE(w, x, 0);
      JYE(w, x, ny) = JYE(w, x, 0);
    }
  }
}

static void collide(const orc_params *p, const work_t *w, double *fout) {
  const int nx = p->nx, ny = p->ny;
  const size_t S = (size_t)nx * ny;
  const double omega = 1.0 / p->tau;
  int nt = p->nthreads;
#ifdef _OPENMP
  if (nt <= 0) nt = omp_get_max_threads();
#else
  (void)nt;
#endif
#pragma omp parallel for num_threads(nt) if (nt > 1)
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t s = (size_t)y * nx + x;
      double phi[9], dnx, dny, dJx, dJy, tmp, jx_dummy;
      /* 9. grad n and div(n u*) with the same first-derivative stencil. */
      gather(w->n, nx, 2, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &dnx, &dny, &tmp);
      gather(w->Jx, nx, 1, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &dJx, &jx_dummy, &tmp);
      gather(w->Jy, nx, 1, x, y, phi);
      orc_stencils(p->N, p->Q, phi, &tmp, &dJy, &jx_dummy);
      double divJ = dJx + dJy;
      double n = NEXT(w, x, y);
      double ux = JXE(w, x, y) / n;
      double uy = JYE(w, x, y) / n;
      /* 10. equilibrium, forcing term, BGK relaxation (Eq. evoleq). */
      double feq[9], Fi[9];
      orc_feq(n, ux, uy, p->T, feq);
      orc_forcing(p->tau, p->T, ux, uy, w->Fx[s], w->Fy[s], dnx, dny, divJ, Fi);
      for (int i = 0; i < 9; i++) {
        double fi = w->fp[i * S + s];
        fout[i * S + s] = (fi - omega * (fi - feq[i])) + Fi[i];
      }
    }
}

/* Advance the state f (post-collision populations [9][ny][nx]) by nsteps.
 * Returns 0, or -1 on allocation failure / bad arguments.                   */
int orc_step(const orc_params *p, double *f, int64_t nsteps) {
  if (p->nx < 1 || p->ny < 1 || (p->walls && p->ny < 3) || nsteps < 0)
    return -1;
  work_t w;
  if (!work_alloc(&w, p->nx, p->ny)) {
    work_free(&w);
    return -1;
  }
  for (int64_t t = 0; t < nsteps; t++) {
    prepare(p, f, &w);
    collide(p, &w, f); /* prepare() keeps everything collide() needs */
  }
  work_free(&w);
  return 0;
}

/* Density n (n-hat on wall rows) and physical velocity u* = (sum f c + F/2)/n
 * at the current time, i.e. steps 1-8 applied to the stored state.
 * Optional outputs Fx, Fy (total force) may be NULL.                       */
int orc_moments(const orc_params *p, const double *f, double *n, double *ux,
                double *uy, double *Fx, double *Fy) {
  if (p->nx < 1 || p->ny < 1 || (p->walls && p->ny < 3)) return -1;
  work_t w;
  if (!work_alloc(&w, p->nx, p->ny)) {
    work_free(&w);
    return -1;
  }
  prepare(p, f, &w);
  for (int y = 0; y < p->ny; y++)
    for (int x = 0; x < p->nx; x++) {
      size_t s = (size_t)y * p->nx + x;
      double nn = NEXT(&w, x, y);
      n[s] = nn;
      ux[s] = JXE(&w, x, y) / nn;
      uy[s] = JYE(&w, x, y) / nn;
      if (Fx) Fx[s] = w.Fx[s];
      if (Fy) Fy[s] = w.Fy[s];
    }
  work_free(&w);
  return 0;
}

/* ------------------------------------------------------------------------
 * 16-bit deviation storage (a storage format of this implementation; the
 * paper stores populations at full precision).
 *
 * For i = 1..8 the stored value is the deviation d_i = f_i - r_i from a
 * reference population r_i (r = rho_ref / 9 on the axis links, rho_ref / 36
 * on the diagonal links, each rounded to FP32: the reference is part of the
 * format), rounded to nearest, ties to even, with p significant bits and a
 * smallest exponent emin (bfloat16: p = 8, emin = -126; IEEE binary16:
 * p = 11, emin = -14).  The rest population is kept at full precision and
 * takes the remainder f_0 = n - sum_{i>=1} f_i with n = sum_i f_i of the
 * unrounded site, so every site keeps its density (Sec. II: mass
 * conservation of the collision and the wall rule).
 * ------------------------------------------------------------------------ */

/* x rounded to p significant bits (ties to even); spacing never below
 * 2^(emin - p + 1) (gradual underflow).  Overflow is not handled: the
 * deviations stay far below the formats' largest finite values.            */
double orc_round_sig(double x, int p, int emin) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  (void)frexp(x, &e); /* |x| in [2^(e-1), 2^e) */
  int lead = e - 1;
  if (lead < emin) lead = emin;
  double ulp = ldexp(1.0, lead - (p - 1));
  return nearbyint(x / ulp) * ulp; /* x / ulp is exact: ulp is a power of 2 */
}

/* Reference population of link i (0 for the rest link). */
static double ref_pop(int i, double rho_ref) {
  if (i == 0) return 0.0;
  return (double)(float)(i <= 4 ? rho_ref / 9.0 : rho_ref / 36.0);
}

/* Replace the state f[9][S] by the value it has after a store in the 16-bit
 * deviation format.  dev_unrounded (8*S doubles, may be NULL) receives the
 * deviations before rounding, plane i-1 for link i.                        */
void orc_quantize(int p, int emin, double rho_ref, size_t S, double *f,
                  double *dev_unrounded) {
  for (size_t s = 0; s < S; s++) {
    double n = 0.0;
    for (int i = 0; i < 9; i++) n += f[i * S + s];
    double rest = n;
    for (int i = 1; i < 9; i++) {
      double r = ref_pop(i, rho_ref);
      double d = f[i * S + s] - r;
      if (dev_unrounded) dev_unrounded[(size_t)(i - 1) * S + s] = d;
      f[i * S + s] = r + orc_round_sig(d, p, emin);
      rest -= f[i * S + s];
    }
    f[s] = rest;
  }
}
