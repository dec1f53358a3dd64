// lb_sweep.cu -- strip-sweep kernel: one fused time step of the vdW lattice
// Boltzmann scheme (arXiv:1307.6703, Sec. II) streamed through shared memory
// by TMA, for FP32 storage and for 16-bit deviation storage.
//
// Work decomposition.  The lattice is cut into column strips of W interior
// columns (W <= 116 for FP32 storage, <= 112 for 16-bit storage, strip
// origins on 16-byte TMA coordinates) and row segments of up to 64 rows.  One
// CTA of 124 threads, one per column of the 124-column window x0-4 ..
// x0+119 (strip plus 4-column halos), sweeps its segment upwards, two rows
// per iteration.  Every row of the previous state is read from HBM once by
// the TMA engine: tensor copies bring a pair of rows of all nine population
// planes into a 5-slot ring in shared memory (one mbarrier per slot, waits
// bounded): pair k+2 is requested as iteration k starts, into the slot that
// iteration k-1 freed, and first read in iteration k+1.
//
// Iteration k (a = ya - 3 + 2k) runs four stages, separated by CTA barriers
// (and preceded by one that frees the oldest ring slot), each on two rows:
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
// Storage formats.  FP32: the nine populations as floats.  16-bit deviation
// storage (bfloat16 or IEEE half): for i = 1..8 the deviation d_i = f_i - r_i
// from a reference population (r = rho_ref/9 on axis links, rho_ref/36 on
// diagonal links, rounded to FP32) is stored rounded to nearest even; the
// rest population stays a float and takes the remainder n - sum_{i>=1} f_i
// of the ROUNDED values, so each site keeps its density to FP32 round-off.
// Arithmetic is FP32 in both formats; with 16-bit storage it runs on the
// deviations themselves: the references cancel in the momentum, add one
// constant to the density, and enter the collision as one constant per link
// class, so decoding and encoding are a conversion each.
//
// On the last step of a call (or every step while a monitoring ring is set)
// every CTA also writes FP64 partial sums of mass and momentum of the state
// it stored, and a flag for non-finite or out-of-range sites; the CTA that
// finishes last adds them up, so the global sums of the new state need no
// further kernel.
//
// Consecutive steps are programmatic dependent launches: step k+1 may be
// scheduled once every CTA of step k has left its main loop, and waits
// (griddepcontrol.wait) for step k to complete before it touches global
// memory, which hides the launch gap between the two grids.
#include <cstddef>
#include <type_traits>
#include <vector>
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbk {

namespace {

constexpr int kPairs = 5;                   // population ring, in pairs of rows
constexpr int kSeg = 64;                    // rows per segment
constexpr uint32_t kWaitLimit = 1u << 22;

constexpr int round128(int b) { return ((b + 127) / 128) * 128; }

// FP32 storage: one 3D box {kCols, 2, 9} (columns, rows, planes) per pair.
// A CTA has one thread per window column (kCols threads): the window is
// the strip plus 4 halo columns on each side.  124 columns keep four CTAs'
// shared memory within an SM.
struct StoreF32 {
  static constexpr int kCols = 124;           // columns x0-4 .. x0+119
  static constexpr bool kDev = false;
  static constexpr int kQuantum = 4;          // 16-byte x coordinates of float boxes
  static constexpr int kMaxW = kCols - 8;     // 116
  static constexpr unsigned kTxBytes = 9 * 2 * kCols * sizeof(float);
  static constexpr int kSlotBytes = round128(kTxBytes);
  static constexpr int kMinBlocks = 4;
  using Row = const float *;  // row r of a slot; plane q starts q * 2 * kCols later
  __device__ static Row row(const unsigned char *slot, int r) {
    return reinterpret_cast<const float *>(slot) + r * kCols;
  }
  __device__ static float get(Row p, int q, int c, const SweepArgs &) { return p[q * 2 * kCols + c]; }
  __device__ static float getd(Row p, int q, int c, const SweepArgs &) { return p[q * 2 * kCols + c]; }
};

// 16-bit deviation storage: a float box {kCols, 2, 1} of the rest plane and a
// 16-bit box {128, 2, 8} of the deviation planes (256-byte rows) per pair.
// The window is 128 columns (four full warps): five CTAs per SM still fit.
template <class H>
struct StoreDev {
  static constexpr int kCols = 128;           // columns x0-4 .. x0+123
  static constexpr bool kDev = true;
  static constexpr int kQuantum = 8;          // 16-byte x coordinates of 16-bit boxes
  static constexpr int kMaxW = kCols - 8;     // 120
  static constexpr int kDevCols = 128;
  static constexpr int kRestBytes = 2 * kCols * sizeof(float);
  static constexpr int kDevOffset = round128(kRestBytes);
  static constexpr int kDevBytes = 8 * 2 * kDevCols * 2;
  static constexpr unsigned kTxBytes = kRestBytes + kDevBytes;
  static constexpr int kSlotBytes = round128(kDevOffset + kDevBytes);
  static constexpr int kMinBlocks = 5;
  struct Row {
    const float *f0;
    const H *d;
  };
  __device__ static Row row(const unsigned char *slot, int r) {
    return {reinterpret_cast<const float *>(slot) + r * kCols,
            reinterpret_cast<const H *>(slot + kDevOffset) + r * kDevCols};
  }
  __device__ static float dec(H v);
  __device__ static H enc(float v);
  __device__ static float get(const Row &p, int q, int c, const SweepArgs &A) {
    if (q == 0) return p.f0[c];
    return (q <= 4 ? A.ref_ax : A.ref_dg) + dec(p.d[(q - 1) * 2 * kDevCols + c]);
  }
  // Deviation d_q = f_q - r_q of a moving population (q >= 1); the rest
  // population (q = 0) is stored in full and returned as it is.
  __device__ static float getd(const Row &p, int q, int c, const SweepArgs &) {
    if (q == 0) return p.f0[c];
    return dec(p.d[(q - 1) * 2 * kDevCols + c]);
  }
};
template <>
__device__ __forceinline__ float StoreDev<__nv_bfloat16>::dec(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 StoreDev<__nv_bfloat16>::enc(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ float StoreDev<__half>::dec(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ __half StoreDev<__half>::enc(float v) { return __float2half_rn(v); }

using StoreBF16 = StoreDev<__nv_bfloat16>;
using StoreFP16 = StoreDev<__half>;

// Rings of row pairs.  A row y belongs to pair (y - y0) / 2 of a ring with
// origin y0: populations y0 = ya - 4, density ya - 3, P/L ya - 4, n u*
// ya - 5, chosen so that iteration k writes pair k of every ring.  Each
// ring is long enough that no stage overwrites a slot another thread may
// still read without a barrier in between.
template <int SlotBytes, int kCols>
struct __align__(128) SweepSmem {
  unsigned char pops[kPairs][SlotBytes];  // one row pair of every plane per slot
  // four pairs: stage A of iteration k+1 writes pair k+1 into a slot that
  // stage D of iteration k (pairs k-2 and k-1) does not read
  float n[4][2][kCols];
  float2 PL[2][2][kCols];  // (P, lap n): one 64-bit load per stencil tap
  float2 J[2][2][kCols];   // (n u*_x, n u*_y)
  unsigned long long full[kPairs];
  int abort;  // set by a thread whose copy wait gave up; read after a barrier
  static_assert(SlotBytes % 128 == 0, "TMA destinations must be 128-byte aligned");
  static_assert(kPairs * SlotBytes >= (int)(sizeof(double) * 4 * kCols + sizeof(unsigned)),
                "the end-of-kernel reduction reuses the population ring");
};
template <class St>
using SmemOf = SweepSmem<St::kSlotBytes, St::kCols>;
static_assert(offsetof(SmemOf<StoreF32>, pops) == 0 && offsetof(SmemOf<StoreBF16>, pops) == 0,
              "the ring starts the (128-byte aligned) block");
static_assert(StoreBF16::kDevOffset % 128 == 0, "16-bit boxes must land on 128-byte boundaries");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

// Wait for phase `parity` of an mbarrier; gives up after a bounded number
// of polls, reports it and returns false (the data are then meaningless but
// every address the kernel touches stays in bounds; the caller stops the
// CTA at its next barrier and drains the copies still in flight).
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
  if (mbar_try(bar, parity, kWaitLimit)) return true;
  atomicOr(err, 1);
  return false;
}

__device__ __forceinline__ void tma_box(const CUtensorMap *map, uint32_t dst, uint32_t bar, int xpad, int ypad,
                                        uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(xpad), "r"(ypad), "r"(0), "r"(bar), "l"(policy)
      : "memory");
}

// L2 policies for the population boxes.  A tile's first four pairs (its
// 4-row warm-up and first 4 rows) are the rows the segment below reads last,
// about one tile-duration later: they are kept (evict-last) so that read
// comes from L2; the tile's other rows get the normal policy.
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
  uint64_t p;
  if (keep)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
constexpr int kKeepPairs = 4;

// Two rows (all nine planes, the window's columns) of the padded state into
// a ring slot, completing on the slot's mbarrier.
template <class St>
__device__ __forceinline__ void tma_pair(const CUtensorMap *m0, const CUtensorMap *m1, uint32_t dst, uint32_t bar,
                                         int xpad, int ypad, uint64_t policy) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(St::kTxBytes)
               : "memory");
  tma_box(m0, dst, bar, xpad, ypad, policy);
  if constexpr (St::kDev) tma_box(m1, dst + St::kDevOffset, bar, xpad, ypad, policy);
}

__device__ __forceinline__ int dec(int s, int n) { return s == 0 ? n - 1 : s - 1; }

// 1/v by the PTX approximate reciprocal (v > 0 and finite here: densities
// and 1 - b n on the liquid-vapour branch).
__device__ __forceinline__ float rcp(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ int inc(int s, int n) { return s == n - 1 ? 0 : s + 1; }

// Arithmetic on one site (V = float) or on the two rows a thread computes
// in a stage at once (V = float2: row j = 0 in .x, j = 1 in .y, executed as
// the packed FP32 pair instructions of sm_100 and later).  Each operation is
// rounded once, as written, so both forms give the same bits for the same
// site and the result of a site does not depend on which form (and so which
// tiling) computed it -- with one rule for the callers: no product feeds an
// addition or subtraction.  The code generator fuses a pair multiply into
// the pair add that consumes it (one rounding instead of two; measured on
// GB300, and unlike the scalar forms, which stay as written), so every such
// combination is written as an explicit fma in both forms.
template <class V>
struct Op;
template <>
struct Op<float> {
  __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  __device__ static float neg(float a) { return -a; }
  __device__ static float k(float a) { return a; }
  __device__ static float inv(float v) { return rcp(v); }
};
template <>
struct Op<float2> {
  __device__ static float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  __device__ static float2 sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
    return *reinterpret_cast<float2 *>(&d);
  }
  __device__ static float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  __device__ static float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
  __device__ static float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
  __device__ static float2 k(float a) { return make_float2(a, a); }
  __device__ static float2 inv(float2 v) { return make_float2(rcp(v.x), rcp(v.y)); }
};

// Density and raw momentum sum_i f_i c_i of the pulled populations (16-bit
// storage: deviations, n gets the references' sum r_sum):
// E = f1 + f5 + f8 and W = f3 + f6 + f7 serve n and the x momentum.
template <class V>
__device__ __forceinline__ void site_sums(const V *f, float r_sum, bool dev, V &n, V &sx, V &sy) {
  using O = Op<V>;
  const V E = O::add(O::add(f[1], f[5]), f[8]), W = O::add(O::add(f[3], f[6]), f[7]);
  sx = O::sub(E, W);
  n = O::add(O::add(f[0], O::add(f[2], f[4])), O::add(E, W));
  if (dev) n = O::add(n, O::k(r_sum));
  sy = O::sub(O::add(O::add(f[2], f[5]), f[6]), O::add(O::add(f[4], f[7]), f[8]));
}

// P = p^i - p^w = nT - nT/(1 - bn) + a n^2 (Eq. eqstate).
template <class V>
__device__ __forceinline__ V pressure_diff(V c, float T, float a, float b) {
  using O = Op<V>;
  const V nT = O::mul(c, O::k(T));
  const V r = O::inv(O::fma(c, O::k(-b), O::k(1.0f)));
  return O::fma(O::mul(c, O::k(a)), c, O::fma(O::neg(nT), r, nT));  // nT - nT r in one rounding
}

// x-derivative, y-derivative and Laplacian stencils of Eqs. (xstencil,
// laplstencil) at column t of row r1, rows r0 = y-1 and r2 = y+1.  Every
// operation is rounded as written (explicit intrinsics, no contraction), so
// a site's value does not depend on the code path that computed it.
struct Sten {
  float N, M, Q, R, four_QR;
};
// N d1 + M (d2 + d0) for the differences d of the three rows
__device__ __forceinline__ float dstencil(const Sten &s, float d1, float d2, float d0) {
  return __fmaf_rn(s.N, d1, __fmul_rn(s.M, __fadd_rn(d2, d0)));
}
__device__ __forceinline__ float sdx(const Sten &s, const float *r0, const float *r1, const float *r2, int t) {
  return dstencil(s, __fsub_rn(r1[t + 1], r1[t - 1]), __fsub_rn(r2[t + 1], r2[t - 1]), __fsub_rn(r0[t + 1], r0[t - 1]));
}
__device__ __forceinline__ float sdy(const Sten &s, const float *r0, const float *r2, int t) {
  return dstencil(s, __fsub_rn(r2[t], r0[t]), __fsub_rn(r2[t + 1], r0[t + 1]), __fsub_rn(r2[t - 1], r0[t - 1]));
}
__device__ __forceinline__ float slap(const Sten &s, const float *r0, const float *r1, const float *r2, int t) {
  const float s1 = __fadd_rn(__fadd_rn(r1[t + 1], r1[t - 1]), __fadd_rn(r2[t], r0[t]));
  const float s2 = __fadd_rn(__fadd_rn(r2[t + 1], r2[t - 1]), __fadd_rn(r0[t + 1], r0[t - 1]));
  return __fmaf_rn(s.Q, s1, __fmaf_rn(s.R, s2, __fmul_rn(-s.four_QR, r1[t])));
}

// x- and y-derivative stencils applied to both components of float2 rows.
__device__ __forceinline__ float2 sdx2(const Sten &s, const float2 *r0, const float2 *r1, const float2 *r2, int t) {
  const float2 a = r1[t + 1], b = r1[t - 1], c = r2[t + 1], d = r2[t - 1], e = r0[t + 1], f = r0[t - 1];
  return make_float2(dstencil(s, __fsub_rn(a.x, b.x), __fsub_rn(c.x, d.x), __fsub_rn(e.x, f.x)),
                     dstencil(s, __fsub_rn(a.y, b.y), __fsub_rn(c.y, d.y), __fsub_rn(e.y, f.y)));
}
__device__ __forceinline__ float2 sdy2(const Sten &s, const float2 *r0, const float2 *r2, int t) {
  const float2 g = r2[t], h = r0[t], c = r2[t + 1], e = r0[t + 1], d = r2[t - 1], f = r0[t - 1];
  return make_float2(dstencil(s, __fsub_rn(g.x, h.x), __fsub_rn(c.x, e.x), __fsub_rn(d.x, f.x)),
                     dstencil(s, __fsub_rn(g.y, h.y), __fsub_rn(c.y, e.y), __fsub_rn(d.y, f.y)));
}

// Propagated populations of the site in column t of row r1 (pull).  With
// 16-bit storage f[1..8] are the deviations d_i = f_i - r_i and f[0] is the
// rest population; with FP32 storage they are the populations.
template <class St>
__device__ __forceinline__ void pull(const typename St::Row &r0, const typename St::Row &r1,
                                     const typename St::Row &r2, int t, float *f, const SweepArgs &A) {
  f[0] = St::getd(r1, 0, t, A); f[1] = St::getd(r1, 1, t - 1, A); f[3] = St::getd(r1, 3, t + 1, A);
  f[2] = St::getd(r0, 2, t, A); f[5] = St::getd(r0, 5, t - 1, A); f[6] = St::getd(r0, 6, t + 1, A);
  f[4] = St::getd(r2, 4, t, A); f[7] = St::getd(r2, 7, t + 1, A); f[8] = St::getd(r2, 8, t - 1, A);
}

// Deviations <-> populations of the moving links (16-bit storage only).
__device__ __forceinline__ void add_refs(float *f, float r_ax, float r_dg) {
#pragma unroll
  for (int q = 1; q < 9; ++q) f[q] += q <= 4 ? r_ax : r_dg;
}

// One collision (Eqs. evoleq, eqfunc, forceterm, coeff) in the moment form
//   f*_i = (1 - omega) f_i + w_i E_i,
//   E_i = omega n [A_i + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2] + 3 c.B + 9/2 C:cc - 3/2 tr C,
// for the eight moving populations (the rest population is the remainder,
// taken by the caller after any storage rounding).  With on = omega n,
// S_i = on (c.u)^2 + C:cc and T_i = on c.u + c.B, w_i E_i splits into a part
// even in c, h_i = e_i + 9/2 w_i S_i with e_i = w_i (on A_i - 3/2 (S_x + S_y))
// (S_x + S_y = on u^2 + tr C), and an odd part t_i = 3 w_i T_i.  On the
// axes (w = 1/9) h_x = e_a + S_x / 2, t_x = T_x / 3; on the diagonals
// (w = 1/36) S_(+-) = S_x + S_y +- 2 X with X = on u_x u_y + C_xy and
// T_(+-) = T_y +- T_x, so h_(+-) = e_d + (S_x + S_y) / 8 +- X / 4 and
// t_(+-) = T_(+-) / 12.  kDev: f holds the deviations d_i = f_i - r_i
// and fs receives d*_i = f*_i - r_i = (1 - omega) d_i + w_i E_i - omega r_i;
// wr_ax and wr_dg are omega r_i on the axes and diagonals and join e_a, e_d.
template <bool kDev, class V>
__device__ __forceinline__ void collide(const SweepArgs &A, const V *f, V n, V Jx, V Jy, V Fx, V Fy, V dnx, V dny,
                                        V divJ, V *fs, float wr_ax = 0.f, float wr_dg = 0.f) {
  using O = Op<V>;
  const V rn = O::inv(n);
  const V ux = O::mul(Jx, rn), uy = O::mul(Jy, rn);
  const V on = O::mul(O::k(A.omega), n);
  const V onux = O::mul(on, ux), onuy = O::mul(on, uy);
  const V ux2 = O::mul(O::k(2.f), ux), uy2 = O::mul(O::k(2.f), uy);
  // C / g (Eq. coeff)
  const V th = O::k(A.th), g = O::k(A.g);
  const V cxx = O::fma(th, O::fma(ux2, dnx, divJ), O::mul(ux2, Fx));
  const V cyy = O::fma(th, O::fma(uy2, dny, divJ), O::mul(uy2, Fy));
  const V cxy = O::fma(th, O::fma(ux, dny, O::mul(uy, dnx)), O::fma(ux, Fy, O::mul(Fx, uy)));
  const V Sx = O::fma(onux, ux, O::mul(g, cxx)), Sy = O::fma(onuy, uy, O::mul(g, cyy));
  const V X = O::fma(onux, uy, O::mul(g, cxy));
  const V Sxy = O::add(Sx, Sy);  // on u^2 + tr C
  V ea, ed;
  if constexpr (kDev) {
    ea = O::fma(on, O::k(A.A_ax * (1.f / 9.f)), O::fma(O::k(-1.f / 6.f), Sxy, O::k(-wr_ax)));
    ed = O::fma(on, O::k(A.A_diag * (1.f / 36.f)), O::fma(O::k(-1.f / 24.f), Sxy, O::k(-wr_dg)));
  } else {
    ea = O::fma(on, O::k(A.A_ax * (1.f / 9.f)), O::mul(Sxy, O::k(-1.f / 6.f)));
    ed = O::fma(on, O::k(A.A_diag * (1.f / 36.f)), O::mul(Sxy, O::k(-1.f / 24.f)));
  }
  const V hx = O::fma(O::k(0.5f), Sx, ea), hy = O::fma(O::k(0.5f), Sy, ea);
  const V h5 = O::fma(O::k(0.125f), Sxy, O::fma(O::k(0.25f), X, ed));
  const V h6 = O::fma(O::k(0.125f), Sxy, O::fma(O::k(-0.25f), X, ed));
  // odd parts: t_x = T_x / 3, t_(+-) = (T_y +- T_x) / 12
  const V Tx = O::fma(g, Fx, onux), Ty = O::fma(g, Fy, onuy);
  const V Tp = O::add(Ty, Tx), Tm = O::sub(Ty, Tx);
  const V third = O::k(1.f / 3.f), mthird = O::k(-1.f / 3.f), twelfth = O::k(1.f / 12.f), mtwelfth = O::k(-1.f / 12.f);
  const V om1 = O::k(A.one_minus_omega);
  fs[1] = O::fma(om1, f[1], O::fma(Tx, third, hx));
  fs[3] = O::fma(om1, f[3], O::fma(Tx, mthird, hx));
  fs[2] = O::fma(om1, f[2], O::fma(Ty, third, hy));
  fs[4] = O::fma(om1, f[4], O::fma(Ty, mthird, hy));
  fs[5] = O::fma(om1, f[5], O::fma(Tp, twelfth, h5));
  fs[7] = O::fma(om1, f[7], O::fma(Tp, mtwelfth, h5));
  fs[6] = O::fma(om1, f[6], O::fma(Tm, twelfth, h6));
  fs[8] = O::fma(om1, f[8], O::fma(Tm, mtwelfth, h6));
}

// The rest population as the remainder: n - sum_{i>=1} f*_i (16-bit
// storage: (n - sum r_i) - sum d*_i), which keeps the site's mass exact.
template <class V>
__device__ __forceinline__ V rest_remainder(V n, const V *fs) {
  using O = Op<V>;
  return O::sub(n, O::add(O::add(O::add(fs[1], fs[3]), O::add(fs[2], fs[4])),
                          O::add(O::add(fs[5], fs[7]), O::add(fs[6], fs[8]))));
}

}  // namespace

// Where one step's results go: the new state (fout; the deviation planes of
// 16-bit storage at fdev) and, when arrivals is set, the fused global sums:
// the CTA that finishes last adds the nrec records at recs into total (if
// set) and monitor (if set, with mon_step) and resets *arrivals.
struct StepIO {
  float *fout;
  void *fdev;
  const double *recs;
  unsigned nrec;
  unsigned *arrivals;
  double *total;
  double *monitor;
  double mon_step;
};

// One CTA's work: strip `strip`, segment `seg` of the lattice described by
// A, whose input state the tensor maps tin (and tdev, the deviation planes
// of 16-bit storage) describe; results as O says; the CTA's mass/momentum
// record goes to rec.  Returns false when a copy wait gave up (the CTA then
// stopped at its next barrier and drained the copies still in flight).
// kPersist: called once per tile by the multi-step kernel, which does not
// hand its SM slots to a dependent grid early.
struct NoDone {
  __device__ void operator()() const {}
};

template <class St, bool kPersist = false, class Done = NoDone>
__device__ __forceinline__ bool sweep_body(const CUtensorMap *tin, const CUtensorMap *tdev, const SweepArgs &A,
                                           const StepIO &O, const int strip, const int seg, double *rec,
                                           const bool records, const Done &done = Done{}) {
  using Row = typename St::Row;
  using Smem = SmemOf<St>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(smem_raw);

  const int t = threadIdx.x;
  const int x0 = strip * A.base_w + St::kQuantum * min(strip, A.extra);
  const int W = A.base_w + (strip < A.extra ? St::kQuantum : 0);
  const int ya = seg * A.seg_h;
  const int yb = min(A.ny, ya + A.seg_h);
  const int nx = A.nx, ny = A.ny;
  const bool walls = A.walls != 0;
  const int x = x0 - 4 + t;  // interior column of this thread (may be a halo column)
  const bool actA = t >= 1 && t <= W + 6;
  const bool actB = t >= 2 && t <= W + 5;
  const bool actC = t >= 3 && t <= W + 4;
  const bool actD = t >= 4 && t <= W + 3;
  // Steady iterations run every stage on every thread, at column tcl (the
  // thread's own column for every active thread; clamped so that the
  // neighbours stay inside the window) and store ring values at column t:
  // the columns an inactive thread writes are never read by the next
  // stage's active threads, so only the global stores need a guard.
  constexpr int kCols = St::kCols, kThreads = St::kCols;
  const int tcl = min(max(t, 1), kCols - 2);
  const int kmax = (yb - ya + 5) >> 1;  // last iteration
  const int npairs = kmax + 2;          // rows ya-4 .. ya+2*kmax+3
  const Sten st{A.N, A.M, A.Q, A.R, A.four_QR};
  float sinx = 0.f;
  float *col = O.fout + A.off + x;  // f* (rest plane for 16-bit storage) of this column at interior row 0
  const int pitch = A.pitch, plane = (int)A.plane;
  const int gx = (x < 4) ? nx : ((x >= nx - 4) ? -nx : 0);  // periodic image column
  // 16-bit storage: sum of the moving links' reference populations, and the
  // collision's offsets omega r_ax, omega r_dg.
  const float r_sum = St::kDev ? 4.f * (A.ref_ax + A.ref_dg) : 0.f;
  const float wr_ax = St::kDev ? A.omega * A.ref_ax : 0.f;
  const float wr_dg = St::kDev ? A.omega * A.ref_dg : 0.f;

  if (actC) sinx = A.sinx[x < 0 ? x + nx : (x >= nx ? x - nx : x)];  // a constant table
  if (t == 0) {
    for (int s = 0; s < kPairs; ++s) mbar_init(smem_u32(&S.full[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.abort = 0;
  }
  // Launched as a programmatic dependent of the previous step: wait until
  // that grid has finished and its writes are visible before any other
  // global access (its output is this step's input, and this step's output
  // buffer was its input).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // TMA writes need 128-byte aligned destinations: refuse to run otherwise.
  if (smem_u32(&S.pops[0][0]) & 127u) {
    if (t == 0) atomicOr(A.err, 2);
    return false;
  }
  int issued = min(kPairs, npairs);  // pairs requested so far (thread 0's count)
  if (t == 0) {
    for (int P = 0; P < issued; ++P)
      tma_pair<St>(tin, tdev, smem_u32(S.pops[P]), smem_u32(&S.full[P]), x0, ya + 2 * P,
                   l2_policy(P < kKeepPairs));
  }
  __syncthreads();
  if (!mbar_wait(smem_u32(&S.full[0]), 0, A.err)) S.abort = 1;

  float sxa[2] = {0.f, 0.f}, sya[2] = {0.f, 0.f};  // raw momentum of rows a-2, a-1 (from last A)
  float Fx_prev = 0.f, Fy_prev = 0.f;              // force of row a-3 (from last C)
  float acc_m = 0.f, acc_x = 0.f, acc_y = 0.f;
  int bad = 0;
  int s5 = 0, s3 = 0;
  uint32_t par = 0;  // phase parity of pair k+1

  // One iteration; kSteady instantiates it for iterations whose rows are all
  // interior rows of the segment (no wall rows or their mirrors, no warm-up
  // rows, no periodic ghost images in y), where every per-row condition
  // below is known to hold and the two rows of a stage are independent.
  auto iteration = [&](const int k, auto steady_tag) -> bool {
    constexpr bool kSteady = decltype(steady_tag)::value;
    const int s5m1 = dec(s5, kPairs), s5m2 = dec(s5m1, kPairs), s5p1 = inc(s5, kPairs);
    const int s3m1 = (s3 + 3) & 3, s3m2 = (s3 + 2) & 3;  // density ring: 4 pairs
    const int s2 = k & 1, s2m1 = s2 ^ 1;
    // Every thread is past iteration k-1 (whose stage D last read pair
    // k-3): refill that slot with pair k-3+kPairs now, one stage earlier.
    if (k >= 3) {
      __syncthreads();
      if (t == 0 && k - 3 + kPairs < npairs) {
        const int slot = dec(s5m2, kPairs);
        tma_pair<St>(tin, tdev, smem_u32(S.pops[slot]), smem_u32(&S.full[slot]), x0, ya + 2 * (k - 3 + kPairs),
                     l2_policy(k - 3 + kPairs < kKeepPairs));
        ++issued;
      }
    }
    if (!mbar_wait(smem_u32(&S.full[s5p1]), par, A.err)) S.abort = 1;  // newest pair needed: k+1
    if (s5p1 == kPairs - 1) par ^= 1u;
    const int a = ya - 3 + 2 * k;

    // ---------------------------------------- A: rows a, a+1 -- n, raw momentum
    // (Steady iterations compute both rows of each stage at once wherever
    // the arithmetic needs no neighbour data: row j in lane j of a float2.)
    {
      const Row q0 = St::row(S.pops[s5], 0), q1 = St::row(S.pops[s5], 1);      // rows a-1, a
      const Row q2 = St::row(S.pops[s5p1], 0), q3 = St::row(S.pops[s5p1], 1);  // rows a+1, a+2
      float sx_new[2] = {0.f, 0.f}, sy_new[2] = {0.f, 0.f};
      const int tc = kSteady ? tcl : t;
      // Each stage computes both rows before it stores either, so that the
      // two rows' independent arithmetic can interleave.
      float nv[2] = {0.f, 0.f};
      bool nw[2] = {false, false};
      if constexpr (kSteady) {
        float fa[9], fb[9];
        pull<St>(q0, q1, q2, tc, fa, A);
        pull<St>(q1, q2, q3, tc, fb, A);
        float2 f2[9], n2, sx2, sy2;
#pragma unroll
        for (int q = 0; q < 9; ++q) f2[q] = make_float2(fa[q], fb[q]);
        site_sums<float2>(f2, r_sum, St::kDev, n2, sx2, sy2);
        nv[0] = n2.x; nv[1] = n2.y;
        sx_new[0] = sx2.x; sx_new[1] = sx2.y;  // the reference populations cancel in the momentum
        sy_new[0] = sy2.x; sy_new[1] = sy2.y;
        nw[0] = nw[1] = true;
      } else {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int y = a + j;
          const Row r0 = j ? q1 : q0, r1 = j ? q2 : q1, r2 = j ? q3 : q2;
          if (actA && (!walls || (y >= 0 && y <= ny - 1))) {
            float f[9];
            pull<St>(r0, r1, r2, tc, f, A);
            float n;
            if constexpr (St::kDev) {
              if (walls && (y == 0 || y == ny - 1)) add_refs(f, A.ref_ax, A.ref_dg);
            }
            if (walls && y == 0) {
              n = St::get(r1, 0, t, A) + St::get(r1, 4, t, A) + St::get(r1, 7, t, A) + St::get(r1, 8, t, A) +
                  f[1] + f[3] + f[4] + f[7] + f[8];
            } else if (walls && y == ny - 1) {
              n = St::get(r1, 0, t, A) + St::get(r1, 2, t, A) + St::get(r1, 6, t, A) + St::get(r1, 5, t, A) +
                  f[1] + f[3] + f[2] + f[6] + f[5];
            } else {
              site_sums<float>(f, r_sum, St::kDev, n, sx_new[j], sy_new[j]);
            }
            nv[j] = n;
            nw[j] = true;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (nw[j]) S.n[s3][j][t] = nv[j];
      __syncthreads();
      // A copy wait that gave up (this iteration's or an earlier one's) was
      // recorded before the barrier: every thread leaves here together.
      if (S.abort) return false;

      // -------------------------------------- B: rows a-1, a -- P, lap n
      {
        const float *n0 = S.n[s3m1][0], *n1 = S.n[s3m1][1];  // rows a-2, a-1
        const float *n2 = S.n[s3][0], *n3 = S.n[s3][1];      // rows a, a+1
        float2 plv[2];
        bool plw[2] = {false, false};
        if constexpr (kSteady) {
          const float2 P2 = pressure_diff<float2>(make_float2(n1[tc], n2[tc]), A.T, A.a, A.b);
          plv[0] = make_float2(P2.x, slap(st, n0, n1, n2, tc));
          plv[1] = make_float2(P2.y, slap(st, n1, n2, n3, tc));
          plw[0] = plw[1] = true;
        } else {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int y = a - 1 + j;
            const float *r0 = j ? n1 : n0, *r1 = j ? n2 : n1, *r2 = j ? n3 : n2;
            if (actB && y >= ya - 2 && (!walls || (y >= 0 && y <= ny - 1))) {
              if (walls && y == 0) r0 = r2;
              if (walls && y == ny - 1) r2 = r0;
              plv[j] = make_float2(pressure_diff<float>(r1[tc], A.T, A.a, A.b), slap(st, r0, r1, r2, tc));
              plw[j] = true;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (plw[j]) S.PL[s2][j][t] = plv[j];
      }
      __syncthreads();

      // -------------------------------------- C: rows a-2, a-1 -- F, n u*
      float Fx_cur[2] = {0.f, 0.f}, Fy_cur[2] = {0.f, 0.f};
      {
        const float2 *P0 = S.PL[s2m1][0], *P1 = S.PL[s2m1][1], *P2 = S.PL[s2][0], *P3 = S.PL[s2][1];
        float2 jv[2];
        bool jw[2] = {false, false};
        float sxv[2] = {sxa[0], sxa[1]}, syv[2] = {sya[0], sya[1]};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int y = a - 2 + j;
          if (!(kSteady || (actC && y >= ya - 1 && (!walls || (y >= 0 && y <= ny - 1))))) continue;
          const float2 *p0 = j ? P1 : P0, *p1 = j ? P2 : P1, *p2 = j ? P3 : P2;
          if (!kSteady && walls && y == 0) p0 = p2;
          if (!kSteady && walls && y == ny - 1) p2 = p0;
          const float n = S.n[s3m1][j][tc];
          const float kn = __fmul_rn(A.kappa, n);
          // D P + kappa n D L = D G with G = P + kappa n L at the neighbours
          // (n is the site's own density, a constant of the stencil)
          auto G = [kn](const float2 v) { return __fmaf_rn(kn, v.y, v.x); };
          const float g0m = G(p0[tc - 1]), g0c = G(p0[tc]), g0p = G(p0[tc + 1]);
          const float g1m = G(p1[tc - 1]), g1p = G(p1[tc + 1]);
          const float g2m = G(p2[tc - 1]), g2c = G(p2[tc]), g2p = G(p2[tc + 1]);
          const float Fx = __fmaf_rn(A.A0, sinx, dstencil(st, __fsub_rn(g1p, g1m), __fsub_rn(g2p, g2m),
                                                          __fsub_rn(g0p, g0m)));
          const float Fy = dstencil(st, __fsub_rn(g2c, g0c), __fsub_rn(g2p, g0p), __fsub_rn(g2m, g0m));
          if (!kSteady && walls && (y == 0 || y == ny - 1)) {
            // populations of rows y-1 .. y+1: pairs k-1 and k of the ring
            const Row w0 = St::row(S.pops[s5m1], 0), w1 = St::row(S.pops[s5m1], 1);
            const Row w2 = St::row(S.pops[s5], 0), w3 = St::row(S.pops[s5], 1);
            float f[9];
            pull<St>(j ? w1 : w0, j ? w2 : w1, j ? w3 : w2, t, f, A);
            if constexpr (St::kDev) add_refs(f, A.ref_ax, A.ref_dg);
            const bool top = y != 0;
            wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx, Fy, n, f);
            sxv[j] = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
            syv[j] = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
          }
          jw[j] = true;
          Fx_cur[j] = Fx;
          Fy_cur[j] = Fy;
        }
        // n u* = sum f c + F / 2 (Eq. newvel)
        if constexpr (kSteady) {
          using O2 = Op<float2>;
          const float2 h = O2::k(0.5f);
          const float2 jx = O2::fma(h, make_float2(Fx_cur[0], Fx_cur[1]), make_float2(sxv[0], sxv[1]));
          const float2 jy = O2::fma(h, make_float2(Fy_cur[0], Fy_cur[1]), make_float2(syv[0], syv[1]));
          jv[0] = make_float2(jx.x, jy.x);
          jv[1] = make_float2(jx.y, jy.y);
        } else {
#pragma unroll
          for (int j = 0; j < 2; ++j)
            jv[j] = make_float2(Op<float>::fma(0.5f, Fx_cur[j], sxv[j]), Op<float>::fma(0.5f, Fy_cur[j], syv[j]));
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (jw[j]) S.J[s2][j][t] = jv[j];
      }
      sxa[0] = sx_new[0]; sxa[1] = sx_new[1];
      sya[0] = sy_new[0]; sya[1] = sy_new[1];
      __syncthreads();

      // -------------------------------------- D: rows a-3, a-2 -- collide, store
      {
        const float *n0 = S.n[s3m2][0], *n1 = S.n[s3m2][1], *n2 = S.n[s3m1][0], *n3 = S.n[s3m1][1];
        const float2 *J0 = S.J[s2m1][0], *J1 = S.J[s2m1][1], *J2 = S.J[s2][0], *J3 = S.J[s2][1];
        // population rows a-4 .. a-1: pair k-2 row 1, pair k-1 rows 0, 1, pair k row 0
        const Row q0p = St::row(S.pops[s5m2], 1), q1p = St::row(S.pops[s5m1], 0);
        const Row q2p = St::row(S.pops[s5m1], 1), q3p = St::row(S.pops[s5], 0);
        // inputs of the collision of row a-3+j: gradients from the rings,
        // n, n u*, F; pulled populations in f
        struct In {
          float n, Jx, Jy, Fx, Fy, dnx, dny, divJ;
        };
        auto inputs = [&](const int j, const int y, float *f) -> In {
          const float *m0 = j ? n1 : n0, *m1 = j ? n2 : n1, *m2 = j ? n3 : n2;
          const float2 *j0p = j ? J1 : J0, *j1p = j ? J2 : J1, *j2p = j ? J3 : J2;
          const float Fx = j ? Fx_cur[0] : Fx_prev, Fy = j ? Fy_cur[0] : Fy_prev;
          const bool bot = !kSteady && walls && y == 0, top = !kSteady && walls && y == ny - 1;
          float dJy, dJx;
          if (bot || top) {
            // mirror rows across the wall: n and J_x even, J_y odd
            float sgm = 1.f, sgp = 1.f;
            if (bot) { m0 = m2; j0p = j2p; sgm = -1.f; }
            if (top) { m2 = m0; j2p = j0p; sgp = -1.f; }
            const float2 g = j2p[t], h = j0p[t], c = j2p[t + 1], e = j0p[t + 1], d = j2p[t - 1], ff = j0p[t - 1];
            dJy = st.N * (sgp * g.y - sgm * h.y) + st.M * ((sgp * c.y - sgm * e.y) + (sgp * d.y - sgm * ff.y));
            dJx = sdx2(st, j0p, j1p, j2p, t).x;
          } else {
            dJx = sdx2(st, j0p, j1p, j2p, tc).x;
            dJy = sdy2(st, j0p, j2p, tc).y;
          }
          In in;
          in.n = m1[tc];
          in.dnx = sdx(st, m0, m1, m2, tc);
          in.dny = sdy(st, m0, m2, tc);
          in.divJ = __fadd_rn(dJx, dJy);
          const float2 Jc = j1p[tc];
          in.Jx = Jc.x;
          in.Jy = Jc.y;
          in.Fx = Fx;
          in.Fy = Fy;
          pull<St>(j ? q1p : q0p, j ? q2p : q1p, j ? q3p : q2p, tc, f, A);
          if (bot || top) {
            if constexpr (St::kDev) add_refs(f, A.ref_ax, A.ref_dg);
            wall_fill<float>(top, top ? A.u_top : A.u_bot, Fx, Fy, in.n, f);
            if constexpr (St::kDev) add_refs(f, -A.ref_ax, -A.ref_dg);
          }
          return in;
        };
        // store row y and add it to the CTA's records; fs[0] is the rest
        // population's remainder for FP32 storage, computed after the
        // rounding for 16-bit storage
        auto emit = [&](const int y, float *fs, const In &in) {
          const float n = in.n, Jx = in.Jx, Jy = in.Jy, Fx = in.Fx, Fy = in.Fy;
          const int gy = (kSteady || walls) ? 0 : ((y < 4) ? ny : ((y >= ny - 4) ? -ny : 0));
          float *o = col + (long long)y * pitch;
          if constexpr (!St::kDev) {
            // The new state is streamed out (evict-first stores): it is
            // read again only by the next step.
#pragma unroll
            for (int q = 0; q < 9; ++q) __stcs(o + q * plane, fs[q]);
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
          } else {
            // Round the deviations (fs[1..8] hold d*_i), then let the rest
            // population carry the remainder of the rounded values (site
            // density kept): f*_0 = (n - sum r_i) - sum rounded d*_i.
            using H = decltype(St::enc(0.f));
            H code[8];
#pragma unroll
            for (int q = 1; q < 9; ++q) {
              code[q - 1] = St::enc(fs[q]);
              fs[q] = St::dec(code[q - 1]);
            }
            fs[0] = rest_remainder<float>(Op<float>::sub(n, r_sum), fs);
            H *od = reinterpret_cast<H *>(O.fdev) + (A.off + x + (long long)y * pitch);
            o[0] = fs[0];
#pragma unroll
            for (int q = 0; q < 8; ++q) od[q * plane] = code[q];
            if (gx != 0) {
              o[gx] = fs[0];
#pragma unroll
              for (int q = 0; q < 8; ++q) od[q * plane + gx] = code[q];
            }
            if (gy != 0) {
              float *oy = o + (long long)gy * pitch;
              H *ody = od + (long long)gy * pitch;
              oy[0] = fs[0];
#pragma unroll
              for (int q = 0; q < 8; ++q) ody[q * plane] = code[q];
              if (gx != 0) {
                oy[gx] = fs[0];
#pragma unroll
                for (int q = 0; q < 8; ++q) ody[q * plane + gx] = code[q];
              }
            }
          }
          // Mass and momentum of the stored site: sum f* = n (by
          // construction), sum f* c = n u* + F/2 (identity of the collision).
          if (records) {
            if (!(n > 0.f && n < A.nmax && fabsf(Jx) + fabsf(Jy) < 3.0e38f)) bad = 1;
            acc_m += n;
            if constexpr (!St::kDev) {
              acc_x += Jx + 0.5f * Fx;
              acc_y += Jy + 0.5f * Fy;
            } else {  // momentum of the stored (rounded) populations; refs cancel
              acc_x += ((fs[1] - fs[3]) + (fs[5] - fs[6])) + (fs[8] - fs[7]);
              acc_y += ((fs[2] - fs[4]) + (fs[5] + fs[6])) - (fs[7] + fs[8]);
            }
          }
        };
        if constexpr (kSteady) {
          // both rows at once (the collision in float2 lanes), then their
          // stores (inactive columns store nothing)
          float fa[9], fb[9];
          const In ia = inputs(0, a - 3, fa), ib = inputs(1, a - 2, fb);
          float2 f2[9], fs2[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) f2[q] = make_float2(fa[q], fb[q]);
          const float2 n2 = make_float2(ia.n, ib.n);
          collide<St::kDev, float2>(A, f2, n2, make_float2(ia.Jx, ib.Jx), make_float2(ia.Jy, ib.Jy),
                                    make_float2(ia.Fx, ib.Fx), make_float2(ia.Fy, ib.Fy),
                                    make_float2(ia.dnx, ib.dnx), make_float2(ia.dny, ib.dny),
                                    make_float2(ia.divJ, ib.divJ), fs2, wr_ax, wr_dg);
          if constexpr (!St::kDev) fs2[0] = rest_remainder<float2>(n2, fs2);
          if (actD) {
            float fsa[9], fsb[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
              fsa[q] = fs2[q].x;
              fsb[q] = fs2[q].y;
            }
            emit(a - 3, fsa, ia);
            emit(a - 2, fsb, ib);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int y = a - 3 + j;
            if (!(actD && y >= ya && y < yb)) continue;
            float f[9], fs[9];
            const In in = inputs(j, y, f);
            collide<St::kDev, float>(A, f, in.n, in.Jx, in.Jy, in.Fx, in.Fy, in.dnx, in.dny, in.divJ, fs, wr_ax,
                                     wr_dg);
            if constexpr (!St::kDev) fs[0] = rest_remainder<float>(in.n, fs);
            emit(y, fs, in);
          }
        }
      }
      Fx_prev = Fx_cur[1];
      Fy_prev = Fy_cur[1];
    }
    s5 = s5p1;
    s3 = (s3 + 1) & 3;
    return true;
  };
  // Iteration k (a = ya - 3 + 2k) is steady -- every row of its four stages
  // interior, see the lambda's note -- when k >= 3, a - 2 < yb and, with
  // walls, 1 <= a - 3 and a + 1 <= ny - 2 (periodic: 4 <= a - 3 and
  // a + 1 < ny - 4).  These are lower and upper bounds on k, so the steady
  // iterations are the range [klo, khi).
  auto ceil2 = [](int v) { return (v + 1) >> 1; };  // ceil(v / 2), any sign
  const int klo = max(3, ceil2((walls ? 7 : 10) - ya));
  const int khi = min(min(kmax + 1, ceil2(yb - ya + 5)), walls ? ((ny - ya) >> 1) + 1 : ceil2(ny - ya - 2));
  int k = 0;
  bool ok = true;
  for (; ok && k < min(klo, kmax + 1); ++k) ok = iteration(k, std::false_type{});
  for (; ok && k < khi; ++k) ok = iteration(k, std::true_type{});
  for (; ok && k <= kmax; ++k) ok = iteration(k, std::false_type{});
  if (!ok) {
    // A copy wait gave up: wait (again bounded) for every copy this CTA may
    // still have in flight -- the last kPairs requested -- so that none
    // lands in shared memory after the CTA has moved on, then stop.
    if (t == 0) {
      for (int P = max(0, issued - kPairs); P < issued; ++P)
        (void)mbar_try(smem_u32(&S.full[P % kPairs]), (uint32_t)((P / kPairs) & 1), kWaitLimit);
    }
    __syncthreads();
    return false;
  }
  // The next step may be scheduled now (it waits for this grid to finish).
  if constexpr (!kPersist) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // Every thread is here: the tile's stores are done.  A persistent caller
  // publishes its completion now -- the records below touch only this CTA's
  // shared memory and the record slots, so dependent tiles need not wait.
  done();

  // CTA partial sums of the stored state (FP64, fixed order), when asked
  // for.  Every TMA copy has been waited for, so the population ring is
  // free for them.
  if (!records) return true;
  double *red = reinterpret_cast<double *>(&S.pops[0][0]);
  __syncthreads();
  red[0 * kThreads + t] = (double)acc_m;
  red[1 * kThreads + t] = (double)acc_x;
  red[2 * kThreads + t] = (double)acc_y;
  red[3 * kThreads + t] = (double)bad;
  __syncthreads();
  // Warp 0 (a full warp) sums them in a fixed order: lane l takes columns
  // l, l+32, l+64, l+96, then a shuffle tree.  FP64 throughput is low on
  // this part, so the tree keeps the FP64 work off the critical path.
  if (t < 32) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double sum = 0.0;
      for (int i = t; i < kThreads; i += 32) sum += red[q * kThreads + i];
      v[q] = sum;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if (t == 0) {
#pragma unroll
      for (int q = 0; q < 4; ++q) rec[q] = v[q];
    }
  }
  if (O.arrivals == nullptr) return true;

  // The last CTA to finish sums every CTA's record (FP64, fixed order:
  // thread t takes records t, t + 124, ..., then warp 0's tree), so the
  // global sums of the new state need no further kernel.
  const unsigned nrec = O.nrec;
  unsigned *last = reinterpret_cast<unsigned *>(red + 4 * kThreads);
  if (t == 0) {
    __threadfence();  // this CTA's record before its arrival
    *last = (atomicAdd(O.arrivals, 1u) == nrec - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (*last == 0u) return true;
  __threadfence();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned b = t; b < nrec; b += kThreads) {
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += __ldcg(O.recs + 4 * (size_t)b + q);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q * kThreads + t] = acc[q];
  __syncthreads();
  if (t < 32) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double sum = 0.0;
      for (int i = t; i < kThreads; i += 32) sum += red[q * kThreads + i];
      v[q] = sum;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    }
    if (t == 0) {
      const double r[5] = {v[0], v[1], v[2], v[3] != 0.0 ? 1.0 : 0.0, __ldcg(A.err) != 0 ? 1.0 : 0.0};
      if (O.total) {
#pragma unroll
        for (int q = 0; q < 5; ++q) O.total[q] = r[q];
      }
      if (O.monitor) {
#pragma unroll
        for (int q = 0; q < 5; ++q) O.monitor[q] = r[q];
        O.monitor[5] = O.mon_step;
      }
      *O.arrivals = 0u;
    }
  }
  return true;
}

template <class St>
__global__ void __launch_bounds__(St::kCols, St::kMinBlocks)
sweep_step_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tdev,
                  const SweepArgs A) {
  const StepIO O{A.fout, A.fdev, A.partials, gridDim.x * gridDim.y, A.total ? A.arrivals : nullptr,
                 A.total, A.monitor, A.mon_step};
  (void)sweep_body<St>(&tin, &tdev, A, O, blockIdx.x, blockIdx.y,
                       A.partials + 4 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x), A.records != 0);
}

// Batched step: CTA b works on items[b] (instance, strip, segment) of a
// work list over many independent lattices.  Arguments and tensor maps of
// each instance sit in device memory for both buffer parities; an instance
// reads buffer (item.par0 ^ kpar).
template <class St>
__global__ void __launch_bounds__(St::kCols, St::kMinBlocks)
sweep_batch_kernel(const BatchItem *__restrict__ items, const SweepArgs *__restrict__ args,
                   const CUtensorMap *__restrict__ maps, int kpar, int records) {
  __shared__ SweepArgs A;
  const BatchItem it = items[blockIdx.x];
  const int par = it.par0 ^ kpar;
  const CUtensorMap *m = maps + 4 * it.inst + 2 * par;  // [instance][input buffer][map]
  if (threadIdx.x == 0) {
    A = args[2 * it.inst + par];
    // the maps were written through the generic proxy (a host copy)
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m + 1) : "memory");
  }
  __syncthreads();
  const StepIO O{A.fout, A.fdev, A.partials, 0u, nullptr, nullptr, nullptr, 0.0};
  (void)sweep_body<St>(m, m + 1, A, O, it.strip, it.seg, A.partials + 4 * (size_t)it.rec, records != 0);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Multi-step sweeps.  One launch runs P.nsteps steps.  CTAs take
// (step, item) tickets from a counter in step-major order, items in
// work-list order.  Instead of a grid-wide barrier between steps, every
// item (one tile of one lattice) carries a completion counter done[item]
// (the steps it has finished, offset by P.epoch): before step k of an item,
// its threads wait until every item it depends on -- the tiles of the same
// lattice whose stored sites (ghost images included) its TMA boxes read,
// and the tiles whose boxes read its own sites (they must have read the
// buffer it is about to overwrite) -- has reached epoch + k.  A tile starts
// as soon as its neighbourhood has finished the previous step and a CTA
// that is done takes the next ticket, so SMs do not idle at step
// boundaries; lattices of a batch never wait for one another.  All CTAs are
// co-resident (cooperative launch) and no step-(k+1) ticket is handed out
// before every step-k ticket, so the smallest unfinished ticket always has
// its dependencies done and can proceed.  Every wait is bounded: on give-up
// the CTA sets the lattice's error flag (bit 4 for a dependency wait) and
// stops, and the items that depend on it give up in turn.

// The next ticket (thread 0 draws, the barrier publishes).
__device__ __forceinline__ unsigned next_ticket(const PersistArgs &P, unsigned *slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(P.next, 1u);
  __syncthreads();
  return *slot;
}

// Bounded wait of the CTA's threads (one per dependency) until every item
// item i depends on has finished `target` steps; false on give-up.  The
// caller's next barrier publishes *ok.
__device__ __forceinline__ void wait_deps(const PersistArgs &P, int i, unsigned target, int *err, int *ok) {
  for (int d = P.dep_ofs[i] + (int)threadIdx.x; d < P.dep_ofs[i + 1]; d += (int)blockDim.x) {
    const unsigned *f = P.done + P.dep_idx[d];
    uint32_t n = 0;
    while ((int)(ld_acquire_gpu(f) - target) < 0) {
      if (++n > kWaitLimit) {
        *ok = 0;
        atomicOr(err, 4);
        break;
      }
      __nanosleep(64);
    }
  }
}

// Release item i's step: its stores (generic proxy) before the counter,
// ordered for the neighbours' TMA (async proxy) reads.
__device__ __forceinline__ void release_item(const PersistArgs &P, int i, unsigned value) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release_gpu(P.done + i, value);
  }
}

// Before a CTA's second and later items: the ring's mbarriers are
// initialised again by the sweep body.
template <class St>
__device__ __forceinline__ void inval_ring() {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  auto &S = *reinterpret_cast<SmemOf<St> *>(smem_raw);
  for (int q = 0; q < kPairs; ++q)
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&S.full[q])) : "memory");
}

// Batched form: items[i] names the lattice, tile and record; arguments and
// tensor maps of every lattice (both buffer parities) in device memory.
template <class St>
__global__ void __launch_bounds__(St::kCols, St::kMinBlocks)
sweep_batch_persist_kernel(const BatchItem *__restrict__ items, const SweepArgs *__restrict__ args,
                           const CUtensorMap *__restrict__ maps, const PersistArgs P) {
  __shared__ SweepArgs A;
  __shared__ int dep_ok;
  __shared__ unsigned ticket;
  const int t = threadIdx.x;
  bool first = true;
  const unsigned total = (unsigned)P.nsteps * (unsigned)P.nitems;
  for (;;) {
    const unsigned tk = next_ticket(P, &ticket);
    if (tk >= total) break;
    const int k = (int)(tk / (unsigned)P.nitems), i = (int)(tk % (unsigned)P.nitems);
    const unsigned target = P.epoch + (unsigned)k;
    const BatchItem it = items[i];
    const int par = it.par0 ^ ((P.kpar0 + k) & 1);
    const CUtensorMap *m = maps + 4 * it.inst + 2 * par;  // [instance][input buffer][map]
    if (t == 0) dep_ok = 1;
    __syncthreads();  // also ends the previous item
    wait_deps(P, i, target, args[2 * it.inst].err, &dep_ok);
    if (t == 0) {
      A = args[2 * it.inst + par];
      // the maps were written through the generic proxy (a host copy)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m + 1) : "memory");
      // the neighbours' stores, made visible by the acquires, for this
      // CTA's TMA (async proxy) reads
      asm volatile("fence.proxy.async.global;" ::: "memory");
      if (!first) inval_ring<St>();
    }
    __syncthreads();
    if (!dep_ok) return;
    first = false;
    const StepIO O{A.fout, A.fdev, A.partials, 0u, nullptr, nullptr, nullptr, 0.0};
    if (!sweep_body<St, true>(m, m + 1, A, O, it.strip, it.seg, A.partials + 4 * (size_t)it.rec,
                              k == P.nsteps - 1, [&] { release_item(P, i, target + 1u); }))
      return;
  }
}

// Single-lattice form: item i is tile i (strip i % nstrips, segment
// i / nstrips); arguments and maps are kernel parameters.  The last step
// writes the per-tile records and the CTA that finishes last adds them into
// `total` (mass, momentum, flags); while monitoring, every step does so into
// its own record slot and writes its record into the host ring.
template <class St>
__global__ void __launch_bounds__(St::kCols, St::kMinBlocks)
sweep_multi_kernel(const __grid_constant__ CUtensorMap tin0, const __grid_constant__ CUtensorMap tdev0,
                   const __grid_constant__ CUtensorMap tin1, const __grid_constant__ CUtensorMap tdev1,
                   const SweepArgs A, const PersistArgs P, const MultiOut Q) {
  __shared__ int dep_ok;
  __shared__ unsigned ticket;
  const int t = threadIdx.x;
  bool first = true;
  const unsigned total = (unsigned)P.nsteps * (unsigned)P.nitems;
  for (;;) {
    const unsigned tk = next_ticket(P, &ticket);
    if (tk >= total) break;
    const int k = (int)(tk / (unsigned)P.nitems), i = (int)(tk % (unsigned)P.nitems);
    const unsigned target = P.epoch + (unsigned)k;
    const int par = (P.kpar0 + k) & 1;  // input buffer of step k
    const bool last = k == P.nsteps - 1;
    if (t == 0) dep_ok = 1;
    __syncthreads();  // also ends the previous item
    wait_deps(P, i, target, A.err, &dep_ok);
    if (t == 0) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      if (!first) inval_ring<St>();
    }
    __syncthreads();
    if (!dep_ok) {
      if (t == 0) Q.total[4] = 1.0;  // the sums of this launch will not be written
      return;
    }
    first = false;
    const bool mon = Q.mon_ring != nullptr;
    StepIO O;
    O.fout = par ? Q.fout[1] : Q.fout[0];  // (no dynamic indexing of the parameter space)
    O.fdev = par ? Q.fdev[1] : Q.fdev[0];
    O.recs = mon ? Q.mon_recs + 4 * (size_t)P.nitems * k : A.partials;
    O.nrec = (unsigned)P.nitems;
    O.arrivals = mon ? Q.mon_arr + k : (last ? Q.arrivals : nullptr);
    O.total = last ? Q.total : nullptr;
    O.monitor = mon ? Q.mon_ring + 6 * ((Q.mon_step0 + k) % Q.mon_cap) : nullptr;
    O.mon_step = (double)(Q.mon_step0 + k);
    if (!sweep_body<St, true>(par ? &tin1 : &tin0, par ? &tdev1 : &tdev0, A, O, i % A.nstrips, i / A.nstrips,
                              const_cast<double *>(O.recs) + 4 * (size_t)i, last || mon,
                              [&] { release_item(P, i, target + 1u); })) {
      if (t == 0) Q.total[4] = 1.0;
      return;
    }
  }
}

// 16-bit storage -> nine float planes: f_0 as stored, f_i = r_i + d_i.
template <class St, typename H>
__global__ void widen_kernel(const float *__restrict__ f0, const H *__restrict__ d, float *__restrict__ out,
                             long long plane, float ref_ax, float ref_dg) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane;
       e += (long long)gridDim.x * blockDim.x) {
    out[e] = f0[e];
#pragma unroll
    for (int q = 1; q < 9; ++q) out[q * plane + e] = (q <= 4 ? ref_ax : ref_dg) + St::dec(d[(q - 1) * plane + e]);
  }
}

// Nine float planes -> 16-bit storage (the rounding of the step kernel's
// store, with n the float sum of the nine values).
template <class St, typename H>
__global__ void narrow_kernel(const float *__restrict__ in, float *__restrict__ f0, H *__restrict__ d,
                              long long plane, float ref_ax, float ref_dg) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < plane;
       e += (long long)gridDim.x * blockDim.x) {
    float f[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = in[q * plane + e];
    const float n = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
      const float r = q <= 4 ? ref_ax : ref_dg;
      const H c = St::enc(f[q] - r);
      d[(q - 1) * plane + e] = c;
      f[q] = r + St::dec(c);
    }
    f0[e] = n - (((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8])));
  }
}

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point.
typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_map(CUtensorMapDataType type, int esize, void *base, int pitch, int ny, long long plane,
                       int nplanes, int box_cols, CUtensorMap *map) {
  static encode_tiled_fn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (encode_tiled_fn)fn;
  }
  // 3D view (column, padded row, plane); one box = box_cols columns x 2
  // rows x nplanes planes.
  const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)(ny + 8), (cuuint64_t)nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)plane * esize};
  const cuuint32_t box[3] = {(cuuint32_t)box_cols, 2, (cuuint32_t)nplanes};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int quantum_of(int store) {
  return store == kStoreF32 ? StoreF32::kQuantum : (store == kStoreBF16 ? StoreBF16::kQuantum : StoreFP16::kQuantum);
}
int maxw_of(int store) {
  return store == kStoreF32 ? StoreF32::kMaxW : (store == kStoreBF16 ? StoreBF16::kMaxW : StoreFP16::kMaxW);
}

template <class St>
cudaError_t prepare_one(size_t *smem_bytes) {
  *smem_bytes = sizeof(SmemOf<St>);
  cudaError_t e = cudaFuncSetAttribute(sweep_step_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)*smem_bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_batch_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem_bytes);
  return e;
}

template <class St>
cudaError_t launch_batch_one(const BatchItem *items, int nitems, const SweepArgs *args, const CUtensorMap *maps,
                             int kpar, int records, size_t smem, cudaStream_t st) {
  sweep_batch_kernel<St><<<nitems, St::kCols, smem, st>>>(items, args, maps, kpar, records);
  return cudaGetLastError();
}

template <class St>
cudaError_t launch_one(const CUtensorMap &m0, const CUtensorMap &m1, const SweepArgs &A, size_t smem,
                       cudaStream_t st) {
  // Programmatic dependent launch: the kernel may start while the previous
  // step finishes; it waits for that grid (griddepcontrol.wait) before
  // touching global memory.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)A.nstrips, (unsigned)A.nseg);
  cfg.blockDim = dim3(St::kCols);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_step_kernel<St>, m0, m1, A);
}

template <class St>
cudaError_t launch_batch_persist_one(const BatchItem *items, const SweepArgs *args, const CUtensorMap *maps,
                                     const PersistArgs &P, int grid, size_t smem, cudaStream_t st) {
  // Cooperative launch: the runtime refuses a grid that cannot be resident
  // all at once, which the dependency waits rely on.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(St::kCols);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_batch_persist_kernel<St>, items, args, maps, P);
}

template <class St>
cudaError_t launch_multi_one(const CUtensorMap (&m)[2][2], const SweepArgs &A, const PersistArgs &P,
                             const MultiOut &Q, int grid, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sweep_multi_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(St::kCols);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_multi_kernel<St>, m[0][0], m[0][1], m[1][0], m[1][1], A, P, Q);
}

template <class St>
cudaError_t persist_capacity_one(size_t smem, int *blocks) {
  // the smaller residency of the two multi-step kernels
  cudaError_t e = cudaFuncSetAttribute(sweep_batch_persist_kernel<St>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sweep_multi_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, per_sm2 = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_batch_persist_kernel<St>, St::kCols, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, sweep_multi_kernel<St>, St::kCols, smem);
  per_sm = std::min(per_sm, per_sm2);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *blocks = per_sm * sms;
  return e;
}

unsigned elementwise_blocks(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

bool sweep_supported(int store, int nx, int ny) {
  if (store != kStoreF32 && store != kStoreBF16 && store != kStoreFP16) return false;
  const double pitch = (double)(((nx + 8 + 31) / 32) * 32);
  return nx % quantum_of(store) == 0 && nx >= 8 && ny >= 8 && 9.0 * pitch * (double)(ny + 8) < 2147483647.0;
}

size_t sweep_buffer_bytes(int store, long long plane) {
  return store == kStoreF32 ? 9 * (size_t)plane * sizeof(float) : (size_t)plane * (sizeof(float) + 8 * 2);
}

cudaError_t sweep_make_maps(int store, void *base, int pitch, int ny, long long plane, CUtensorMap *m0,
                            CUtensorMap *m1) {
  if (store == kStoreF32) {
    static_assert(StoreF32::kTxBytes == 9 * 2 * StoreF32::kCols * sizeof(float), "TMA box must match the slot");
    cudaError_t e = encode_map(CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, pitch, ny, plane, 9, StoreF32::kCols, m0);
    *m1 = *m0;
    return e;
  }
  static_assert(StoreBF16::kRestBytes == 2 * StoreBF16::kCols * sizeof(float) &&
                    StoreBF16::kDevBytes == 2 * StoreBF16::kDevCols * 8 * 2 && StoreBF16::kCols == StoreFP16::kCols,
                "TMA boxes must match the slot");
  cudaError_t e = encode_map(CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, pitch, ny, plane, 1, StoreBF16::kCols, m0);
  if (e != cudaSuccess) return e;
  void *dev = static_cast<char *>(base) + (size_t)plane * sizeof(float);
  return encode_map(store == kStoreBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, dev,
                    pitch, ny, plane, 8, StoreBF16::kDevCols, m1);
}

void sweep_strips(int store, int nx, int nstrips, int *base_w, int *extra) {
  const int qn = quantum_of(store);
  *base_w = qn * (nx / (qn * nstrips));
  *extra = (nx - *base_w * nstrips) / qn;
}

int sweep_min_strips(int store, int nx) { return (nx + maxw_of(store) - 1) / maxw_of(store); }

void sweep_plan(int store, int nx, int ny, int *nstrips, int *base_w, int *extra, int *seg_h, int *nseg) {
  const int qn = quantum_of(store), maxw = maxw_of(store);
  *nstrips = (nx + maxw - 1) / maxw;
  *base_w = qn * (nx / (qn * *nstrips));
  *extra = (nx - *base_w * *nstrips) / qn;
  *seg_h = ny < kSeg ? ny : kSeg;
  *nseg = (ny + *seg_h - 1) / *seg_h;
}

cudaError_t sweep_prepare(int store, size_t *smem_bytes) {
  switch (store) {
    case kStoreF32: return prepare_one<StoreF32>(smem_bytes);
    case kStoreBF16: return prepare_one<StoreBF16>(smem_bytes);
    case kStoreFP16: return prepare_one<StoreFP16>(smem_bytes);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep(int store, const CUtensorMap &m0, const CUtensorMap &m1, const SweepArgs &A,
                         size_t smem, cudaStream_t st) {
  switch (store) {
    case kStoreF32: return launch_one<StoreF32>(m0, m1, A, smem, st);
    case kStoreBF16: return launch_one<StoreBF16>(m0, m1, A, smem, st);
    case kStoreFP16: return launch_one<StoreFP16>(m0, m1, A, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_batch(int store, const BatchItem *items, int nitems, const SweepArgs *args,
                               const CUtensorMap *maps, int kpar, int records, size_t smem, cudaStream_t st) {
  if (nitems < 1) return cudaSuccess;
  switch (store) {
    case kStoreF32: return launch_batch_one<StoreF32>(items, nitems, args, maps, kpar, records, smem, st);
    case kStoreBF16: return launch_batch_one<StoreBF16>(items, nitems, args, maps, kpar, records, smem, st);
    case kStoreFP16: return launch_batch_one<StoreFP16>(items, nitems, args, maps, kpar, records, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t persist_capacity(int store, size_t smem, int *blocks) {
  switch (store) {
    case kStoreF32: return persist_capacity_one<StoreF32>(smem, blocks);
    case kStoreBF16: return persist_capacity_one<StoreBF16>(smem, blocks);
    case kStoreFP16: return persist_capacity_one<StoreFP16>(smem, blocks);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_multi(int store, const CUtensorMap (&maps)[2][2], const SweepArgs &A, const PersistArgs &P,
                               const MultiOut &Q, int grid, size_t smem, cudaStream_t st) {
  switch (store) {
    case kStoreF32: return launch_multi_one<StoreF32>(maps, A, P, Q, grid, smem, st);
    case kStoreBF16: return launch_multi_one<StoreBF16>(maps, A, P, Q, grid, smem, st);
    case kStoreFP16: return launch_multi_one<StoreFP16>(maps, A, P, Q, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sweep_batch_persist(int store, const BatchItem *items, const SweepArgs *args,
                                       const CUtensorMap *maps, const PersistArgs &P, int grid, size_t smem,
                                       cudaStream_t st) {
  switch (store) {
    case kStoreF32: return launch_batch_persist_one<StoreF32>(items, args, maps, P, grid, smem, st);
    case kStoreBF16: return launch_batch_persist_one<StoreBF16>(items, args, maps, P, grid, smem, st);
    case kStoreFP16: return launch_batch_persist_one<StoreFP16>(items, args, maps, P, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

// Tiles each tile of the sweep depends on (see sweep_batch_persist_kernel): the
// owners of every site its TMA boxes read -- columns x0-4 .. x0+123 and
// rows ya-4 .. yb+4, periodic images mapped back to the site they copy
// (rows outside the lattice with walls are never written) -- and,
// symmetrically, every tile whose window reads its sites.
void sweep_deps(int store, int nx, int ny, int walls, int nstrips, int base_w, int extra, int seg_h,
                std::vector<int> &ofs, std::vector<int> &idx) {
  const int qn = quantum_of(store);
  const int nseg = (ny + seg_h - 1) / seg_h;
  const int ntiles = nstrips * nseg;
  std::vector<int> strip_of(nx);
  for (int s = 0; s < nstrips; ++s) {
    const int x0 = s * base_w + qn * std::min(s, extra);
    const int W = base_w + (s < extra ? qn : 0);
    for (int x = x0; x < x0 + W; ++x) strip_of[x] = s;
  }
  std::vector<std::vector<int>> deps(ntiles);
  std::vector<int> cs, gs;
  for (int s = 0; s < nstrips; ++s) {
    const int x0 = s * base_w + qn * std::min(s, extra);
    cs.clear();
    // the widest box: 128 columns of the 16-bit deviation planes
    for (int x = x0 - 4; x < x0 - 4 + StoreBF16::kDevCols; ++x) cs.push_back(strip_of[((x % nx) + nx) % nx]);
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    for (int g = 0; g < nseg; ++g) {
      const int ya = g * seg_h, yb = std::min(ny, ya + seg_h);
      gs.clear();
      for (int y = ya - 4; y <= yb + 4; ++y) {
        if (walls && (y < 0 || y >= ny)) continue;
        gs.push_back((((y % ny) + ny) % ny) / seg_h);
      }
      std::sort(gs.begin(), gs.end());
      gs.erase(std::unique(gs.begin(), gs.end()), gs.end());
      const int a = s + nstrips * g;
      for (int s2 : cs)
        for (int g2 : gs) {
          const int b = s2 + nstrips * g2;
          deps[a].push_back(b);  // a reads b's sites
          deps[b].push_back(a);  // so b must not overwrite them before a has read them
        }
    }
  }
  ofs.assign(ntiles + 1, 0);
  idx.clear();
  for (int a = 0; a < ntiles; ++a) {
    std::sort(deps[a].begin(), deps[a].end());
    deps[a].erase(std::unique(deps[a].begin(), deps[a].end()), deps[a].end());
    idx.insert(idx.end(), deps[a].begin(), deps[a].end());
    ofs[a + 1] = (int)idx.size();
  }
}

cudaError_t launch_widen(int store, const void *buf, float *wide, long long plane, float ref_ax, float ref_dg,
                         cudaStream_t st) {
  const float *f0 = static_cast<const float *>(buf);
  const void *d = static_cast<const char *>(buf) + (size_t)plane * sizeof(float);
  const unsigned blocks = elementwise_blocks(plane);
  if (store == kStoreBF16)
    widen_kernel<StoreBF16><<<blocks, 256, 0, st>>>(f0, (const __nv_bfloat16 *)d, wide, plane, ref_ax, ref_dg);
  else if (store == kStoreFP16)
    widen_kernel<StoreFP16><<<blocks, 256, 0, st>>>(f0, (const __half *)d, wide, plane, ref_ax, ref_dg);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_narrow(int store, const float *wide, void *buf, long long plane, float ref_ax, float ref_dg,
                          cudaStream_t st) {
  float *f0 = static_cast<float *>(buf);
  void *d = static_cast<char *>(buf) + (size_t)plane * sizeof(float);
  const unsigned blocks = elementwise_blocks(plane);
  if (store == kStoreBF16)
    narrow_kernel<StoreBF16><<<blocks, 256, 0, st>>>(wide, f0, (__nv_bfloat16 *)d, plane, ref_ax, ref_dg);
  else if (store == kStoreFP16)
    narrow_kernel<StoreFP16><<<blocks, 256, 0, st>>>(wide, f0, (__half *)d, plane, ref_ax, ref_dg);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace lbk
