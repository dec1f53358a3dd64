// lb_internal.h -- launchers shared between the translation units of the
// library (FP64 parity build, FP32 build, host API).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

namespace lbk {

// Arguments of the strip-sweep kernel (lb_sweep.cu).  The state buffers use
// the padded layout: plane q, interior site (x, y) at element
// q * plane + off + y * pitch + x, with 4 ghost columns and 4 ghost rows on
// each side.  FP32 storage: nine float planes at fout.  16-bit deviation
// storage: the rest population as one float plane at fout, the deviations
// d_i = f_i - r_i (i = 1..8) as eight 16-bit planes at fdev (same pitch,
// plane and offset, counted in 16-bit elements).
struct SweepArgs {
  int nx, ny, walls;
  int pitch;
  long long plane, off;
  int seg_h, nseg, nstrips, base_w, extra;
  float T, a, b, kappa, omega, one_minus_omega, g, th, A0, u_bot, u_top;
  float N, M, Q, R, four_QR;
  float A_rest, A_ax, A_diag;  // rest factors 1 + (T - T0)(c.c - 2 T0) / (2 T0^2)
  float nmax;                  // 1/b (upper bound of a valid density)
  float ref_ax, ref_dg;        // reference populations r_i of the 16-bit format
  const float *sinx;
  float *fout;
  void *fdev;
  double *partials;            // 4 doubles per CTA: mass, J_x, J_y, bad-site flag
  int records;                 // write the per-CTA records (0: skip them)
  int *err;                    // set when a bounded wait gave up
  // Non-null (single-lattice launches with records only): the last CTA to
  // finish sums every CTA's record in a fixed order into total[0..4] --
  // mass, J_x, J_y, 1.0 if any record flags a bad site, 1.0 if *err is set
  // -- and resets *arrivals (a counter that is zero between launches).
  double *total;
  unsigned *arrivals;
  // Non-null: the same last CTA also writes {total[0..4], mon_step} here
  // (device address of a record in a mapped host ring).
  double *monitor;
  double mon_step;
};

// Storage formats of the sweep kernel (values of lb_precision).
constexpr int kStoreF32 = 1, kStoreBF16 = 2, kStoreFP16 = 3;

// Whether the sweep kernel of storage `store` can run an nx x ny lattice
// (column quantum of its TMA boxes, ghost bands, 32-bit plane offsets).
bool sweep_supported(int store, int nx, int ny);
cudaError_t sweep_prepare(int store, size_t *smem_bytes);
// Strips (widths base_w or base_w + quantum, the first `extra` wider; the
// quantum is 4 columns for FP32 storage and 8 for 16-bit storage) and row
// segments of the sweep kernel for an nx x ny lattice.
void sweep_plan(int store, int nx, int ny, int *nstrips, int *base_w, int *extra, int *seg_h, int *nseg);
// Widths of nstrips strips (>= sweep_min_strips) over nx columns: base_w or
// base_w + quantum, the first `extra` wider.
void sweep_strips(int store, int nx, int nstrips, int *base_w, int *extra);
int sweep_min_strips(int store, int nx);
// TMA descriptors of one padded state buffer with the boxes the kernel's
// ring expects (built next to the kernel so the two cannot differ).  FP32:
// one map of the nine planes (m1 is a copy).  16-bit storage: m0 maps the
// float rest plane at base, m1 the eight deviation planes that follow it.
cudaError_t sweep_make_maps(int store, void *base, int pitch, int ny, long long plane, CUtensorMap *m0,
                            CUtensorMap *m1);
// Bytes of one padded state buffer of the given storage.
size_t sweep_buffer_bytes(int store, long long plane);
cudaError_t launch_sweep(int store, const CUtensorMap &m0, const CUtensorMap &m1, const SweepArgs &A,
                         size_t smem, cudaStream_t st);

// Dependency lists of the tiles (CSR): tile a waits for the tiles
// idx[ofs[a] .. ofs[a+1]) before each step.
void sweep_deps(int store, int nx, int ny, int walls, int nstrips, int base_w, int extra, int seg_h,
                std::vector<int> &ofs, std::vector<int> &idx);

// One CTA of the batched sweep: instance `inst`, its strip and segment, the
// index of its mass/momentum record in the instance's record array, and the
// parity of the instance's input buffer at kpar = 0.
struct BatchItem {
  int inst, strip, seg, rec, par0;
};
// Batched step over a work list.  args: 2 per instance (input buffer 0, 1);
// maps: 4 per instance ([input buffer][map], map 1 = deviation planes of
// 16-bit storage or a copy of map 0), 64-byte aligned device memory.
cudaError_t launch_sweep_batch(int store, const BatchItem *items, int nitems, const SweepArgs *args,
                               const CUtensorMap *maps, int kpar, int records, size_t smem, cudaStream_t st);
// Multi-step batched sweep (one cooperative launch, many steps, per-item
// completion counters instead of a grid-wide barrier between steps).
// Item i of a step whose batch parity is kpar reads the input buffer
// items[i].par0 ^ kpar of its lattice; kpar = (kpar0 + k) & 1 at step k.
struct PersistArgs {
  int nitems;
  int nsteps;
  int kpar0;
  unsigned epoch;       // value of every done[] counter at launch
  unsigned *done;       // one per item
  const int *dep_ofs;   // item i depends on dep_idx[dep_ofs[i] .. dep_ofs[i+1])
  const int *dep_idx;
  unsigned *next;       // ticket counter, zero at launch
};
// Outputs of the single-lattice multi-step kernel: the step that reads
// buffer b writes fout[b] (and fdev[b], the deviation planes of 16-bit
// storage); the last step's CTA records are summed into total[0..4] by the
// CTA that finishes last (arrival counter *arrivals, zero between
// launches).
struct MultiOut {
  float *fout[2];
  void *fdev[2];
  double *total;
  unsigned *arrivals;
  // Monitoring (mon_ring non-null): every step k writes its records into
  // slot k of mon_recs (4 doubles per tile) and counts on mon_arr[k]; the
  // CTA that finishes step k last adds them and writes the step's record
  // {mass, J_x, J_y, unstable, wait error, step number} at
  // mon_ring + 6 * ((mon_step0 + k) % mon_cap).
  double *mon_recs;
  unsigned *mon_arr;
  double *mon_ring;
  int mon_cap;
  long long mon_step0;
};
// One lattice, P.nsteps steps in one cooperative launch (P.kpar0 = the
// input buffer of the first step; items are the tiles in index order).
cudaError_t launch_sweep_multi(int store, const CUtensorMap (&maps)[2][2], const SweepArgs &A, const PersistArgs &P,
                               const MultiOut &Q, int grid, size_t smem, cudaStream_t st);
// Resident CTAs of the multi-step batched kernel on this device (its grid
// may not exceed this: the dependency waits need every CTA resident).
cudaError_t persist_capacity(int store, size_t smem, int *blocks);
// P.nsteps batch steps in one cooperative launch of `grid` CTAs; the mass /
// momentum records of the last step go to each instance's record array.
cudaError_t launch_sweep_batch_persist(int store, const BatchItem *items, const SweepArgs *args,
                                       const CUtensorMap *maps, const PersistArgs &P, int grid, size_t smem,
                                       cudaStream_t st);
// Copy the periodic images into the ghost band of `nplanes` planes of
// `elem_bytes`-byte elements (4 or 2).
cudaError_t launch_ghost_fill(void *f, int elem_bytes, int nplanes, int nx, int ny, int pitch, long long plane,
                              long long off, int walls, cudaStream_t st);
// 16-bit storage <-> nine float planes (same padded layout, every element
// of the planes, ghost bands included).  narrow: d_i = f_i - r_i rounded to
// nearest even, rest plane = n - sum_{i>=1} (r_i + d_i).
cudaError_t launch_widen(int store, const void *buf, float *wide, long long plane, float ref_ax, float ref_dg,
                         cudaStream_t st);
cudaError_t launch_narrow(int store, const float *wide, void *buf, long long plane, float ref_ax, float ref_dg,
                          cudaStream_t st);

template <typename real_t>
struct StepArgs;

// One fused time step fin -> fout.
cudaError_t launch_step(const double *fin, double *fout, const StepArgs<double> &A, cudaStream_t st);
cudaError_t launch_step(const float *fin, float *fout, const StepArgs<float> &A, cudaStream_t st);

// Moments (n, u*) of the stored state; dtype 0 = double, 1 = float outputs.
cudaError_t launch_moments(const double *fin, const StepArgs<double> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);
cudaError_t launch_moments(const float *fin, const StepArgs<float> &A, void *n, void *ux,
                           void *uy, int dtype, cudaStream_t st);

// Equilibrium initial state from noise (mode 0) or device fields (mode 1).
cudaError_t launch_init(double *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);
cudaError_t launch_init(float *f, int nx, int ny, int pitch, long long plane, long long off, int mode, uint64_t seed, double rho_mean,
                        double amp, const double *rho0, const double *ux0, const double *uy0,
                        double T, cudaStream_t st);

}  // namespace lbk
