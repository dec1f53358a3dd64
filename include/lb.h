/*
 * lb.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for an
 * isothermal two-dimensional van der Waals liquid-vapour fluid under a
 * periodic external force and moving walls (Coclite, Gonnella & Lamura,
 * arXiv:1307.6703, Sec. II).
 *
 * Conventions shared by every entry point
 *  - Units are lattice units: dx = dt = 1, D2Q9 velocities c_i in {0,+-1}^2,
 *    reference temperature T0 = 1/3.  The paper's units (dt = sqrt(3)/3,
 *    |e| = sqrt(3), T0 = 1) map onto these by T -> T/3, a -> a/3,
 *    kappa -> kappa/3; densities, b, tau (in steps), lengths, the force
 *    amplitude A0, shear rates and velocities (in dx/dt) are unchanged.
 *  - Fields are row-major [ny][nx], x fastest.  x is the periodic flow
 *    direction; rows 0 and ny-1 are the walls when walls are on.
 *  - Populations are structure-of-arrays planes [9][ny][nx] in link order
 *    0 rest, 1 E, 2 N, 3 W, 4 S, 5 NE, 6 NW, 7 SW, 8 SE.
 *  - The stored state at time t is the post-collision, not yet propagated
 *    populations f*(r, t-1); one step propagates (pull), rebuilds the wall
 *    links, collides and stores f*(r, t).
 *  - Every call returns LB_OK (0) or a negative LB_ERR_* code; nothing is
 *    thrown across the ABI.  lb_last_error() gives a message for the last
 *    failure on a handle.
 *  - The caller owns every buffer it passes; the library owns the device
 *    memory of a handle (allocated by lb_create, freed by lb_destroy) and
 *    never keeps a caller pointer after a call returns.
 *  - Work is enqueued on the stream given in lb_params; calls that return
 *    host data synchronise that stream.  One handle must not be used from
 *    two host threads at once.
 *  - There is no CPU fallback: every computation runs in this library's
 *    CUDA kernels, and a call without a usable CUDA device fails with
 *    LB_ERR_CUDA.
 */
#ifndef LB_H_
#define LB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LB_OK = 0,
  LB_ERR_ARG = -1,      /* invalid argument or parameter set             */
  LB_ERR_CUDA = -2,     /* CUDA runtime error (no device, launch failure) */
  LB_ERR_OOM = -3,      /* device allocation failed                       */
  LB_ERR_UNSTABLE = -4, /* non-finite or unphysical density detected      */
  LB_ERR_TIMEOUT = -5,  /* a bounded device wait gave up                  */
  LB_ERR_STATE = -6     /* call out of order (e.g. step before init)      */
};

/* Storage / arithmetic precision of a handle. */
enum {
  LB_FP64 = 0,    /* FP64 storage and arithmetic, no fused multiply-add:
                     the evaluation order of the FP64 oracle (parity mode) */
  LB_FP32 = 1,    /* FP32 storage and arithmetic (performance path)        */
  LB_BF16DEV = 2, /* 16-bit deviation storage, bfloat16 (see below)        */
  LB_FP16DEV = 3  /* 16-bit deviation storage, IEEE binary16 (see below)   */
};
/* 16-bit deviation storage (a storage format of this library; the paper
 * keeps full-precision populations).  For i = 1..8 the stored value is the
 * deviation d_i = f*_i - r_i from the reference population r_i = rho_ref/9
 * (axis links) or rho_ref/36 (diagonal links), each rounded to FP32, itself
 * rounded to nearest even in the 16-bit format; the rest population f*_0
 * is stored as FP32 and takes the remainder n - sum_{i>=1} (r_i + d_i), so
 * every site keeps its density and the total mass is conserved to FP32
 * round-off (Sec. II: collision and wall rule conserve mass).  Arithmetic
 * is FP32.  20 bytes per site instead of 36 (FP32).  Needs nx a multiple of
 * 8, nx >= 8 and ny >= 8.                                                  */

/* Element type selector for lb_moments. */
enum { LB_DTYPE_F64 = 0, LB_DTYPE_F32 = 1 };

/* Problem statement (Sec. II and IV of the paper):
 *  Eq. (eqstate)  p^w = n T / (1 - b n) - a n^2
 *  Eq. (force2)   F_int = d(n T - p^w) + kappa n d(lap n)
 *  Eq. (periodicforce)  F_ext = (A0 sin(2 pi x / lambda), 0), x = column
 *  Eqs. (xstencil, laplstencil)  3x3 stencils with parameters N and Q
 *                 (M = (1 - 2N)/4, R = (1 - Q)/2; N = 1/2, Q = 1 is the
 *                 standard central scheme)
 *  Eq. (evoleq)   BGK relaxation time tau (in steps), tau > 1/2
 *  Moving walls   rows 0 and ny-1 move along x with u_bot and u_top; the
 *                 paper's shear rate gamma gives u_bot = -gamma (ny-1)/2,
 *                 u_top = +gamma (ny-1)/2.                               */
typedef struct {
  int32_t nx, ny;    /* columns (periodic) and rows; nx >= 1, ny >= 1, and
                        ny >= 3 when walls are on                           */
  int32_t walls;     /* 1: moving walls on rows 0 and ny-1; 0: periodic y  */
  int32_t precision; /* LB_FP64, LB_FP32, LB_BF16DEV or LB_FP16DEV        */
  double a, b;       /* van der Waals constants (lattice units)            */
  double T;          /* temperature (lattice units; T_c = 8a/(27b))        */
  double kappa;      /* square-gradient (surface tension) coefficient      */
  double tau;        /* relaxation time in steps                           */
  double A0, lambda; /* periodic force amplitude and wavelength (lambda = 0
                        switches the force off)                            */
  double u_bot, u_top; /* wall x-velocities                                */
  double N, Q;       /* stencil parameters                                 */
  double rho_ref;    /* reference density of 16-bit deviation storage; 0
                        selects the vdW critical density 1/(3b) (1 if b = 0);
                        ignored by LB_FP64 and LB_FP32                      */
  void *stream;      /* cudaStream_t to enqueue on; NULL = default stream  */
} lb_params;

typedef struct lb_handle lb_handle;

/* Create a solver for the problem *p and allocate its device state (two
 * population buffers of 9*nx*ny elements -- 16-bit storage: one float and
 * eight 16-bit planes -- plus small work buffers; 16-bit storage adds one
 * float copy of the nine planes for moments, reductions and init).
 * *out receives the handle.  Errors: LB_ERR_ARG (bad sizes, tau <= 1/2,
 * b*n range, precision), LB_ERR_CUDA, LB_ERR_OOM.                          */
int lb_create(const lb_params *p, lb_handle **out);

/* Initial condition: f*_i = f_i^eq(n0, u0) of Eq. (eqfunc), fluid at the
 * given density and velocity with no force correction.
 *  mode 0: noisy uniform density n0 = rho_mean + noise_amp (2U - 1), where
 *          U in [0,1) is the top 53 bits of output y*nx + x of the
 *          counter-based SplitMix64 generator seeded with `seed`
 *          (Steele, Lea & Flood 2014); u0 = 0.  rho0/ux0/uy0 are ignored.
 *  mode 1: n0 = rho0[ny][nx] (double, required); ux0 and uy0 (double,
 *          [ny][nx]) may each be NULL for zero velocity.  Host arrays
 *          (pageable or page-locked) or arrays in the handle's device
 *          memory: page-locked and device arrays are read by the init
 *          kernel in place, pageable ones are first copied to a device
 *          buffer.
 * Resets the step counter to 0.  Synchronises the stream when host arrays
 * are read.  Errors: LB_ERR_ARG, LB_ERR_CUDA.                             */
int lb_init(lb_handle *h, int mode, uint64_t seed, double rho_mean,
            double noise_amp, const double *rho0, const double *ux0,
            const double *uy0);

/* Advance by nsteps >= 0 time steps of Eq. (evoleq) -- propagation,
 * density (n-hat on wall rows), forces of Eq. (force2) + Eq.
 * (periodicforce), wall rule, u* of Eq. (newvel), equilibrium Eq.
 * (eqfunc), forcing Eqs. (forceterm, coeff), BGK collision -- one fused
 * kernel launch per step, enqueued on the handle's stream without
 * synchronising.  Errors: LB_ERR_STATE (not initialised), LB_ERR_CUDA.     */
int lb_step(lb_handle *h, int64_t nsteps);

/* Density n (n-hat on wall rows) and physical velocity u* of Eq. (newvel)
 * at the current time, i.e. the propagation, forces and wall rule of the
 * next step applied to the stored state, written to rho, ux, uy ([ny][nx],
 * element type `dtype`).  Any of the three may be NULL.  on_device = 1:
 * the pointers are device pointers and the call only enqueues work;
 * on_device = 0: host pointers, the call synchronises the stream (the
 * kernel writes page-locked arrays in place; pageable ones receive a copy).
 * Errors: LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA.                          */
int lb_moments(lb_handle *h, void *rho, void *ux, void *uy, int dtype,
               int on_device);

/* Global FP64 sums over the stored state: out[0] = total mass
 * sum_r sum_i f*_i (conserved by the scheme up to rounding, Sec. II),
 * out[1], out[2] = sum_r sum_i f*_i c_i (x, y).  The sums use a fixed
 * reduction order, so the result is deterministic.  Host pointer out[3];
 * synchronises the stream.  Returns LB_ERR_UNSTABLE if any population is
 * non-finite or any site's post-collision mass lies outside (0, 1/b).     */
int lb_reduce(lb_handle *h, double *out);

/* Asynchronous form of lb_reduce for monitoring every step without
 * stalling: enqueues the same sums on the handle's stream and a copy of
 * five doubles to the HOST array out[5]: out[0..2] as lb_reduce, out[3] =
 * 1.0 if a population is non-finite or a site's mass lies outside (0, 1/b)
 * (the condition lb_reduce reports as LB_ERR_UNSTABLE), else 0.0, out[4] =
 * 1.0 if a device-side wait gave up or a layout check failed (lb_reduce's
 * LB_ERR_TIMEOUT), else 0.0.  The values are there once the stream has
 * been synchronised; out must stay valid until then and should be pinned
 * (page-locked) memory -- with pageable memory the copy, and so the call,
 * synchronises.  Several calls may be in flight with different out arrays.
 * Errors: LB_ERR_ARG, LB_ERR_STATE, LB_ERR_CUDA.                          */
int lb_reduce_async(lb_handle *h, double *out);

/* Step-by-step monitoring with no call per step: register a HOST ring of
 * `capacity` records of six doubles in page-locked memory the device can
 * address (cudaHostAlloc, or a pinned torch tensor); host_ring = NULL or
 * capacity = 0 switches it off.  While it is set, every sweep step computes
 * the sums of lb_reduce and its kernel writes record (s mod capacity) =
 * {mass, momentum x, momentum y, unstable flag, wait/layout error flag, s}
 * straight into host memory, s being the step number after that step.  The
 * records of the steps enqueued so far are complete once the stream has
 * been synchronised; the ring must stay allocated while monitoring is on.
 * The call allocates the device-side per-step record slots for the current
 * tiling (synchronising the stream when it replaces smaller ones); while
 * monitoring, lb_step launches at most min(capacity, 64) steps at a time,
 * so each ring record is written once per launch and in step order.
 * Strip-sweep handles only (FP32 and 16-bit storage, not inside a batch).
 * Errors: LB_ERR_ARG (other handles, capacity < 0, memory the device cannot
 * address), LB_ERR_CUDA, LB_ERR_OOM.                                       */
int lb_monitor(lb_handle *h, double *host_ring, int32_t capacity);

/* Checkpoint: copy the stored populations to the HOST buffer buf:
 * [9][ny][nx] elements of the storage precision (double for LB_FP64, float
 * for LB_FP32); for 16-bit storage the float rest plane [ny][nx] followed by
 * the eight 16-bit deviation planes [8][ny][nx] (raw bfloat16 / binary16
 * bits), 20 bytes per site.  *bytes is the buffer size on
 * entry and the bytes needed on return; buf = NULL queries the size.
 * Synchronises the stream.  Errors: LB_ERR_ARG (buffer too small).       */
int lb_get_state(lb_handle *h, void *buf, size_t *bytes);

/* Restore populations written by lb_get_state of a handle with the same
 * nx, ny and precision (HOST buffer, exactly the size lb_get_state
 * reports) and set the step counter to `step`.  Continuing from a restored
 * state is bitwise identical to never having stopped.                      */
int lb_set_state(lb_handle *h, const void *buf, size_t bytes, int64_t step);

/* Tiling autotuner (a performance control of this library; the paper has
 * no counterpart).  Times `steps` steps of the strip-sweep kernel for each
 * candidate tiling -- segment height (rows per CTA, which trades CTAs per SM
 * against re-read warm-up rows) and strip count (the fewest strips and up
 * to three more of at least 64 columns, which changes how the tiles fill
 * the GPU) -- times the three fastest twice more and keeps the one with
 * the smallest of its three timings for later lb_step calls, and writes its
 * segment height to *seg_h (may be NULL; 0 when the handle uses the tile
 * kernel, which has no tiling choice; lb_get_tiling gives both).  The state and the step counter are restored
 * afterwards: the trajectory is the same as without the call.  Needs one
 * extra state buffer of device memory while it runs; synchronises the
 * stream.  Errors: LB_ERR_ARG (steps < 1), LB_ERR_STATE, LB_ERR_CUDA,
 * LB_ERR_OOM.                                                              */
int lb_autotune(lb_handle *h, int steps, int32_t *seg_h);

/* Set the strip-sweep kernel's segment height (rows per CTA) without
 * tuning, e.g. to a value an earlier lb_autotune chose; clamped to
 * [1, ny].  The trajectory does not depend on it beyond FP32 rounding
 * order.  No-op (LB_OK) for a handle on the tile kernel.  Host-side only
 * (may grow the per-CTA record array).  Errors: LB_ERR_ARG (seg_h < 1),
 * LB_ERR_CUDA, LB_ERR_OOM.                                                 */
int lb_set_seg_h(lb_handle *h, int32_t seg_h);

/* The strip-sweep tiling in use: number of column strips and segment
 * height (both 0 for a handle on the tile kernel).  A performance control
 * of this library; the paper has no counterpart.  Errors: LB_ERR_ARG (NULL
 * outputs).                                                                */
int lb_get_tiling(const lb_handle *h, int32_t *nstrips, int32_t *seg_h);

/* Set the tiling without tuning (e.g. one lb_get_tiling reported after
 * lb_autotune): nstrips column strips, at least the fewest the kernel's
 * window allows (ceil(nx / 116) for FP32, ceil(nx / 120) for 16-bit
 * storage) and at most nx / (2 * quantum) (quantum 4 columns for FP32, 8
 * for 16-bit storage); seg_h as lb_set_seg_h.  Strip s starts at column
 * s base + quantum min(s, extra) and is base or base + quantum wide (the
 * first `extra` strips wider), base = quantum floor(nx / (quantum nstrips)).
 * The trajectory is the same bit for bit for every tiling.  No-op for the
 * tile kernel.  Errors: LB_ERR_ARG (out of range), LB_ERR_CUDA, LB_ERR_OOM. */
int lb_set_tiling(lb_handle *h, int32_t nstrips, int32_t seg_h);

/* Dependency lists of the multi-step sweep, for inspection and tests (host
 * computation only, no GPU work; the paper has no counterpart).  For an
 * nx x ny lattice (walls 0 or 1) in `precision` (LB_FP32, LB_BF16DEV or
 * LB_FP16DEV) tiled as lb_set_tiling(nstrips, seg_h) describes, tile
 * t = strip + nstrips * segment (segment g covers rows g seg_h ..
 * min(ny, (g + 1) seg_h) - 1) waits, before each step of a multi-step
 * launch, for every tile in idx[ofs[t] .. ofs[t + 1]) to have finished the
 * previous step: the tiles that write a site (or a periodic image of one)
 * that its TMA window reads -- rows ya - 4 .. yb + 4, columns from x0 - 4
 * over the window's width -- and the tiles whose windows read its sites.
 * ofs: ntiles + 1 entries (HOST); idx: up to cap entries (HOST, may be
 * NULL when cap = 0); *count receives the number of entries.  Errors:
 * LB_ERR_ARG (a lattice or tiling the sweep does not take, or cap below
 * *count, which then holds the size needed).                               */
int lb_sweep_dependencies(int32_t precision, int32_t nx, int32_t ny, int32_t walls, int32_t nstrips,
                          int32_t seg_h, int32_t *ofs, int32_t *idx, int64_t cap, int64_t *count);

/* ------------------------------------------------------------------------
 * Batched solver: many independent lattices (different sizes and physical
 * parameters) advanced together, one kernel launch per step over a work
 * list of every instance's strips and segments (longest first), pairs of
 * steps replayed as a CUDA graph.  The paper solves one lattice at a time;
 * this is a throughput layer for parameter sweeps (e.g. over T, A0, lambda
 * and the wall velocity).
 * ------------------------------------------------------------------------ */
typedef struct lb_batch lb_batch;

/* Create `count` instances from ps[0..count-1].  All share one stream and
 * one precision (LB_FP32, LB_BF16DEV or LB_FP16DEV) and must satisfy the
 * sweep kernel's size rules (nx a multiple of 4, or of 8 for 16-bit
 * storage; nx, ny >= 8).  Errors: LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_OOM
 * (message from lb_batch_last_error(NULL)).                                */
int lb_batch_create(const lb_params *ps, int32_t count, lb_batch **out);

/* Instance i as an lb_handle, for lb_init, lb_moments, lb_reduce,
 * lb_get_state, lb_set_state, lb_get_step and lb_autotune (not lb_destroy:
 * the batch owns it).  Stepping it alone with lb_step is allowed.  NULL if
 * i is out of range.                                                       */
lb_handle *lb_batch_handle(lb_batch *b, int32_t i);

/* Advance every instance by nsteps >= 0 steps (asynchronous on the stream).
 * Afterwards lb_reduce of each instance costs one small kernel.
 * Errors: LB_ERR_STATE (an instance not initialised), LB_ERR_CUDA.         */
int lb_batch_step(lb_batch *b, int64_t nsteps);

/* Tiling autotuner for the batch: times `steps` batch steps for each
 * candidate segment height, first one height for all instances, then per
 * lattice class (ny <= 96, <= 160, > 160) with the others fixed, and keeps
 * the fastest.  seg_h (count entries, may be NULL) receives each instance's
 * choice.  States and step counters are restored.  Synchronises.          */
int lb_batch_autotune(lb_batch *b, int steps, int32_t *seg_h);

/* Release the batch and all its instances.  NULL is accepted. */
int lb_batch_destroy(lb_batch *b);

/* Last error message of a batch call (NULL: of the last lb_batch_create). */
const char *lb_batch_last_error(const lb_batch *b);

/* Number of steps taken since lb_init / lb_set_state. */
int lb_get_step(const lb_handle *h, int64_t *step);

/* Release the handle and its device memory (synchronises the stream).
 * NULL is accepted. */
int lb_destroy(lb_handle *h);

/* Allocation-free variant of lb_reduce (the paper has no counterpart; this
 * is a service for callers that cannot allocate device memory -- code
 * embedded in a host application that owns the device memory budget, or a
 * real-time loop where cudaMalloc may block).  It computes the same FP64
 * sums as lb_reduce (total mass, x and y momentum of the populations, and
 * the non-finite / out-of-range flag) over a caller-owned population buffer,
 * and allocates nothing: its scratch is one partial per lattice row in a
 * fixed device array of LB_NOALLOC_MAX_ROWS entries (32 bytes each, 512 KB
 * in all, held by every GPU that loads the library until process exit).
 *  f          DEVICE pointer, populations [9][ny][nx] (compact, x fastest)
 *             of type double (LB_FP64) or float (LB_FP32)
 *  b          van der Waals b; densities must lie in (0, 1/b) (b = 0: > 0)
 *  out        DEVICE pointer to 3 doubles: mass, momentum x, momentum y
 *  flag       DEVICE pointer to one int set to 1 if any site is non-finite
 *             or outside (0, 1/b), else 0; may be NULL
 *  stream     cudaStream_t to enqueue on (NULL = default stream)
 * Enqueues two kernels and returns without synchronising.  The first call on
 * a device looks up the scratch array's device address (once per device);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after cudaDeviceReset on a device it is stale,
 * so do not call this entry point on a device that has been reset.  All calls share the one
 * scratch array, so calls that overlap on the GPU race and must be
 * serialised by the caller.  The row partials are summed in a fixed order,
 * so results are deterministic; they equal lb_reduce's up to the order of
 * FP64 additions.  Errors: LB_ERR_ARG (null pointer, bad precision,
 * nx < 1, ny < 1 or ny > LB_NOALLOC_MAX_ROWS), LB_ERR_CUDA.                */
#define LB_NOALLOC_MAX_ROWS 16384
int lb_reduce_noalloc(const void *f, int precision, int32_t nx, int32_t ny, double b,
                      double *out, int *flag, void *stream);

/* Message for the last failed call on h (or for the last failed lb_create
 * when h is NULL).  The string stays valid until the next call on h.      */
const char *lb_last_error(const lb_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* LB_H_ */
