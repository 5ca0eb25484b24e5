/*
 * rt.h -- C ABI of the GB300 M1 radiative-transfer subcycle (libm1rt.so).
 *
 * The library advances the photon transport of Zier et al. (2024),
 * "Adapting AREPO-RT for Exascale Computing" (arXiv:2404.17630), on a static
 * unstructured mesh: for every frequency bin the photon number density N and
 * flux F obey the moment equations Eq. (E) and Eq. (F) in the conservative
 * form of Eq. (RT_flux), closed by the M1 Eddington tensor of Eq. (edd), and
 * exchange photons with a H/He gas (Sec. 2.3.1).  One call of rt_step runs
 * n_sub subcycles on the GPU (Sec. 2.3, Fig. overview_subcycling); each
 * subcycle is: source injection + thermochemistry, least-squares gradients
 * with a slope limiter (Sec. 2.3.2), face fluxes (Sec. 2.3.3) and the
 * per-cell gather of the stored face fluxes (Sec. 4.1.3).
 *
 * Conventions
 *  - Every entry point returns an rt_status; none aborts.  The message of the
 *    last failure is available from rt_last_error().
 *  - Array arguments may point to host memory or to device memory of the
 *    context's device; the library tells them apart itself
 *    (cudaPointerGetAttributes).  They are read or written during the call
 *    (copies are ordered on the context's stream and complete before return
 *    for host memory).  The library keeps no caller pointer after a call.
 *  - Cell arrays are indexed by the caller's cell order, face arrays by the
 *    caller's face order.  Multi-component arrays are component-major:
 *    N[b*C + i], F[(3*b + k)*C + i], x5[s*C + i].
 *  - Device memory of the mesh and state is owned by the context
 *    (cudaMalloc in rt_init_mesh, released by rt_destroy).
 *  - Kernels are launched on the stream given to rt_create (NULL = legacy
 *    default stream).  rt_step only enqueues work; device-side conditions
 *    (substep cap, non-finite values) are collected in a status word read
 *    by rt_sync().
 *
 * Units: geometry in a length unit L_u (rt_config.unit_length_cm cm each),
 * time in s, number densities (n_H, N, F/c_red) in cm^-3, photon rates in
 * photons/s, temperature in K, cross-sections in cm^2, energies in erg.
 */
#ifndef M1RT_RT_H
#define M1RT_RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rt_status;
enum {
  RT_OK = 0,
  RT_INVALID_ARG = 1,   /* bad pointer, size or configuration value */
  RT_BAD_MESH = 2,      /* face index out of range, self face, V <= 0, singular gradient matrix */
  RT_CFL = 3,           /* dt / n_sub above cfl * min V^(1/3) / c_red (Eq. timestep), nothing done */
  RT_CHEM_SUBSTEPS = 4, /* a cell needed more than max_substeps chemistry attempts (it stops there) */
  RT_NONFINITE = 5,     /* a photon density became NaN or Inf */
  RT_OOM = 6,           /* device allocation failed */
  RT_CUDA = 7,          /* other CUDA runtime error */
  RT_NOT_READY = 8,     /* call order: mesh or state missing */
  RT_TIMEOUT = 9        /* a kernel's bounded wait for its own asynchronous copies gave up */
};

enum { RT_FP64 = 0, RT_MIXED = 1 };

/* Field selectors of rt_get_fields (bit mask; outputs in this order). */
enum {
  RT_FIELD_N = 1,     /* photon number density, B*C */
  RT_FIELD_F = 2,     /* photon flux F (photons cm^-2 s^-1), 3*B*C */
  RT_FIELD_X = 4,     /* x_HI, x_HII, y_HeI, y_HeII, y_HeIII, 5*C */
  RT_FIELD_T = 8,     /* temperature, C */
  RT_FIELD_NSUB = 16  /* chemistry attempts of each cell in the last subcycle, C (as double) */
};

/* Method parameters (Sec. 2.2, 2.3).  The chemistry's rate coefficients are
 * fits the paper does not print: case-B recombination of HII and HeIII from
 * Hui & Gnedin (1997), HeII case B plus dielectronic recombination,
 * collisional ionisation and the cooling set from Katz, Weinberg & Hernquist
 * (1996). */
typedef struct {
  int n_bins;             /* 1..3 frequency bins (HI-, HeI-, HeII-ionising) */
  int precision;          /* RT_FP64, or RT_MIXED: FP32 transport sweep, FP64 update and chemistry (Sec. 6.2) */
  double c_red;           /* reduced speed of light, cm/s (RSLA, Sec. 2.2) */
  double unit_length_cm;  /* cm per geometry length unit */
  double box;             /* periodic box side in length units; 0 = not periodic */
  double cfl;             /* Courant factor eta of Eq. (timestep) */
  int chem_mode;          /* 0 transport only, 1 isothermal chemistry, 2 chemistry with thermal energy */
  int chem_flags;         /* bit0 recombination, bit1 collisional ionisation, bit2 cooling, bit3 photoheating */
  int limiter;            /* 1: slope limiter of Sec. 2.3.2 on */
  double lim_eps;         /* faces with |g.x| <= lim_eps |g||x| do not limit (1e-5) */
  int order;              /* 1: piecewise-constant states, 2: linear reconstruction */
  double f_s;             /* chemistry substep target change (0.05, Sec. 4.1.1) */
  double f_max;           /* chemistry substep rejection threshold (0.1, Sec. 4.1.1) */
  double x_floor;         /* abundance floor of the relative-change measure (1e-4) */
  int max_substeps;       /* chemistry attempts per cell and subcycle before RT_CHEM_SUBSTEPS */
  double y_he;            /* n_He / n_H */
  double sigma[3][3];     /* grey cross-sections [bin][HI, HeI, HeII], cm^2 */
  double eps[3][3];       /* heat per photoionisation [bin][species], erg */
  int gather_sum;         /* RT_MIXED only: 0 = each FP32 face flux widened and summed in FP64;
                             1 = compensated FP32 pair (error-free two_sum), widened to FP64 once per cell */
  int splitting;          /* 0 = Lie (sources + chemistry over the subcycle, then transport; the order of
                             Fig. overview_subcycling); 1 = Strang (sources + chemistry over half the subcycle
                             on each side of the transport step; the symmetric split of Sec. 2.3) */
  int time_order;         /* 1 = forward-Euler transport (no time extrapolation, Sec. 2.3.3);
                             2 = Heun's method in SSP form: U1 = U + dt L(U), U2 = U1 + dt L(U1),
                             U' = U/2 + U2/2 (second order in time, positive under the same CFL) */
} rt_config;

/* Cells of the static mesh (structure of arrays, n entries each). */
typedef struct {
  int64_t n;
  const double *volume;            /* V_i in L_u^3, > 0 */
  const double *cx, *cy, *cz;      /* centre of mass s_i */
} rt_cells;

/* Faces (interfaces) of the static mesh; each joins two distinct cells. */
typedef struct {
  int64_t n;
  const int32_t *left, *right;     /* cell ids; the unit normal points from left to right */
  const double *area;              /* A_f in L_u^2 */
  const double *nx, *ny, *nz;      /* unit normal */
  const double *fx, *fy, *fz;      /* face centroid */
} rt_faces;

typedef struct rt_ctx rt_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (or
 * NULL).  *out receives the context (NULL on failure). */
rt_status rt_create(const rt_config *cfg, void *stream, rt_ctx **out);

/* Replace the stream later calls enqueue on. */
rt_status rt_set_stream(rt_ctx *ctx, void *stream);

/* Copy the static mesh to the device; build the per-cell face lists (CSR,
 * ascending face index, Fig. GPU_memory_layout) and the per-cell inverse of
 * the least-squares matrix of Eq. (normalEquation), which depends only on
 * geometry (Sec. 2.3.2).  Resets the state to neutral gas at 1e4 K, n_H = 0,
 * no radiation, no sources.  RT_BAD_MESH on an invalid mesh. */
rt_status rt_init_mesh(rt_ctx *ctx, const rt_cells *cells, const rt_faces *faces);

/* Gas: nH[C] (cm^-3), x5[5*C] (x_HI, x_HII, y_HeI, y_HeII, y_HeIII), T[C] (K). */
rt_status rt_set_gas(rt_ctx *ctx, const double *nH, const double *x5, const double *T);

/* Radiation: N[B*C] photon number densities (cm^-3); F[3*B*C] photon
 * fluxes (cm^-2 s^-1), stored internally as F / c_red.  F may be NULL (zero).
 * RT_FP64 keeps both in FP64.  RT_MIXED keeps N in FP64 and F / c_red in
 * FP32 (the state the FP32 sweep reads), so rt_get_fields returns F / c_red
 * rounded to FP32, times c_red. */
rt_status rt_set_radiation(rt_ctx *ctx, const double *N, const double *F);

/* Point sources: source k emits Q[k*B + b] photons/s in bin b into cell
 * cell[k] (S of Eq. E).  Rates of sources sharing a cell add up in source
 * order.  n = 0 removes all sources. */
rt_status rt_set_sources(rt_ctx *ctx, int64_t n, const int64_t *cell, const double *Q);

/* Individual time steps (Sec. 2.1: cells on a power-of-two time-step
 * hierarchy, only the active ones integrated in a step).  active[C] (host or
 * device bytes, nonzero = active) holds for the following rt_step calls;
 * NULL = every cell active (the default).  In each subcycle only active cells
 * get sources and thermochemistry; fluxes are computed for the interfaces
 * with at least one active cell (Sec. 4.1.3) and applied to both of their
 * cells, so a passive cell changes only through the interfaces it shares
 * with active cells and the photon number stays conserved.  The work is
 * proportional to the active cells and their neighbours.  rt_adjoint needs
 * every cell active (RT_INVALID_ARG otherwise). */
rt_status rt_set_active(rt_ctx *ctx, const uint8_t *active);

/* Enqueue one RT step of n_sub subcycles of dt/n_sub seconds each.  Host-side
 * checks only (RT_CFL, RT_NOT_READY, RT_INVALID_ARG); see rt_sync. */
rt_status rt_step(rt_ctx *ctx, double dt, int n_sub);

/* Wait for the context's stream; return and clear the device status word
 * (RT_CHEM_SUBSTEPS, RT_NONFINITE) or a CUDA error. */
rt_status rt_sync(rt_ctx *ctx);

/* Copy the fields selected in mask (RT_FIELD_*) into out[0], out[1], ...
 * in the order of the bits, caller's cell order. */
rt_status rt_get_fields(rt_ctx *ctx, uint32_t mask, double *const *out);

/* Largest subcycle length (s) allowed by Eq. (timestep) on this mesh. */
rt_status rt_max_dt(rt_ctx *ctx, double *out);

/* Mesh statistics: number of cells, faces, and the largest cell degree. */
rt_status rt_mesh_info(rt_ctx *ctx, int64_t *n_cells, int64_t *n_faces, int32_t *max_degree);

/* Stage entry points (same kernels as rt_step, for per-stage checks):
 *  rt_stage_gradients: limited gradients of the current state into
 *    G[((i*B + b)*4 + q)*3 + d] (q: N, F_x/c, F_y/c, F_z/c; d: x, y, z), per L_u;
 *  rt_stage_fluxes: from G (or, if G is NULL, from freshly computed
 *    gradients) the face fluxes A_f * Phi / c_red into flux[(f*B + b)*4 + q];
 *  rt_stage_transport: gradients, fluxes and their application over dt
 *    (both Heun stages when time_order is 2);
 *  rt_stage_chemistry: source injection and thermochemistry over dt. */
rt_status rt_stage_gradients(rt_ctx *ctx, double *G);
rt_status rt_stage_fluxes(rt_ctx *ctx, const double *G, double *flux);
rt_status rt_stage_transport(rt_ctx *ctx, double dt);
rt_status rt_stage_chemistry(rt_ctx *ctx, double dt);

/* Reverse mode of rt_step(dt, n_sub): FP64 precision, any chem_mode (the
 * thermal network included: rate fits and cooling differentiated in T), Lie
 * splitting and forward-Euler transport (other configurations return
 * RT_INVALID_ARG).
 * The paper has no adjoint; this is the exact derivative of the discrete
 * forward map (sources, every chemistry attempt with the substep controller
 * of Sec. 4.1.1, gradients and limiter on their active branch, M1 face
 * fluxes, flux application).  Starting from the context's current state it
 * runs the step (leaving the final state, as rt_step does), keeping a full
 * checkpoint every checkpoint_every subcycles and recording the last
 * segment on the way, then walks back segment by segment, recording each
 * earlier segment again from its checkpoint.  The record of a segment is the
 * state entering each subcycle's chemistry and transport, and every
 * chemistry attempt of the cells whose first attempt was rejected, written
 * by the forward's own worklist pass.  The reverse of those attempts runs
 * their cotangent-independent part in parallel over a subcycle's records,
 * then each cell's serial chain.
 * In (cotangents of the final fields, caller layout, NULL = zero):
 *   lam_N[B*C], lam_F[3*B*C] (w.r.t. F, photons cm^-2 s^-1), lam_x5[5*C], lam_T[C].
 * Out (NULL = not wanted): dL_dQ[n_src*B] per source of the last
 *   rt_set_sources call (photons/s), dL_dnH[C], and the cotangents of the
 *   initial fields lam0_N, lam0_F, lam0_x5, lam0_T (same layouts).
 * Synchronous.  RT_INVALID_ARG for RT_MIXED, Strang splitting or Heun. */
rt_status rt_adjoint(rt_ctx *ctx, double dt, int n_sub, int checkpoint_every, const double *lam_N,
                     const double *lam_F, const double *lam_x5, const double *lam_T, double *dL_dQ,
                     double *dL_dnH, double *lam0_N, double *lam0_F, double *lam0_x5, double *lam0_T);

/* The chemistry tape of the last rt_adjoint call on ctx (all 0 before the
 * first): max_records = the most chemistry records one segment held (one
 * per attempt of each cell whose first attempt was rejected), capacity =
 * the tape's size in records (176 bytes each; it grows, and stays grown,
 * when a subcycle overflows it), redone = subcycle chemistries recorded
 * again after the tape grew.  NULL outputs are skipped; RT_INVALID_ARG for
 * a NULL ctx. */
rt_status rt_adjoint_tape_info(rt_ctx *ctx, long long *max_records, long long *capacity, int *redone);

/* Per-kernel timing: with profiling on, every kernel that rt_step and the
 * stage entry points launch is bracketed by CUDA events on the context's
 * stream.  rt_profile_read waits for the stream and returns, per kernel
 * class k (RT_KERNEL_*), the summed device time ms[k] (milliseconds) and the
 * number of launches[k] since the last reset; reset != 0 clears them.
 * n = length of the caller's arrays (at most RT_KERNEL_COUNT are filled). */
enum { RT_KERNEL_CHEM = 0, RT_KERNEL_GRAD = 1, RT_KERNEL_FLUX = 2, RT_KERNEL_GATHER = 3, RT_KERNEL_COUNT = 4 };
rt_status rt_profile_enable(rt_ctx *ctx, int on);
rt_status rt_profile_read(rt_ctx *ctx, int n, double *ms, int64_t *launches, int reset);

/* Number of subcycle kernels (RT_KERNEL_* classes) launched on ctx since it
 * was created; mesh setup and state transfer kernels are not counted. */
rt_status rt_launch_count(rt_ctx *ctx, int64_t *out);

/* Failure-path check (not a step of the method): enqueues one block that
 * waits on an mbarrier phase nothing completes, giving up after `polls`
 * polls (1..65536) the way every bounded device wait of the library does;
 * the block records the timeout in the status word.  rt_sync then returns
 * RT_TIMEOUT, and the context stays usable.  RT_INVALID_ARG for polls out of
 * range. */
rt_status rt_selftest_wait_timeout(rt_ctx *ctx, uint32_t polls);

/* Measured FP64 peak of the current device, the denominator of the FP64
 * rooflines (the FP64 sweep and the chemistry are bound by the FP64 unit).
 * Not a step of the method: the measurement that the roofline needs.  One
 * kernel of 8 independent fused multiply-add chains per thread, 8 blocks of
 * 256 threads per SM, `iters` iterations (1..2^20), timed with CUDA events on
 * `stream` (NULL: the default stream) after one warm-up launch; the best of
 * `reps` (1..100) launches.  *tflops = 2 x FMAs / time / 1e12; *ms_best (may
 * be NULL) the best launch in milliseconds.  Allocates (and frees) one small
 * output buffer; synchronises on its events.  RT_INVALID_ARG for arguments
 * out of range, RT_CUDA for a failed CUDA call; message from
 * rt_fp64_peak_last_error(). */
rt_status rt_fp64_peak(void *stream, int iters, int reps, double *tflops, double *ms_best);
const char *rt_fp64_peak_last_error(void);

/* Allocation-free gradients, for callers that cannot allocate device memory
 * (a host framework that owns all device memory through its own pool, a
 * real-time loop that must not allocate, a plug-in that only receives device
 * pointers).  The paper has no counterpart: it is an interface of this
 * library, not a step of the method.  It computes the same limited
 * least-squares gradients as rt_stage_gradients, for a mesh and state that
 * the caller passes as DEVICE arrays:
 *   cells: centroids (volume unused); faces: left, right, area, centroids
 *   (normals unused); cell_off[C+1] and cell_faces[2F]: per-cell face lists,
 *   entry (face << 1) | side with side 1 where the cell is the face's right
 *   cell, ascending face order (the layout rt_init_mesh builds);
 *   N[B*C], F_red[3*B*C]: photon densities and reduced fluxes F / c_red;
 *   G[C*B*12] out, layout as rt_stage_gradients; *bad_cell (device int) is
 *   set to 1 if a cell's least-squares matrix is singular, else 0.
 * Every array must be device memory of the current device (or managed
 * memory); anything else, device memory of another GPU included, gets
 * RT_INVALID_ARG before anything is enqueued.  The arrays must describe a
 * valid mesh (ids in range); they are not checked.
 * Its only scratch is a static device array of 6 doubles per cell for at
 * most 262144 cells (12.6 MB held on every GPU that loads the library until
 * the process exits); larger meshes get RT_INVALID_ARG.  Nothing is
 * allocated.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) and caches it with the device's current
 * context; a call made after that context was replaced (cudaDeviceReset)
 * looks it up again.  Make the first call on a device, and the first after
 * a reset, before any stream capture.  All calls on a device share the
 * array: work enqueued by calls that may overlap on the GPU (other streams,
 * unordered host threads) races.  Asynchronous on stream; host-side errors
 * and failed launches of its own kernels are returned as status codes, with
 * a message from rt_noalloc_last_error(); an error the caller left pending
 * in the CUDA runtime is neither reported nor cleared. */
rt_status rt_gradients_noalloc(const rt_cells *cells, const rt_faces *faces, const int32_t *cell_off,
                               const int32_t *cell_faces, int n_bins, int order, int limiter, double lim_eps,
                               double box, const double *N, const double *F_red, double *G, int *bad_cell,
                               void *stream);
const char *rt_noalloc_last_error(void);

/* Message of the last failed call on ctx (or of the last failed rt_create
 * when ctx is NULL).  Valid until the next call. */
const char *rt_last_error(const rt_ctx *ctx);

/* Release all device memory of ctx.  NULL is allowed. */
void rt_destroy(rt_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* M1RT_RT_H */
