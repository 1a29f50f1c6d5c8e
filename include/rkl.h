/*
 * rkl.h - C ABI of the GB300 RKL2 anisotropic-conduction library.
 *
 * The library advances dT/dt = M(T) = -div F, F the face-centred thermal
 * conduction flux of Vaidya et al. 2017 (arXiv:1702.05487), with the s-stage
 * second-order Runge-Kutta-Legendre (RKL2) super-time-step.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Arrays are cell-centred, C-ordered [z][y][x] (x fastest), contiguous,
 *   of the grid's dtype (float for RKL_F32, double for RKL_F64).
 * - The unit field b is ndim contiguous planes [bx][by]([bz]), each one
 *   grid-sized; b is the direction of B (Eq. Fclass), |b| = 1 is not checked.
 * - Face arrays: F_d at cell c holds the flux on the face c + e_d/2.
 * - Pointers passed to the plan functions are DEVICE pointers owned by the
 *   caller, 16-byte aligned; the library never frees them.  rkl_run_host
 *   takes HOST pointers.
 * - Work is enqueued on the plan's CUDA stream.  Functions returning a host
 *   scalar (rkl_dt_expl, rkl_energy, rkl_super_step) synchronise that stream.
 * - Every function returns an rkl_status.  Invalid arguments are rejected
 *   with RKL_ERR_INVALID_ARG before anything is launched.  No C++ exception
 *   crosses this boundary.  rkl_last_error(plan) gives a message.
 * - Physical model (rho = 1, gamma = 2 so the energy variable is T, Section
 *   4.1 of the paper): kappa_par = kappa_par0 (constant) or
 *   kappa_par0 * T^(5/2) (Spitzer); kappa_perp = kappa_perp_ratio *
 *   kappa_par; both evaluated at the face temperature (T_L + T_R)/2.
 */
#ifndef RKL_H
#define RKL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rkl_status {
    RKL_OK = 0,
    RKL_ERR_INVALID_ARG = 1,    /* bad pointer, size, dt, s or option           */
    RKL_ERR_CUDA = 2,           /* a CUDA runtime call failed                   */
    RKL_ERR_NONFINITE = 3,      /* a stage produced NaN or Inf                  */
    RKL_ERR_NONPOSITIVE_T = 4,  /* a stage produced T <= 0 with Spitzer kappa   */
    RKL_ERR_TIMEOUT = 5,        /* a bounded device wait gave up                */
    RKL_ERR_UNSUPPORTED = 6,    /* valid request this build does not implement  */
    RKL_ERR_NOMEM = 7           /* device or host allocation failed             */
} rkl_status;

enum { RKL_PERIODIC = 0, RKL_DIRICHLET = 1 };
enum { RKL_F32 = 0, RKL_F64 = 1 };
enum { RKL_KAPPA_CONST = 0, RKL_KAPPA_SPITZER = 1 };

/* Uniform Cartesian grid. */
typedef struct rkl_grid {
    int ndim;            /* active axes 1, 2 or 3 (x, then y, then z)              */
    int64_t n[3];        /* cells along x, y, z; axes beyond ndim must be 1        */
    double dx[3];        /* spacing along x, y, z (> 0 on active axes)             */
    int bc;              /* RKL_PERIODIC, or RKL_DIRICHLET: ghost cells (edges and
                            corners too) hold T = bc_value and copy b from the
                            nearest interior cell                                  */
    double bc_value;
    int dtype;           /* RKL_F32 or RKL_F64: state and arithmetic type          */
} rkl_grid;

/* Conduction physics (Eqs. Fc, Fclass, Fsat, dt_exp of the paper). */
typedef struct rkl_phys {
    int kappa_model;         /* RKL_KAPPA_CONST or RKL_KAPPA_SPITZER (T^(5/2)) */
    double kappa_par0;       /* > 0                                            */
    double kappa_perp_ratio; /* >= 0                                           */
    int saturate;            /* 1: F = q/(q + |F_class|) F_class (Eq. Fc) with
                                q = 5 phi rho c_iso^3, c_iso = sqrt(T) (Eq. Fsat) */
    double phi;              /* saturation factor (0.3 in the paper)          */
    double rho;              /* density in q only                             */
    int sat_upwind;          /* 1: c_iso from the cell the normal flux leaves;
                                0: from the face temperature                  */
    double cp;               /* parabolic Courant number C_p <= 1/2 (Eq. dt_exp) */
    int limiter;             /* RKL_LIMITER_NONE: transverse gradients are the
                                mean of the four one-sided differences (Eq. qT);
                                RKL_LIMITER_MC: the monotonised-central limiter
                                of Appendix C, MC(MC(up_L, down_L),
                                MC(up_R, down_R)), at faces whose lower
                                temperature is below limiter_floor (generic
                                kernel and the one-cell tiled kernel; the
                                paired-cell kernel for 3D FP32 with the floor
                                at +inf only)                                 */
    double limiter_floor;    /* +inf limits every face (Section 3.4: limiters
                                only where T falls below a floor)            */
} rkl_phys;
enum { RKL_LIMITER_NONE = 0, RKL_LIMITER_MC = 1 };

typedef struct rkl_plan rkl_plan;

/* Human-readable name of a status code (static storage). */
const char *rkl_status_string(rkl_status st);

/* Last error message recorded on a plan ("" if none); NULL plan gives the
 * message of the last failed rkl_plan_create or
 * rkl_dt_expl_energy_noalloc on this thread. */
const char *rkl_last_error(const rkl_plan *plan);

/*
 * Number of RKL2 stages for a super-step dt = ratio * dt_expl: Eq. RKL-s of
 * the paper, dt = dt_p (s^2 + s - 2)/4, solved for real s and rounded as
 * s -> 1 + floor(s) (Section 4.1).  ratio must be finite and > 0.
 * Host only, FP64.  Writes *s_out (>= 2).
 */
rkl_status rkl_num_stages(double ratio, int *s_out);

/*
 * RKL2 coefficients of Appendix A for s >= 2 stages, FP64: w_1 =
 * 4/(s^2+s-2), b_0 = b_1 = b_2 = 1/3, b_j = (j^2+j-2)/(2j(j+1)), a_j = 1 - b_j,
 * mu_j = ((2j-1)/j)(b_j/b_{j-1}), nu_j = -((j-1)/j)(b_j/b_{j-2}),
 * mut_1 = b_1 w_1, mut_j = mu_j w_1, gt_j = -a_{j-1} mut_j.
 * Each output is a caller-owned host array of s + 1 doubles indexed by j;
 * entries without a definition (j = 0, and mu/nu/gt at j = 1) are 0.
 * Host only.  s must be in [2, 4096].
 */
rkl_status rkl_coeffs(int s, double *mu, double *nu, double *mut, double *gt);

/*
 * Super-time-stepping methods of Section 3.3.  RKL2 (Appendix A) is the
 * default and the only second-order one; RKL1 and AAG-STS are the
 * first-order methods the paper compares it with.  All three run through
 * the same stage kernels with different coefficient tables:
 *   RKL1  : stability polynomial P_s(1 + w_1 z), w_1 = 2/(s^2+s); Eq. RKL-s
 *           gives dt/dt_expl = (s^2+s)/2, s = 1 + floor of its root;
 *           stages Y_1 = Y_0 + w_1 tau M(Y_0), Y_j = mu_j Y_{j-1}
 *           + nu_j Y_{j-2} + mu_j w_1 tau M(Y_{j-1}), mu_j = (2j-1)/j,
 *           nu_j = -(j-1)/j (the Legendre recursion, Eq. recLegP).
 *   AAG-STS (damping sts_nu in (0, 1)): N forward-Euler sub-steps tau_j =
 *           dt_p / ((nu-1) cos((2j-1) pi/(2N)) + 1 + nu); N is the smallest
 *           count whose super-step of Eq. AAG-STS reaches dt/dt_expl, and
 *           dt_p = dt / gain(N) so that the sub-steps sum to dt.
 * In the coefficient arrays of rkl_coeffs_method the stage update is
 *   Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + (1 - mu_j - nu_j) Y_0
 *         + mut_j tau M(Y_{j-1}) + gt_j tau M(Y_0)
 * (Y_{-1} := Y_0 at j = 1), so RKL1 has gt = 0 and AAG-STS mu = 1, nu = 0,
 * gt = 0, mut_j = tau_j / dt.
 */
enum { RKL_METHOD_RKL2 = 0, RKL_METHOD_RKL1 = 1, RKL_METHOD_STS = 2 };

/*
 * Stage count of a method for ratio = dt/dt_expl > 0 (sts_nu is read only by
 * RKL_METHOD_STS and must lie in (0, 1)).  Host only, FP64.  Writes *s_out
 * (>= 2 for RKL2, >= 1 otherwise).  RKL_ERR_INVALID_ARG past 4096 stages.
 */
rkl_status rkl_num_stages_method(int method, double ratio, double sts_nu, int *s_out);

/*
 * Coefficients of a method for s stages in the form stated above, FP64, as
 * caller-owned host arrays of s + 1 doubles indexed by j (j = 0 unused).
 * s in [2, 4096] for RKL2, [1, 4096] otherwise.  Host only.
 */
rkl_status rkl_coeffs_method(int method, int s, double sts_nu, double *mu, double *nu,
                             double *mut, double *gt);

/*
 * Create a plan for one grid and physics on a CUDA stream (cudaStream_t
 * passed as void*; NULL is the legacy default stream).  The plan allocates
 * its own device workspace: three stage buffers, M(Y_0), reduction scratch
 * (4 grid arrays plus a few KB) and caches one CUDA graph per distinct
 * (s, T, b) triple used by rkl_super_step.  The device current at creation
 * is used for every later call.  Writes *out; destroy with
 * rkl_plan_destroy.
 */
rkl_status rkl_plan_create(const rkl_grid *grid, const rkl_phys *phys,
                           void *cuda_stream, rkl_plan **out);
rkl_status rkl_plan_destroy(rkl_plan *plan);

/*
 * Explicit parabolic step of Eq. dt_exp: C_p / max_cells sum_d chi_d/dx_d^2
 * with chi_d = kappa_par(T) + kappa_perp(T) (gamma = 2, rho = 1), the max
 * taken in FP64 over the device array T.  Synchronises the stream.
 */
rkl_status rkl_dt_expl(rkl_plan *plan, const void *T, double *dt_out);

/*
 * Face fluxes F_d, d < ndim, of Eqs. Fc/Fclass/Fsat with the normal
 * gradient across the face and the transverse gradients of Eqs. qN/qT
 * averaged to the face from the four neighbouring one-sided differences;
 * b and T on the face are the means of the two cells.  Fx, Fy, Fz are device
 * arrays of grid size (pass NULL for axes beyond ndim).  Asynchronous.
 */
rkl_status rkl_flux(rkl_plan *plan, const void *T, const void *b,
                    void *Fx, void *Fy, void *Fz);

/*
 * M(T) = -sum_d (F_d(c + e_d/2) - F_d(c - e_d/2)) / dx_d, the conservative
 * divergence of Section 3 (one flux per face).  Asynchronous.
 */
rkl_status rkl_apply_M(rkl_plan *plan, const void *T, const void *b, void *MT);

/*
 * One stage of Eq. rkl2scheme (Appendix A) with tau = dt, 1 <= j <= s:
 *   j = 1:  MY0 = M(Y0) (written), Y1 = Y0 + mut_1 tau MY0
 *   j >= 2: Yj = mu_j Yjm1 + nu_j Yjm2 + (1 - mu_j - nu_j) Y0
 *                + mut_j tau M(Yjm1) + gt_j tau MY0
 * j = 1 ignores Yjm1 and Yjm2.  s = 1 is accepted as forward Euler
 * (Yj = Y0 + tau M(Y0)).  The coefficients are those of the plan's method
 * (rkl_plan_set_method; RKL2 by default).  For j >= 2 Yj may alias Y0 (Y0 is read only at
 * the cell being written) but no other input; for j = 1 Yj aliases nothing
 * (M reads Y0 at neighbouring cells).  Asynchronous.
 */
rkl_status rkl_stage(rkl_plan *plan, int j, int s, double dt, const void *b,
                     const void *Y0, void *MY0, const void *Yjm1,
                     const void *Yjm2, void *Yj);

/*
 * One RKL2 super-step of length dt applied in place to the device array T:
 * dt_expl from T (Eq. dt_exp), s = rkl_num_stages(dt/dt_expl) (or
 * rkl_num_stages_method for the plan's method), FP64
 * coefficients (rounded once to the grid dtype), then the s stages launched
 * as one cached CUDA graph.  Optionally the FP64 energy sum_c T_c dV before
 * and after (pass NULL to skip).  *s_used receives s (may be NULL).
 * Returns RKL_ERR_NONFINITE / RKL_ERR_NONPOSITIVE_T if a stage of this or an
 * earlier, unchecked super-step produced such values (the state is then
 * undefined).  Synchronises the stream once for dt_expl and once more only
 * when energies are requested.
 */
rkl_status rkl_super_step(rkl_plan *plan, double dt, void *T, const void *b,
                          int *s_used, double *energy_before, double *energy_after);

/*
 * As rkl_super_step, but s is given (s >= 2; s >= 1 for RKL1 and AAG-STS)
 * instead of chosen from dt_expl;
 * no synchronisation unless energies are requested.
 */
rkl_status rkl_super_step_s(rkl_plan *plan, double dt, int s, void *T, const void *b,
                            double *energy_before, double *energy_after);

/*
 * Operator splitting (Section 3: the hyperbolic step without the conduction
 * flux, then Eq. scalar_diffusion).  The hyperbolic part provided here is
 * the passive advection dT/dt = -div(u T) of the energy density by a
 * cell-centred velocity u (device array [3][ncell] in the grid dtype, x, y,
 * z components; ghosts copy the nearest interior cell).
 *
 * rkl_dt_hyperbolic: Eq. dt_h with lambda_d = |u_d| (a passive flow has no
 * sound speed): C_h / max_cells sum_d |u_d| / dx_d, or 0 if u = 0.  Uses one
 * stage buffer of the plan as scratch; synchronises.
 *
 * rkl_advect: one conservative first-order donor-cell step,
 * T_out = T_in - dt sum_d (F_d(c + 1/2) - F_d(c - 1/2)) / dx_d with face
 * flux F = u_f T(upwind cell), u_f the mean of the two cells' u; monotone
 * and positive for dt <= rkl_dt_hyperbolic(C_h = 1).  T_out must not alias
 * T_in.  Asynchronous.
 */
rkl_status rkl_dt_hyperbolic(rkl_plan *plan, const void *u, double C_h, double *dt_out);
rkl_status rkl_advect(rkl_plan *plan, double dt, const void *u, const void *T_in, void *T_out);

/* FP64 energy sum_c T_c dV of a device array.  Synchronises. */
rkl_status rkl_energy(rkl_plan *plan, const void *T, double *E_out);

/*
 * Kernel choice for the stage launches of this plan: 0 = automatic (the
 * row-pair kernel where it applies, else the paired-cell kernel, else the
 * tiled kernel, else the generic kernel), 1 = the generic one-thread-per-cell kernel, 2 = the
 * tiled FP32 3D kernel (32 x 8 tiles, one cell per thread), 3 and 4 = the
 * paired-cell FP32 3D kernel (64 x 4 tiles, two cells per thread in packed
 * f32x2 arithmetic; needs nx % 4 == 0) built for 20 (variant 3) or 24
 * (variant 4) resident warps per SM, 5 = the two-stage kernel (stages j and
 * j + 1 per pass over the grid, 60 x 7 tiles; periodic only; allocates a
 * fourth stage buffer), 6 = the paired-cell kernel with its plane bundles
 * copied by the TMA engine (cp.async.bulk rows with mbarrier completion;
 * periodic grids with nx >= 72, else as 3), 7 = the paired-cell kernel with
 * the Y0 / Y_{j-2} / M(Y0) bundles of stages j >= 2 copied by the TMA engine
 * from tensor maps (cp.async.bulk.tensor, one issuing thread; as 3 where the
 * driver offers no tensor-map encoder), 8 = the paired-cell kernel with
 * every plane bundle (T and b with their halo ring, Y0, Y_{j-2}, M(Y0))
 * copied by the TMA engine from tensor maps, the periodic images at the
 * grid's edges patched in by a few threads (periodic grids with nx >= 72
 * and ny >= 6, no limiter; else as 3), 9 = the paired-cell kernel with
 * tiles 32 columns wide and 8 rows high (two rows of 16 lanes per warp;
 * for grids whose width is an odd multiple of 32, where 64-column tiles
 * leave a quarter to a half of the last tile idle; no limiter, else as 3),
 * 10 = the row-pair kernel (the paired-cell arithmetic with two cell pairs
 * per thread, rows 2w and 2w + 1 of 64 x 8 tiles, three CTAs per SM; the
 * same bits as the paired-cell kernel; periodic grids with fewer than 2^31
 * cells, nx % 4 == 0, no limiter or the MC limiter at every face
 * (limiter_floor = +inf, a limited build with 64-column tiles), else
 * RKL_ERR_UNSUPPORTED; nzchunk <= 0 picks the chunk length), 11 = the row-pair kernel with tiles 32 columns
 * wide and 16 rows high (two row pairs per warp, one per half-warp; same
 * conditions and bits as 10; variant 0 takes it where the width is an odd
 * multiple of 32).  With the MC limiter at every face
 * (limiter_floor = +inf) variants 0, 10 and 11 launch the row-pair kernel's
 * limited build on periodic grids, variants 3, 4, 6 and 7 the paired-cell
 * kernel's (20 resident warps per SM, per-thread copies; the same bits);
 * with a finite floor neither applies.
 * RKL_ERR_UNSUPPORTED if the kernel does not apply to the grid.  nzchunk = planes per CTA of the paired-cell
 * kernels (0: chosen from the grid and the SM count, at least 3.5 waves of
 * CTAs where the grid has that many and a last wave that is nearly full); a
 * negative value selects the balanced schedule instead: one launch of 5 (or
 * 6) CTAs per SM in which every CTA marches an equal run
 * of the grid's (tile column, plane) pairs.  Drops cached graphs.  Results
 * of all kernels and schedules agree within FP32 rounding.
 */
rkl_status rkl_plan_set_variant(rkl_plan *plan, int variant, int nzchunk);

/*
 * Selects the super-time-stepping method used by rkl_super_step,
 * rkl_super_step_s and rkl_stage (RKL_METHOD_RKL2 by default; sts_nu is the
 * AAG-STS damping, read only for RKL_METHOD_STS).  A plan created for RKL2
 * keeps its workspace; the coefficient table is rebuilt at the next call.
 */
rkl_status rkl_plan_set_method(rkl_plan *plan, int method, double sts_nu);

/*
 * Autotuner: times one super-step of length dt (s from dt / dt_expl(T))
 * with every kernel variant and z-chunk that applies to the grid (generic;
 * tiled; paired-cell at 5 and 6 CTAs per SM, automatic, balanced or with 16,
 * 32, 64 planes per CTA; two-stage; bulk and tensor-map copies; row-pair) on a
 * scratch copy of T (T is not changed), keeps the fastest with
 * rkl_plan_set_variant and returns it.  Allocates and frees one grid-sized
 * scratch array.  Synchronises.
 */
rkl_status rkl_plan_autotune(rkl_plan *plan, double dt, const void *T, const void *b,
                             int *variant_out, int *nzchunk_out, double *ms_out);

/*
 * Waits for the plan's stream and returns the device status word collected
 * by the stage kernels since the last check (RKL_OK, RKL_ERR_NONFINITE or
 * RKL_ERR_NONPOSITIVE_T), then clears it.
 */
rkl_status rkl_plan_check(rkl_plan *plan);

/*
 * Per-launch timing of the hot stage kernel.  With timing on, the graphs of
 * rkl_super_step record CUDA events on the plan's stream around stages
 * 2..s; rkl_plan_timing synchronises, adds up the elapsed times of all
 * completed super-steps since timing was switched on and returns the total
 * milliseconds and the number of stage launches they cover.
 */
rkl_status rkl_plan_set_timing(rkl_plan *plan, int on);
rkl_status rkl_plan_timing(rkl_plan *plan, double *ms_total, int64_t *launches);

/*
 * End-to-end run from host memory: copies T_host and b_host to the device,
 * performs n_super super-steps of length dt (s chosen per super-step as in
 * rkl_super_step) and copies T back into T_host.  Host buffers should be
 * page-locked for full copy speed.  Allocates (and frees) device buffers
 * for T and b on each call unless they fit the plan's cached staging
 * buffers, which are kept for reuse.  *s_last receives the last s
 * (may be NULL).  Synchronises.
 */
rkl_status rkl_run_host(rkl_plan *plan, double dt, int n_super, void *T_host,
                        const void *b_host, int *s_last);

/*
 * Streams n_jobs independent problems of the plan's grid through the GPU:
 * job i copies T_host[i] and b_host[i] (the layouts of rkl_super_step) to
 * the device, performs n_super super-steps of length dt and copies T back
 * into T_host[i]; s_last[i] receives its last s (s_last may be NULL).  Three
 * device staging sets (kept with the plan) and two private copy streams
 * let the copy-in of job i + 1 and the copy-out of job i - 1 overlap the
 * super-steps of job i on the plan's stream and each other, so with
 * page-locked buffers the jobs cost about max(copy-in, compute, copy-out)
 * each.  Job i's buffers must not alias those of jobs i - 1 and i + 1; a
 * T_host[i] equal to T_host[i - 2] is allowed (its copy-in then waits for
 * job i - 2's copy-out).  Synchronises.
 */
rkl_status rkl_run_host_batch(rkl_plan *plan, double dt, int n_super, int n_jobs, void *const *T_host,
                              const void *const *b_host, int *s_last);

/* ------------------------------------------------------------------------
 * Ensembles: many independent 3D FP32 problems advanced together, each with
 * its own grid, conductivity, super-step and stage count (Eq. RKL-s per
 * problem), sharing kappa_model and the saturation flag.  Problem p's cells
 * live at [off[p], off[p+1]) of one caller-owned device array T_all and its
 * three b planes at [3 off[p], 3 off[p+1]) of b_all (rkl_ensemble_layout
 * gives off).  The ensemble owns the stage buffers (4 floats per cell).
 */
typedef struct rkl_ensemble rkl_ensemble;

/* grids[p], phys[p] for p < nprob; every grid 3D, RKL_F32, nx % 4 == 0. */
rkl_status rkl_ensemble_create(int nprob, const rkl_grid *grids, const rkl_phys *phys,
                               void *cuda_stream, rkl_ensemble **out);
rkl_status rkl_ensemble_destroy(rkl_ensemble *ens);
const char *rkl_ensemble_last_error(const rkl_ensemble *ens);

/* Writes nprob + 1 cell offsets (multiples of 4) into cell_offsets. */
rkl_status rkl_ensemble_layout(const rkl_ensemble *ens, int64_t *cell_offsets);

/*
 * Schedule of rkl_ensemble_super_step, two flags: bit 0 (persistent = 1 or
 * 3) runs every stage of every problem in one persistent launch (work items
 * (problem, stage, tile) in stage-major order; a tile of stage j waits,
 * with a bounded spin, until all tiles of stage j-1 of its problem are
 * done), else one kernel is launched per problem and stage; bit 1
 * (persistent = 2 or 3) takes the row-pair tile body (64 x 8 tiles, or
 * 32 x 16 for widths that are odd multiples of 32; three CTAs per SM)
 * instead of the paired-cell one (64 x 4, or 32 x 8; five CTAs per SM).
 * The two tile bodies write the same bits.  nzchunk = planes per tile
 * (<= 0: 32).  RKL_ERR_INVALID_ARG for persistent outside 0..3;
 * RKL_ERR_UNSUPPORTED for the row-pair tiles unless every problem is
 * periodic with fewer than 2^31 cells (the autotuner then skips them).
 */
rkl_status rkl_ensemble_set_schedule(rkl_ensemble *ens, int persistent, int nzchunk);

/*
 * One RKL2 super-step of every problem: dt[p] is problem p's super-step
 * (host array); s_p = rkl_num_stages(dt[p] / dt_expl_p) with dt_expl_p from
 * problem p's current T (FP64 per-problem maxima, one synchronisation).
 * T_all is updated in place.  s_used (host, nprob ints) may be NULL.
 * Errors detected by earlier super-steps (NaN, T <= 0, a timed-out wait)
 * are returned here or by rkl_ensemble_check.
 */
rkl_status rkl_ensemble_super_step(rkl_ensemble *ens, const double *dt, void *T_all,
                                   const void *b_all, int *s_used);

/* Waits for the stream; returns and clears the device status word. */
rkl_status rkl_ensemble_check(rkl_ensemble *ens);

/*
 * Autotuner: times one super-step of every candidate schedule (persistent
 * with nzchunk 8, 16, 32; per-launch with 16, 32; each with either tile
 * body; persistent row-pair with 48, 64) on a scratch copy of
 * T_all (T_all itself is not changed), keeps the fastest and returns it.
 * Allocates and frees one T_all-sized scratch array.
 */
rkl_status rkl_ensemble_autotune(rkl_ensemble *ens, const double *dt, const void *T_all,
                                 const void *b_all, int *persistent_out, int *nzchunk_out,
                                 double *ms_out);

/*
 * Failure-detection self-test of the persistent kernel: launches it on a
 * work list whose dependency can never be met, with a short spin limit;
 * the kernel must give up, raise the timeout bit and return.  Writes
 * RKL_ERR_TIMEOUT to *status_out when the bounded wait worked.
 */
rkl_status rkl_ensemble_selftest_timeout(rkl_ensemble *ens, int *status_out);

/* ------------------------------------------------------------------------
 * Learned surrogate of one super-step (no counterpart in the paper; the
 * RKL2 super-step above is its fallback and the reference for its error).
 * Network: 6 periodic 3x3x3 convolutions, channels 6 -> 32 -> 32 -> 32 ->
 * 32 -> 32 -> 3, ReLU between layers, BF16 weights and activations with
 * FP32 accumulation on tensor cores.  Inputs per cell: T - 1, b_x, b_y,
 * b_z, log10(kappa_par(T) / 0.01), (dt/dt_expl) / 100.  The three output
 * channels are face fluxes G_d and the predicted increment is
 *   dT = -head_scale * sum_d (G_d(c) - G_d(c - e_d)) / dx_d,
 * a conservative divergence, so sum dT = 0 (exact energy conservation up
 * to rounding).  Patch: D x H x W periodic cells with D % 4 == H % 8 ==
 * W % 16 == 0.  Layer l has weights [27][cout][cin] (offset o = ((dz+1) 3 +
 * dy+1) 3 + dx+1, channels padded: layer 0 cin 16 (6 used), layer 5 cout 16
 * (3 used), padded entries must stay 0) and bias [cout]; FP32 masters on
 * the device, Adam moments kept per parameter.  All device work runs on
 * the stream given at creation; rkl_sur_super_step also uses the plan's
 * stream, which must be the same stream.
 */
typedef struct rkl_surrogate rkl_surrogate;

rkl_status rkl_sur_layer_shape(int layer, int *cout, int *cin);
rkl_status rkl_sur_create(int D, int H, int W, const double *dx, void *cuda_stream,
                          rkl_surrogate **out);
rkl_status rkl_sur_destroy(rkl_surrogate *sur);
const char *rkl_sur_last_error(const rkl_surrogate *sur);
/* host <-> device copies of layer parameters (w: 27*cout*cin floats, b: cout) */
rkl_status rkl_sur_set_params(rkl_surrogate *sur, int layer, const float *w, const float *b);
rkl_status rkl_sur_get_params(rkl_surrogate *sur, int layer, float *w, float *b);
/* gradients of the last rkl_sur_backward / rkl_sur_train_step */
rkl_status rkl_sur_get_grads(rkl_surrogate *sur, int layer, float *gw, float *gb);
/* input channels from device arrays T [cells] and b [3][cells] */
rkl_status rkl_sur_features(rkl_surrogate *sur, const void *T, const void *b, double kappa_par0,
                            int spitzer, double dt_over_dtexpl);
/*
 * Convolution backend of the forward and backward-data passes: 0 the
 * warp-level mma.sync kernels, 1 the tcgen05 kernels (M = 128-voxel blocks
 * of one plane, accumulators in tensor memory; needs W % 8 == 0 and
 * H % 16 == 0, else RKL_ERR_UNSUPPORTED).  The default is 1 where the
 * patch allows it.  Weight gradients use the warp-level kernel either way.
 */
rkl_status rkl_sur_set_backend(rkl_surrogate *sur, int backend);
/*
 * The input features with three more channels (6, 7, 8): flux_scale times
 * the face fluxes F_x, F_y, F_z of T (Eqs. Fclass, qN, qT, Fsat as the
 * plan evaluates them, rkl_flux: the flux on face i + 1/2 stored at i).
 * T's flux carries the field-aligned product b (b . grad T) that a ReLU
 * network would otherwise have to learn; the kappa model is the plan's.
 * The plan must describe the surrogate's periodic 3D FP32 patch.
 */
rkl_status rkl_sur_features_flux(rkl_surrogate *sur, rkl_plan *plan, const void *T, const void *b,
                                 double ratio, double flux_scale);
/* c > 0: rkl_sur_super_step builds its features with rkl_sur_features_flux
 * and flux_scale = c dt / head_scale (dt: the super-step); c = 0 (the
 * default): rkl_sur_features */
rkl_status rkl_sur_set_flux_features(rkl_surrogate *sur, double c);
/* waits for the stream; RKL_ERR_TIMEOUT if a tcgen05 kernel's bounded wait
 * gave up since the last check (the word is then cleared) */
rkl_status rkl_sur_check(rkl_surrogate *sur);
/* forward pass; the increment dT goes to dT_out (device floats) if not NULL */
rkl_status rkl_sur_forward(rkl_surrogate *sur, double head_scale, void *dT_out);
/* MSE loss 0.5 mean((dT - target)^2) of the last forward and all gradients */
rkl_status rkl_sur_backward(rkl_surrogate *sur, const void *target, double *loss);
/* one Adam step on every parameter (bias-corrected, step counter kept) */
rkl_status rkl_sur_adam(rkl_surrogate *sur, double lr, double beta1, double beta2, double eps);
/* forward + backward + Adam (beta1 0.9, beta2 0.999, eps 1e-8) */
rkl_status rkl_sur_train_step(rkl_surrogate *sur, double head_scale, const void *target, double lr,
                              double *loss);
/*
 * One layer of the network on caller-owned device buffers, with the
 * surrogate's current BF16 weights of that layer and its patch size
 * (voxel v = (z H + y) W + x, channels last; asynchronous on the stream).
 * These are the kernels rkl_sur_forward / rkl_sur_backward run, exposed one
 * at a time so that each can be checked on its own (all three are periodic
 * 3x3x3 cross-correlations, offset o = 9 (dz+1) + 3 (dy+1) + (dx+1)):
 *   forward:       in bf16 [V][cin] -> out bf16 [V][cout] = ReLU(bias +
 *                  sum_o sum_ci w[o][co][ci] in[v + o][ci]), or for the
 *                  last layer f32 [V][16] without the ReLU;
 *   backward_data: layer >= 1; dz bf16 [V][cout], mask bf16 [V][cin] ->
 *                  out bf16 [V][cin] = (sum_o sum_co w[o][co][ci]
 *                  dz[v - o][co]) where mask > 0, else 0;
 *   weight_grad:   dz bf16 [V][cout], x bf16 [V][cin] -> the layer's
 *                  gradients (read with rkl_sur_get_grads): dW[o][co][ci] =
 *                  sum_v dz[v][co] x[v + o][ci], db[co] = sum_v dz[v][co],
 *                  summed in a fixed order (the same result every run).
 * The forward and backward-data passes use the backend of
 * rkl_sur_set_backend; the weight gradient is the warp-level kernel.
 * (cin, cout) of a layer: rkl_sur_layer_shape.
 */
rkl_status rkl_sur_layer_forward(rkl_surrogate *sur, int layer, const void *in, void *out);
rkl_status rkl_sur_layer_backward_data(rkl_surrogate *sur, int layer, const void *dz, const void *mask,
                                       void *out);
rkl_status rkl_sur_layer_weight_grad(rkl_surrogate *sur, int layer, const void *dz, const void *x);

/*
 * One super-step of length dt with the surrogate: predicts dT, computes the
 * trapezoidal-rule residual rho = ||dT - (dt/2)(M(T) + M(T + dT))|| / ||dT||
 * (two applications of M; with flux features, rkl_sur_set_flux_features,
 * M(T) is the divergence of the face fluxes the features already evaluated,
 * so only M(T + dT) is a full evaluation), accepts T + dT if rho <= threshold, otherwise
 * runs rkl_super_step (the fallback).  *accepted, *residual, *s_used (0
 * when accepted) are written.  The plan must describe the same periodic 3D
 * FP32 patch.
 */
rkl_status rkl_sur_super_step(rkl_surrogate *sur, rkl_plan *plan, double dt, void *T,
                              const void *b, double head_scale, double threshold,
                              int *accepted, double *residual, int *s_used);

/*
 * dt_expl and energy without allocating.  The paper has no counterpart to
 * this entry point; it exists for callers that cannot allocate device
 * memory where they need these numbers (creating a plan allocates, and
 * cudaMalloc / cudaFree may synchronise the whole device): for example a
 * host code that hands the library a fixed memory budget up front, or a
 * time-step loop that must not stall on an allocation.
 *
 * Computes the same dt_expl as rkl_dt_expl and the same FP64 energy
 * (sum T dV) as rkl_energy for the device array T of the given grid,
 * without a plan, on cuda_stream (void* cudaStream_t), and synchronises
 * that stream.  Writes *dt_out and *energy_out (host).  One difference:
 * this entry point always reads every cell of T and fails with
 * RKL_ERR_NONFINITE if any holds NaN or Inf, whatever the kappa model
 * (rkl_dt_expl does not read T under constant kappa, and rkl_energy sums
 * NaN without an error).
 *
 * Scratch: a fixed array inside the library (about 1.5 MB, held on every
 * GPU that loads the library until the process exits), enough for grids of
 * at most 2^27 = 134217728 cells; larger grids are rejected with
 * RKL_ERR_INVALID_ARG before anything is launched.  No cudaMalloc, cudaFree
 * or other allocating routine is called.  The first call on each device
 * looks up the array's device address (once per device, with that device
 * current), so make that first call before any stream capture.  All calls
 * share the one array: calls whose GPU work overlaps (unordered streams)
 * race on it.  Each call overwrites every scratch entry it reads.
 * Errors: RKL_ERR_INVALID_ARG (bad grid/phys, an axis d >= ndim with
 * n[d] != 1, or too many cells),
 * RKL_ERR_NONFINITE (T holds NaN/Inf), RKL_ERR_NONPOSITIVE_T (T <= 0 under
 * Spitzer kappa), RKL_ERR_CUDA; the message is in rkl_last_error(NULL).
 */
rkl_status rkl_dt_expl_energy_noalloc(const rkl_grid *grid, const rkl_phys *phys,
                                      const void *T, void *cuda_stream,
                                      double *dt_out, double *energy_out);

#ifdef __cplusplus
}
#endif

#endif /* RKL_H */
