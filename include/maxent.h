/*
 * maxent.h -- C-ABI of the GB300 (sm_103a) maximum-entropy moment solver.
 *
 * The library advances the 5-moment (1D1V) and 14-moment (3D3V) fourth-order
 * maximum-entropy systems with the interpolative closure of McDonald &
 * Torrilhon, as used by Boccelli, Kaufmann, Magin & McDonald (JCP 2024,
 * arXiv 2401.15233), with an explicit cell-centred finite-volume scheme:
 * MUSCL reconstruction of primitive moments with one shared limiter
 * (Sec. 3.2; a field whose two stencil differences are both within 1e-10
 * of its natural scale -- rho, sqrt(p/rho), p, p sqrt(p/rho), p^2/rho --
 * counts as flat and does not limit the others, so round-off in a field
 * that is uniform in exact arithmetic cannot drop the scheme to first
 * order), HLL or Rusanov face fluxes (Sec. 3.1) with the approximate
 * wave speeds of Sec. 5 / Appendix B, BGK relaxation sources (Sec. 2.3,
 * 2.4), forward Euler or midpoint RK2 in time (Sec. 3) under a CFL condition.
 *
 * The calls follow the paper's statement of the problem: an initial state,
 * boundary states imposed in ghost cells (Sec. 6), a relaxation time
 * (Sec. 2.1, Sec. 4), time marching, and moments read back.
 *
 * Ownership and threading
 *   - A context owns all device memory it allocates; mxe_destroy frees it.
 *   - Pointers passed in are borrowed for the duration of the call only.
 *   - Work is issued on the context's CUDA stream (mxe_set_stream); calls
 *     that return host data synchronise that stream.  A context must not be
 *     used from two host threads at once.
 *   - Every call returns an mxe_status; MXE_OK is 0.  On error the context's
 *     message (mxe_last_error) says what failed; no call aborts the process.
 *
 * Array layouts (double precision, structure of arrays)
 *   2D grid:  soa[k * ny * nx + j * nx + i], k = field, j = row (y), i = column (x)
 *   1D tubes: fields of tube n follow each other: soa[k * ncells_n + i],
 *             tubes concatenated in order (mxe_batch_* calls).
 *   5-moment primitive fields : (rho, u, P, q, r)                  Sec. 2.3
 *   14-moment primitive fields: (rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz,
 *                                Pzz, qx, qy, qz, R)                Sec. 2.4
 *   q is the full third central moment (q_i = Q_ijj, twice the fluid heat
 *   flux, Sec. 2.1).  Conserved fields are the balance-law densities.
 */
#ifndef MAXENT_H
#define MAXENT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MXE_OK = 0,
    MXE_EINVAL = 1,          /* bad argument (size, enum, pointer, range)      */
    MXE_ENOMEM = 2,          /* device or host allocation failed               */
    MXE_ECUDA = 3,           /* a CUDA runtime call failed                     */
    MXE_EUNREALIZABLE = 4,   /* input state not realizable (rho<=0, P not SPD,
                                sigma > 1)                                     */
    MXE_ENONFINITE = 5,      /* a non-finite value appeared in the state       */
    MXE_ETIMEOUT = 6,        /* a bounded device wait gave up                  */
    MXE_ESTATE = 7           /* call not valid in the context's current state  */
} mxe_status;

enum { MXE_FP64 = 0, MXE_MIXED = 1 };                 /* precision            */
enum { MXE_FLUX_HLL = 0, MXE_FLUX_RUSANOV = 1 };      /* Sec. 3.1             */
enum { MXE_LIM_MINMOD = 0, MXE_LIM_VANALBADA = 1 };   /* Sec. 3.2             */
enum { MXE_FE = 0, MXE_RK2 = 1 };                     /* Sec. 3               */
enum { MXE_BC_TRANSMISSIVE = 0, MXE_BC_PERIODIC = 1, MXE_BC_DIRICHLET = 2 };
enum { MXE_SIDE_XLO = 0, MXE_SIDE_XHI = 1, MXE_SIDE_YLO = 2, MXE_SIDE_YHI = 3 };
enum { MXE_TAU_NONE = 0, MXE_TAU_CONST = 1, MXE_TAU_HARDSPHERE = 2 };
enum { MXE_PRIMITIVE = 0, MXE_CONSERVED = 1, MXE_SIGMA = 2, MXE_CONSERVED_RESTORE = 3 };
enum { MXE_SOURCE_EXPLICIT = 0, MXE_SOURCE_POINT_IMPLICIT = 1 };

typedef struct {
    int    system;       /* 5 (1D1V, Sec. 2.3) or 14 (3D3V, Sec. 2.4)            */
    int    nx, ny;       /* cells; ny == 1 means one space dimension (x)          */
    double x0, x1, y0, y1;                    /* domain                            */
    int    precision;    /* MXE_FP64 or MXE_MIXED (FP32 stage arithmetic, FP64
                            state accumulator and FP64 closure near sigma -> 0 or
                            sigma -> 1)                                         */
    int    flux;         /* MXE_FLUX_*                                            */
    int    limiter;      /* MXE_LIM_* (shared most-stringent limiter, Sec. 3.2)   */
    int    order;        /* 1 (piecewise constant) or 2 (MUSCL)                   */
    int    integrator;   /* MXE_FE or MXE_RK2 (midpoint)                          */
    double cfl;          /* Courant number (0.5 in Sec. 6)                        */
    double sigma_lim;    /* lower bound on sigma inside closure and wave speeds
                            (Appendix A; 1e-4 in the paper)                      */
    double k_ws;         /* wave-speed inflation k >= 1 (Sec. 5.1)                */
} mxe_config;

typedef struct {
    double    t;                /* simulated time                                  */
    double    last_dt;          /* last time step taken                            */
    long long steps;            /* steps taken since mxe_set_state                 */
    double    max_rate;         /* CFL denominator sum_d max|lambda_d|/dx_d        */
    double    min_sigma;        /* minimum raw sigma over cells (14- or 5-moment)  */
    long long n_sigma_below_lim;/* cells with sigma < sigma_lim                    */
    long long n_sigma_above_one;/* cells with sigma > 1 (unrealizable)             */
    long long n_nonpositive;    /* cells with rho <= 0 or a non-positive pressure  */
    long long n_nonfinite;      /* cells with a non-finite conserved value         */
    long long n_fp64_closures;  /* MIXED: face states re-evaluated in FP64 since
                                   mxe_set_state                                   */
    long long n_closures;       /* MIXED: face states evaluated since mxe_set_state*/
    double    sums[14];         /* sum over cells of each conserved field          */
    long long planar;           /* 1 if the 2D 14-moment state is planar (u_z,
                                   P_xz, P_yz, q_z zero in the state and all
                                   boundary states): those moments stay zero
                                   and are neither stored nor computed        */
} mxe_diag;

typedef struct mxe_ctx mxe_ctx;

/* ---- context ------------------------------------------------------------- */

/* Create a solver for one grid (ny >= 1).  Validates the configuration
 * (system in {5,14}; 5-moment requires ny == 1; nx >= 4; cfl > 0;
 * 0 <= sigma_lim < 1; k_ws >= 1) and allocates the device state.
 * Default BCs: transmissive on every side; default relaxation: none. */
mxe_status mxe_create(const mxe_config *cfg, mxe_ctx **out);

/* Free all device memory of the context.  NULL is allowed. */
void mxe_destroy(mxe_ctx *ctx);

/* Issue all further work on `stream` (a cudaStream_t; NULL = the context's
 * own non-blocking stream).  The stream is borrowed, not owned. */
mxe_status mxe_set_stream(mxe_ctx *ctx, void *stream);
void      *mxe_get_stream(const mxe_ctx *ctx);

/* Set the state from a SoA array of nf*ny*nx doubles (kind PRIMITIVE or
 * CONSERVED; primitives are converted on the device).  on_device != 0: soa
 * is a device pointer; otherwise a host pointer: page-locked host memory
 * (pinned or registered) is read once by the checking kernel itself over the
 * host link, pageable memory is copied to the device first.  Resets t = 0
 * and the step count.  Every cell is
 * checked (rho > 0, finite, positive pressure); a failing state returns
 * MXE_EUNREALIZABLE with the first offending cell in the message and
 * leaves the previous state in place.  Kind CONSERVED_RESTORE takes a
 * conserved state verbatim without the realizability check: it restores a
 * state this solver produced (a checkpoint read with mxe_get_moments),
 * which the scheme itself may have left slightly outside sigma <= 1. */
mxe_status mxe_set_state(mxe_ctx *ctx, int kind, const double *soa, int on_device);

/* Read the state into a SoA array (kind PRIMITIVE, CONSERVED; or SIGMA: one
 * field, the raw sigma of Eq. (sigma-mapping-5mom/14mom)).  A page-locked
 * host array is written directly by the conversion kernel, a pageable one
 * through a device copy.  Synchronises. */
mxe_status mxe_get_moments(mxe_ctx *ctx, int kind, double *soa, int on_device);

/* Boundary condition of one side (Sec. 6: states imposed in two ghost
 * layers).  type TRANSMISSIVE copies the nearest interior cell, PERIODIC
 * wraps (must be set on both opposite sides), DIRICHLET imposes the
 * primitive state `prim` (nf values).  With lo < hi and type DIRICHLET the
 * state is imposed only on ghost cells whose tangential centre coordinate
 * lies in [lo, hi] (an inflow slot); up to 4 slots per side, the rest of
 * the side keeps its base type.  lo >= hi sets the base type of the side
 * and clears its slots. */
mxe_status mxe_set_bc(mxe_ctx *ctx, int side, int type, double lo, double hi,
                      const double *prim);

/* Relaxation time of the BGK source (Sec. 2.1, Sec. 4):
 *   NONE       collisionless (no source)
 *   CONST      tau = tau_ref everywhere
 *   HARDSPHERE tau = tau_ref (rho_ref/rho) sqrt(T_ref/T), T = P/rho (1D1V) or
 *              tr(P)/(3 rho) (3D3V); with tau_ref = Kn L_ref / sqrt(8 T_ref/pi)
 *              this is lambda/v_th with lambda proportional to 1/rho. */
mxe_status mxe_set_relaxation(mxe_ctx *ctx, int model, double tau_ref, double rho_ref,
                              double T_ref);

/* How the BGK source enters a stage (the closing remark of Sec. 4.3: once
 * the source limits an explicit step, below Kn ~ 1e-4, a simple
 * point-implicit treatment suffices).  MXE_SOURCE_EXPLICIT (default): the
 * source is part of the stage residual.  MXE_SOURCE_POINT_IMPLICIT: the
 * stage advances the flux divergence only, V = U_base + h (-div F) with h
 * the stage's step (dt/2 for the RK2 midpoint stage, dt otherwise), and
 * then solves dU/dt = -(U - U_M)/tau by backward Euler over h; the source
 * keeps density, momentum and energy, so the Maxwellian U_M and tau are V's
 * and U = U_M + (V - U_M)/(1 + h/tau) in closed form (density and momentum
 * are kept as they are).  The CFL step is unchanged (it never included the
 * source).  Applies to every tube of a batch.  MXE_EINVAL for another
 * value.  The adjoint entry points return MXE_ESTATE on a context with the
 * point-implicit source. */
mxe_status mxe_set_source_scheme(mxe_ctx *ctx, int scheme);

/* March until t_end or max_steps steps, with dt = min(cfl/max_rate, t_end-t)
 * recomputed every step on the device (Sec. 3; the CFL reading of the
 * oracle).  t_out / steps_out (may be NULL) receive the new time and the
 * steps taken in this call; passing either synchronises, and so does every
 * chunk of a call with max_steps > 4.  Returns MXE_ENONFINITE if a
 * non-finite value appeared, MXE_EUNREALIZABLE if a cell lost positivity
 * (rho <= 0 or a diagonal pressure <= 0: the scheme does not guarantee
 * realizability, and the wave speeds of such a state are undefined) or if
 * the CFL step size collapsed to zero before t_end (a non-finite wave
 * speed); the state is left as the last step wrote it.  These are found
 * from the device clock, i.e. when the call synchronises; an asynchronous
 * call (max_steps <= 4, no t_out / steps_out) reports them on the next
 * synchronising call or through mxe_get_diagnostics. */
mxe_status mxe_step(mxe_ctx *ctx, int max_steps, double t_end, double *t_out,
                    int *steps_out);

/* Take n steps with prescribed time steps dts[0..n-1] (host array) instead
 * of the CFL value (e.g. a recorded sequence). */
mxe_status mxe_step_dt(mxe_ctx *ctx, int n, const double *dts);

/* MXE_MIXED only: which face states are re-evaluated in FP64 (raw sigma in
 * [sigma_lim, sigma_lo) near the Junk subspace, sigma > sigma_hi near the
 * realizability boundary, or det P* < det_min for an ill-conditioned
 * pressure tensor; defaults 0 (off), 0.999, 1e-3) and how often (in steps)
 * the FP32 primitive cache is re-derived from the FP64 conserved state
 * (default 16).  det_min > 1 sends every face state to FP64 (det P* <= 1
 * always, since tr P* = 3). */
mxe_status mxe_set_mixed_policy(mxe_ctx *ctx, double sigma_lo, double sigma_hi,
                                double det_min, int resync_every);

/* 2D MXE_MIXED only: launch shape of the fused stage kernels (planar
 * ten-field and general fourteen-field).  blocks_per_sm = 3 (default): at
 * most 80 registers per thread, three blocks per SM, the final stage's own
 * cells prefetched into L2; 2: up to 128 registers per thread, two blocks per
 * SM (planar: the final stage prefetches its own cells' U^n and W^n into
 * shared memory).  The results do not depend on it (the arithmetic is the
 * same).  MXE_EINVAL for another value, MXE_ESTATE on another kind of
 * context. */
mxe_status mxe_set_stage_occupancy(mxe_ctx *ctx, int blocks_per_sm);

/* 2D MXE_MIXED only, planar states at three blocks per SM: how the two face
 * states of a face are evaluated (closure Eqs. closure-14mom-Qijk/Rijkk/
 * Sijjkk, wave speeds Eq. 14mom-approx-ws-equations, Sec. 3.1 flux).
 * packed = 1 (default): as one pair in packed FP32 (f32x2) arithmetic, the
 * left state in one lane and the right state in the other; a face whose
 * closure is ill-conditioned in either state (mxe_set_mixed_policy) takes
 * both states in FP64.  packed = 0: one state after the other in scalar
 * FP32, only the ill-conditioned state in FP64.  The two agree to FP32
 * rounding.  MXE_EINVAL for another value, MXE_ESTATE on another kind of
 * context. */
mxe_status mxe_set_face_packing(mxe_ctx *ctx, int packed);

/* Diagnostics of the current state (synchronises). */
mxe_status mxe_get_diagnostics(mxe_ctx *ctx, mxe_diag *out);

/* Last error message of the context (never NULL; "" if none). */
const char *mxe_last_error(const mxe_ctx *ctx);

/* ---- batched 1D tubes ---------------------------------------------------- */

/* Create n independent 1D problems (cfg->ny must be 1; cfg->nx is ignored):
 * tube b has ncells[b] cells on [0, length[b]].  All tubes share system,
 * precision, scheme, CFL and boundary conditions (transmissive by default);
 * each has its own state, relaxation time and clock.  mxe_set_state /
 * mxe_get_moments act on the concatenation of all tubes.  The whole batch
 * advances in one persistent launch.  MXE_FP64: one thread block per tube.
 * MXE_MIXED (14-moment system): teams of CTAs (thread-block clusters of
 * 1, 2, 4 or 8 CTAs of 128 or 256 threads, see mxe_batch_autotune) take
 * tubes from a device work queue, longest expected work (cells / dx) first;
 * each mxe_batch_run / mxe_step replays a cached CUDA graph of that launch.
 * Errors: MXE_EINVAL for a bad tube list (n < 1, ncells[b] < 4, length[b]
 * <= 0), MXE_ENOMEM / MXE_ECUDA when device allocation fails. */
mxe_status mxe_batch_create(const mxe_config *cfg, int n, const int *ncells,
                            const double *length, mxe_ctx **out);

/* Per-tube relaxation (same models as mxe_set_relaxation). */
mxe_status mxe_batch_set_relaxation(mxe_ctx *ctx, int tube, int model, double tau_ref,
                                    double rho_ref, double T_ref);

/* Per-tube times and step counts (host arrays of n, may be NULL). */
mxe_status mxe_batch_get_clock(mxe_ctx *ctx, double *t, long long *steps);

/* Advance every tube until its own t reaches t_end or it has taken
 * max_steps steps in this call.  MXE_FP64: one launch, one block per tube.
 * MXE_MIXED: one persistent launch of teams of CTAs (clusters) over a work
 * queue ordered by expected work (largest first); when the teams cannot use
 * every CTA slot of the device (clusters are placed whole within a GPU
 * processing cluster), a second, concurrent launch of single CTAs takes the
 * smallest tubes (see mxe_batch_get_layout).  Dividing the tubes estimates
 * each tube's steps from its current CFL rate (a small kernel, and a
 * synchronisation of the context stream, whenever the run's graph is
 * captured: a new t_end, max_steps, block shape or launch argument).
 * Results do not depend on which launch, team or CTA advances a tube. */
mxe_status mxe_batch_run(mxe_ctx *ctx, int max_steps, double t_end);

/* MXE_MIXED tube contexts: time every block shape (128 or 256 threads per
 * CTA x teams of 1, 2, 4 or 8 CTAs) on the current state advanced by t_probe
 * (each candidate from the same saved state and clocks, which are restored
 * afterwards) and keep the fastest for later runs.  Shapes that cannot be
 * resident on the device are skipped.  Outputs (may be NULL): the chosen
 * threads per CTA, CTAs per team and its time in ms.  Allocates (and frees)
 * one temporary copy of the state; synchronises the context stream.
 * Errors: MXE_ESTATE (not an MXE_MIXED 1D context, or no state),
 * MXE_EINVAL (t_probe <= 0), MXE_ECUDA. */
mxe_status mxe_batch_autotune(mxe_ctx *ctx, double t_probe, int *nt_out, int *cl_out,
                              double *ms_out);

/* MXE_MIXED tube contexts: set the block shape directly (nt in {128, 256},
 * cl in {1, 2, 4, 8}); the default is 128 x 1. */
mxe_status mxe_batch_set_shape(mxe_ctx *ctx, int nt, int cl);

/* MXE_MIXED tube contexts: the launch layout of the last mxe_batch_run;
 * before the first run, or after mxe_batch_set_shape or mxe_batch_autotune,
 * that of the team launch alone.  Outputs (may be NULL): teams of the team
 * launch, the tubes handed to it (the largest, in work order), and the CTAs
 * of the fill launch of single CTAs that takes the remaining tubes (0: no
 * fill launch).
 * The fill share is the largest tail of the work order whose estimated time
 * on the fill CTAs stays within the teams' estimate, with no tube longer
 * alone than that estimate; a tube's estimate is CTA passes over a chunk
 * times its steps in the run, min(max_steps, (t_end - t) m / CFL) with m the
 * CFL rate of its current state (prescribed steps count as given).
 * Errors: MXE_ESTATE (not an MXE_MIXED 1D context), MXE_ECUDA. */
mxe_status mxe_batch_get_layout(mxe_ctx *ctx, int *teams, int *team_tubes, int *fill_ctas);

/* The division mxe_batch_run makes, as a host-only computation (no context,
 * no device): n tubes in work order (largest first) with cells[q] cells and
 * an estimated steps[q] steps in the run, chunks of `chunk` cells per CTA
 * pass, `teams` teams of cl CTAs and `fill` single fill CTAs.  Output: the
 * number of leading tubes for the teams (the rest go to the fill CTAs; n when
 * fill is 0) and the estimated run time in CTA-pass units (may be NULL).
 * MXE_EINVAL for n < 1, a NULL array, chunk, cl or teams < 1, fill < 0, a tube
 * of < 1 cell or a negative or non-finite step estimate. */
mxe_status mxe_batch_plan_fill(int n, const int *cells, const double *steps, int chunk, int cl,
                               int teams, int fill, int *team_tubes, double *est_time);

/* ---- time-step history (2D grids) --------------------------------------- */

/* Keep the dt of every step in a device buffer of `capacity` entries
 * (entry s = step s counted from the last mxe_set_state; later steps are
 * not kept); 0 switches it off.  Synchronises; MXE_ESTATE for 1D contexts. */
mxe_status mxe_set_dt_history(mxe_ctx *ctx, long long capacity);

/* Copy the first n kept step sizes to the host array out (synchronises).
 * MXE_EINVAL if n exceeds the capacity. */
mxe_status mxe_get_dt_history(mxe_ctx *ctx, long long n, double *out);

/* ---- discrete adjoint (2D 14-moment, planar state, MXE_FP64) ------------ */

/* Sec. 3 scheme as a map U^{n+1} = Phi(U^n; imposed boundary states, tau_ref)
 * with the step sizes held fixed.  mxe_adjoint_record advances the current
 * state by n steps of the given sizes (as mxe_step_dt) and keeps U^n and,
 * for RK2, U* of every step on the device (the tape: 2 n copies of the
 * state; replaces the previous tape).  dts == NULL: n steps at the CFL
 * step size instead (as mxe_step), recorded as they are taken, so that a
 * forward run can keep its own tape; their sizes are read from the dt
 * history, which must cover them (mxe_set_dt_history), and the call
 * synchronises.  The context must hold a planar state (u_z, P_xz, P_yz,
 * q_z zero) and planar boundary states.
 * Errors: MXE_ESTATE (not an FP64 2D 14-moment planar context, no state,
 * dt history too short), MXE_EINVAL (n < 1, dt <= 0), MXE_EUNREALIZABLE /
 * MXE_ENONFINITE (CFL recording: as mxe_step), MXE_ENOMEM / MXE_ECUDA. */
mxe_status mxe_adjoint_record(mxe_ctx *ctx, int n, const double *dts);

/* Reverse sweep over the tape (hand-written reverse mode of primitive
 * recovery, shared limiter + MUSCL, closure, wave speeds, HLL / Rusanov and
 * the BGK source; branches as taken by the primal).  ubar (dense
 * (14, ny, nx), host or device per on_device) holds on entry the adjoint of
 * the state after the last recorded step and receives the adjoint of the
 * state before the first.  Adds to gbar ([4][1 + MAX_SPANS][14] host
 * array: side, slot 0 = base Dirichlet state / 1 + n = span n, primitive
 * field) the adjoint of the imposed primitive states, and to *taubar the
 * adjoint of tau_ref (either may be NULL).  Synchronises.  MXE_ENONFINITE
 * if the adjoint state or these adjoints are not finite (the FP32
 * face-state reverse can leave its range); gbar and *taubar are then left
 * unchanged, so that the caller can sweep again from a kept copy of ubar
 * with the FP64 reverse. */
mxe_status mxe_adjoint_run(mxe_ctx *ctx, double *ubar, int on_device, double *gbar,
                           double *taubar);

/* Arithmetic of the face-state reverse in later mxe_adjoint_run /
 * mxe_adjoint_residual calls: MXE_FP64 (default: exact linearisation, the
 * face states recomputed and reversed in FP64) or MXE_MIXED (the face states
 * recomputed from the FP64 tape and reversed in FP32; cell terms, the
 * adjoint state and all accumulations stay FP64).  MXE_EINVAL otherwise. */
mxe_status mxe_set_adjoint_precision(mxe_ctx *ctx, int precision);

/* Linearisation of the shared limiter in the adjoint.  frozen = 0 (default):
 * the exact derivative of the branch the primal takes, the limiter's
 * sub-gradient included (what the oracle's tangent computes).  frozen = 1:
 * the limiter value phi is held constant in the derivative, a common choice
 * for adjoints of limited schemes: the shared most-stringent limiter is not
 * differentiable at the scale of finite differences where a field's
 * differences are small, and its derivative there scales as the inverse of
 * those differences (differences at round-off level count as flat and do
 * not select phi in either mode).  MXE_EINVAL for another value. */
mxe_status mxe_set_adjoint_limiter(mxe_ctx *ctx, int frozen);

/* Adjoint of the residual L(U) = -div F + C at the conserved state U
 * (dense (14, ny, nx)): out = (dL/dU)^T V, and adds (dL/dg)^T V to gbar
 * and (dL/dtau_ref)^T V to *taubar.  For checking the reverse sweep one
 * residual at a time; allocates a temporary per call; synchronises. */
mxe_status mxe_adjoint_residual(mxe_ctx *ctx, const double *U, const double *V, double *out,
                                int on_device, double *gbar, double *taubar);

/* ---- fixed-scratch 1D solve (allocates nothing) -------------------------- */

/* No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory -- a host program whose device memory is
 * wholly owned by its own pool allocator (an outside cudaMalloc fails under
 * the pool's cap or breaks its accounting), or a time-critical loop that
 * cannot pay for cudaMalloc/cudaFree, which synchronise the device.
 *
 * Advances one 1D problem (cfg->ny == 1, cfg->nx <= 16384 cells, FP64) with
 * the same persistent kernel as mxe_step, from time t0 until t_end or
 * max_steps steps.  U is a device array of nf*nx doubles (conserved SoA,
 * field-major), read and overwritten in place; the caller owns it.  BCs are
 * transmissive or periodic (bc_lo, bc_hi); relaxation as in
 * mxe_set_relaxation.  Every other buffer (stage buffer, descriptor, clock)
 * is a fixed file-scope device array of the library: 1.75 MiB plus a few
 * hundred bytes, held on every GPU that loads the library until the process
 * exits.  No cudaMalloc, cudaFree or other allocating routine is called.
 *
 *  - The first call on a device looks up the arrays' device addresses
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the arrays, which keep the last call's contents; the
 *    clock is re-initialised by every call.  Calls that overlap on the GPU
 *    (other streams, other host threads) race on the shared arrays and must
 *    be serialised by the caller.
 *  - t_out / steps_out (host, may be NULL) receive the final time and the
 *    steps taken; passing either synchronises `stream` (a cudaStream_t, NULL
 *    for the default stream).  A non-finite state (MXE_ENONFINITE) is
 *    detected from the clock read back for them, so it is reported only
 *    when t_out or steps_out is given; with both NULL the call returns
 *    MXE_OK once the work is queued.
 *  - U must hold nf*nx doubles on the current device; the library cannot
 *    check a raw pointer's extent (the Python binding checks it).
 * Returns MXE_EINVAL for nx > 16384 or any other invalid argument, before
 * any device work. */
mxe_status mxe_tube_run_noalloc(const mxe_config *cfg, int bc_lo, int bc_hi, int tau_model,
                                double tau_ref, double rho_ref, double T_ref, double *U,
                                double t0, double t_end, int max_steps, double *t_out,
                                int *steps_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
