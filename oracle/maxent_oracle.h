/*
 * maxent_oracle.h -- plain FP64 CPU oracle for the 5- and 14-moment
 * maximum-entropy systems with interpolative closure (Boccelli, Kaufmann,
 * Magin, McDonald, "Numerical simulation of rarefied supersonic flows using a
 * fourth-order maximum-entropy moment method with interpolative closure",
 * JCP 2024, arXiv 2401.15233).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Conventions
 *   5-moment primitive vector  (rho, u, P, q, r)                      Sec. 2.3
 *   14-moment primitive vector (rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy,
 *                               Pyz, Pzz, qx, qy, qz, R)              Sec. 2.4
 *   q is the full third central moment (q_i = Q_ijj), i.e. twice the
 *   fluid-dynamic heat flux (Sec. 2.1).
 *   Conserved vectors are the balance-law densities of Eq. (5mom-sys-eqs)
 *   and the 14-moment system of Sec. 2.4.
 *
 * Parity status per function is listed in the oracle's tests; the exact
 * 14x14 eigenvalues are not computed here (parity unpinned for physical
 * accuracy of the wave-speed fit, which the paper only claims to ~20%).
 */
#ifndef MAXENT_ORACLE_H
#define MAXENT_ORACLE_H

/* Type of the physical quantities held by the configuration (imposed
 * boundary states, relaxation parameters): double, except in the tangent
 * build, which substitutes a dual-number type. */
#ifndef OR_REAL
#define OR_REAL double
#endif
typedef OR_REAL or_real;

#ifndef OR_TANGENT_BUILD
#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- 5-moment (1D1V) point functions ---------------- */
void   or5_prim2cons(const double *Q, double *U);
void   or5_cons2prim(const double *U, double *Q);
double or5_sigma(const double *Q);                         /* raw, unclamped */
double or5_closure(const double *Q, double sigma_lim);     /* s, dimensional */
void   or5_flux_given_s(const double *Q, double s, double *F);
void   or5_flux(const double *Q, double sigma_lim, double *F);
double or5_lambda_star_max(double qs, double sig);         /* Baradaran fit */
void   or5_wavespeeds(const double *Q, double sigma_lim, double k,
                      double *lmin, double *lmax);
void   or5_source(const double *Q, double tau, double *C);

/* ---------------- 14-moment (3D3V) point functions ---------------- */
void   or14_prim2cons(const double *Q, double *U);
void   or14_cons2prim(const double *U, double *Q);
double or14_sigma(const double *Q);                        /* raw, unclamped */
/* closing moments, dimensional: Qt[27] = Q_ijk (i*9+j*3+k),
   Rt[9] = R_ijkk (i*3+j), S[3] = S_ijjkk */
void   or14_closure(const double *Q, double sigma_lim,
                    double *Qt, double *Rt, double *S);
void   or14_flux_given_closure(const double *Q, const double *Qt,
                               const double *Rt, const double *S, int dir,
                               double *F);
void   or14_flux(const double *Q, double sigma_lim, int dir, double *F);
double or14_lambda_star_max(double Pdd, double qd, double qperp, double sig);
void   or14_wavespeeds(const double *Q, int dir, double sigma_lim, double k,
                       double *lmin, double *lmax);
void   or14_source(const double *Q, double tau, double *C);

/* bulk conversions of n cells (AoS) */
void   or_prim2cons_n(int nf, long n, const double *Q, double *U);
void   or_cons2prim_n(int nf, long n, const double *U, double *Q);

#ifdef __cplusplus
}
#endif
#endif /* OR_TANGENT_BUILD */

/* ---------------- finite-volume scheme ---------------- */
enum { OR_BC_TRANSMISSIVE = 0, OR_BC_PERIODIC = 1, OR_BC_DIRICHLET = 2 };
enum { OR_FLUX_HLL = 0, OR_FLUX_RUSANOV = 1 };
enum { OR_LIM_MINMOD = 0, OR_LIM_VANALBADA = 1 };
enum { OR_TAU_NONE = 0, OR_TAU_CONST = 1, OR_TAU_HARDSPHERE = 2 };
enum { OR_FE = 0, OR_RK2 = 1 };
enum { OR_SRC_EXPLICIT = 0, OR_SRC_POINT_IMPLICIT = 1 };
#define OR_MAX_SPANS 4

typedef struct {
    int    base_type;                 /* OR_BC_* for the whole side        */
    or_real base_state[14];           /* primitive state if DIRICHLET      */
    int    nspans;                    /* Dirichlet spans overriding base   */
    double span_lo[OR_MAX_SPANS], span_hi[OR_MAX_SPANS];
    or_real span_state[OR_MAX_SPANS][14];
} or_side;

typedef struct {
    int    system;        /* 5 or 14                                       */
    int    nx, ny;        /* ny == 1 -> one space dimension (x)            */
    double x0, x1, y0, y1;
    int    order;         /* 1 or 2 (MUSCL)                                */
    int    integrator;    /* OR_FE or OR_RK2                               */
    int    flux;          /* OR_FLUX_*                                     */
    int    limiter;       /* OR_LIM_*                                      */
    double cfl, sigma_lim, k_ws;
    int    tau_model;     /* OR_TAU_*                                      */
    or_real tau_ref, rho_ref, T_ref;
    or_side side[4];      /* 0 xlo, 1 xhi, 2 ylo, 3 yhi                    */
    int    source_scheme; /* OR_SRC_*: BGK source explicit in the stage or
                             point-implicit after it                       */
    int    frozen_limiter;/* derivative builds only: the shared limiter phi
                             is held constant in the derivative (the primal
                             is unchanged)                                 */
} or_cfg;

/* A block is a rectangle of cells [i0, i0+w) x [j0, j0+h) of the global
 * grid, stored cell-major (AoS, nf values per cell) with a margin of M=4
 * cells on every side that is not a space dimension's trivial axis
 * (M = 0 in y when ny == 1).  Sides where the block touches the domain
 * boundary are filled from the boundary conditions; the other sides must
 * carry real neighbour data in all 4 margin layers. */
#define OR_MARGIN 4

#ifndef OR_TANGENT_BUILD
#ifdef __cplusplus
extern "C" {
#endif

/* One time step of size dt on a block.  Ub is the block with margins
 * (size (w+2M)*(h+2My)*nf); Uout receives the w*h interior cells.
 * Returns 0 on success. */
int or_block_step(const or_cfg *c, int i0, int j0, int w, int h,
                  const double *Ub, double dt, double *Uout);

/* Residual L(U) = -div F + C on the interior of a block whose BC sides are
 * filled here; margins as in or_block_step. Lout is w*h*nf.  With the
 * point-implicit source the residual is the explicit part -div F. */
int or_block_residual(const or_cfg *c, int i0, int j0, int w, int h,
                      const double *Ub, double *Lout);

/* Whole-grid helpers: U is the interior nx*ny*nf (AoS, row-major). */
double or_max_rate(const or_cfg *c, const double *U);   /* CFL denominator */
double or_dt(const or_cfg *c, const double *U, double t, double t_end);
int    or_step(const or_cfg *c, double *U, double dt);  /* in place */
/* March until t_end or max_steps; returns steps taken, updates *t.
 * dt_hist (may be NULL) receives each dt. */
int    or_run(const or_cfg *c, double *U, double *t, double t_end,
              int max_steps, double *dt_hist);

/* tau at a primitive state (relaxation model of the Sod and jet cases). */
double or_tau(const or_cfg *c, const double *Q);

#ifdef __cplusplus
}
#endif
#endif /* OR_TANGENT_BUILD */
#endif
