/*
 * maxent_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Slow, literal implementation of the maximum-entropy moment method of
 * Boccelli et al. (JCP 2024, arXiv 2401.15233):
 *   - conserved <-> primitive moments      Sec. 2.3 (5-moment), Sec. 2.4 (14)
 *   - parabolic mapping sigma               Eq. (sigma-mapping-5mom/14mom)
 *   - interpolative closure                 Eq. (closure-1D1V-s-approx),
 *                                           Eqs. (closure-14mom-Qijk/Rijkk/
 *                                           Sijjkk) with B, K, W as printed
 *   - sigma limiting                        Appendix A
 *   - approximate wave speeds               Eq. (ws-max-baradaran-orig),
 *                                           Eq. (14mom-approx-ws-equations)
 *   - BGK sources                           Sec. 2.3, Sec. 2.4
 *   - cell-centred FV, MUSCL on primitives with one shared limiter,
 *     HLL / Rusanov face fluxes, forward Euler / midpoint RK2     Sec. 3
 *
 * The closure is evaluated in dimensionless form and re-dimensionalised
 * afterwards (Sec. 3.3).  The rank-4 tensor K and the matrix W are formed
 * explicitly, exactly as printed.  Readings of the paper where it is silent
 * or ambiguous (limiter formula, sigma > 1, stable root for sigma, tau model,
 * CFL in 2D, clamped wave-speed discriminant) are listed in the repository's
 * design notes; each is marked "reading" below.
 *
 * No blocking, fusion or reordering beyond the method's own steps.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use this file.
 */
#include "maxent_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Timing build (-fopenmp): the loops over rows, columns and cells of the
 * scheme run on all host cores.  Every cell's arithmetic and the order of
 * the contributions to it are those of the serial build, so both builds
 * give bitwise equal results; without -fopenmp the macros are empty. */
#if defined(_OPENMP) && !defined(__cplusplus)
#include <omp.h>
#define OR_PRAGMA(x) _Pragma(#x)
#define OR_PARALLEL_FOR OR_PRAGMA(omp parallel for schedule(static))
#define OR_PARALLEL_FOR_MAX(v) OR_PRAGMA(omp parallel for schedule(static) reduction(max : v))
int or_threads(void) { return omp_get_max_threads(); }
#else
#define OR_PARALLEL_FOR
#define OR_PARALLEL_FOR_MAX(v)
#ifndef __cplusplus
int or_threads(void) { return 1; }
#endif
#endif

/* Arithmetic type of every moment and derived quantity: double.  The
 * oracle's forward-mode tangent (tangent.cpp) compiles this same file with
 * a dual-number type in its place; nothing else changes. */
typedef or_real real;

/* ======================================================================= */
/* small 3x3 helpers (plain loops)                                          */
/* ======================================================================= */

static void mat_from_prim(const real *Q, real P[3][3]) {
    P[0][0] = Q[4]; P[0][1] = Q[5]; P[0][2] = Q[6];
    P[1][0] = Q[5]; P[1][1] = Q[7]; P[1][2] = Q[8];
    P[2][0] = Q[6]; P[2][1] = Q[8]; P[2][2] = Q[9];
}

static void matmul3(real A[3][3], real B[3][3], real C[3][3]) {
    real T[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int l = 0; l < 3; ++l) s += A[i][l] * B[l][j];
            T[i][j] = s;
        }
    memcpy(C, T, sizeof(T));
}

static real trace3(real A[3][3]) { return A[0][0] + A[1][1] + A[2][2]; }

/* inverse by the adjugate; returns the determinant */
static real inv3(real A[3][3], real Ai[3][3]) {
    real c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    real c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    real c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    real det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    Ai[0][0] = c00 / det;
    Ai[1][0] = c01 / det;
    Ai[2][0] = c02 / det;
    Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    return det;
}

/* Stable evaluation of sigma = [A + sqrt(A^2 + X)] / (4 T).
 * Reading: for A < 0 the algebraically identical rationalised root
 * X / (4 T (sqrt(A^2+X) - A)) is used to avoid cancellation. */
static real sigma_root(real A, real X, real T) {
    real rt = sqrt(A * A + X);
    if (A >= 0.0) return (A + rt) / (4.0 * T);
    return X / (4.0 * T * (rt - A));
}

/* Reading (sigma > 1, Appendix A gives only the lower bound):
 * sigma_bar = min(max(sigma, sigma_lim), 1). */
static real sigma_clamp(real s, real sigma_lim) {
    if (s < sigma_lim) s = sigma_lim;
    if (s > 1.0) s = 1.0;
    return s;
}

/* ======================================================================= */
/* 5-moment system, Sec. 2.3                                                */
/* ======================================================================= */

/* Conserved densities of Eq. (5mom-sys-eqs). */
void or5_prim2cons(const real *Q, real *U) {
    real rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * u * u + P;
    U[3] = rho * u * u * u + 3.0 * u * P + q;
    U[4] = rho * u * u * u * u + 6.0 * u * u * P + 4.0 * u * q + r;
}

void or5_cons2prim(const real *U, real *Q) {
    real rho = U[0];
    real u = U[1] / rho;
    real P = U[2] - rho * u * u;
    real q = U[3] - rho * u * u * u - 3.0 * u * P;
    real r = U[4] - rho * u * u * u * u - 6.0 * u * u * P - 4.0 * u * q;
    Q[0] = rho; Q[1] = u; Q[2] = P; Q[3] = q; Q[4] = r;
}

/* Eq. (sigma-mapping-5mom) in the dimensionless variables of
 * Eq. (dimensionless-variables) with the 1D1V pressure P. */
real or5_sigma(const real *Q) {
    real rho = Q[0], P = Q[2], q = Q[3], r = Q[4];
    real th = P / rho;
    real qs = q / (rho * pow(th, 1.5));
    real rs = r / (rho * th * th);
    real A = 3.0 - rs;
    real X = 8.0 * qs * qs;
    return sigma_root(A, X, 1.0);
}

/* Eq. (closure-1D1V-s-approx): the printed right-hand side is the
 * dimensionless s*; reading: s = s* rho (P/rho)^(5/2). */
real or5_closure(const real *Q, real sigma_lim) {
    real rho = Q[0], P = Q[2], q = Q[3];
    real th = P / rho;
    real qs = q / (rho * pow(th, 1.5));
    real sb = sigma_clamp(or5_sigma(Q), sigma_lim);
    real ss = qs * qs * qs / (sb * sb) + (10.0 - 8.0 * sqrt(sb)) * qs;
    return ss * rho * pow(th, 2.5);
}

/* x-fluxes of Eq. (5mom-sys-eqs) for a given closing moment s. */
void or5_flux_given_s(const real *Q, real s, real *F) {
    real rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    F[0] = rho * u;
    F[1] = rho * u * u + P;
    F[2] = rho * u * u * u + 3.0 * u * P + q;
    F[3] = rho * u * u * u * u + 6.0 * u * u * P + 4.0 * u * q + r;
    F[4] = rho * u * u * u * u * u + 10.0 * u * u * u * P + 10.0 * u * u * q
         + 5.0 * u * r + s;
}

void or5_flux(const real *Q, real sigma_lim, real *F) {
    or5_flux_given_s(Q, or5_closure(Q, sigma_lim), F);
}

/* Hyperbolic bracket  zeta + sqrt(zeta^2 + D0)  with D0 = rest of the
 * discriminant.  Reading: a negative discriminant is clamped to zero; for
 * zeta < 0 the rationalised form D0/(sqrt(.) - zeta) is used. */
static real hyp_bracket(real zeta, real D0) {
    real D = zeta * zeta + D0;
    if (D <= 0.0) return zeta;
    real rt = sqrt(D);
    if (zeta >= 0.0) return zeta + rt;
    return D0 / (rt - zeta);
}

/* Baradaran's 5-moment fit, Eq. (ws-max-baradaran-orig), at a clamped
 * sigma.  Returns the dimensionless maximum wave speed. */
real or5_lambda_star_max(real qs, real sig) {
    real E = 0.8 * sqrt(3.0 - 3.0 * sig);
    real C = sqrt(3.0 - 3.0 * sig);
    real B = 5.0 - 4.0 * sqrt(sig) + sqrt(10.0 - 16.0 * sqrt(sig) + 6.0 * sig);
    real Y = B + E * E - 2.0 * E * sqrt(B);
    real D0 = -0.8 * qs * sig * C + 4.0 * sig * sig * Y;
    return hyp_bracket(qs, D0) / (2.0 * sig) + E;
}

/* lambda_min* = -lambda_max*(-q*), inflation by k, re-dimensionalisation
 * lambda = u + lambda* sqrt(P/rho)  (Sec. 5 and Appendix B). */
void or5_wavespeeds(const real *Q, real sigma_lim, real k,
                    real *lmin, real *lmax) {
    real rho = Q[0], u = Q[1], P = Q[2], q = Q[3];
    real th = P / rho;
    real qs = q / (rho * pow(th, 1.5));
    real sb = sigma_clamp(or5_sigma(Q), sigma_lim);
    real lp = k * or5_lambda_star_max(qs, sb);
    real lm = -k * or5_lambda_star_max(-qs, sb);
    *lmax = u + lp * sqrt(th);
    *lmin = u + lm * sqrt(th);
}

/* BGK sources of Eq. (5mom-sys-eqs). */
void or5_source(const real *Q, real tau, real *C) {
    real rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    C[0] = 0.0;
    C[1] = 0.0;
    C[2] = 0.0;
    C[3] = -q / tau;
    C[4] = -(4.0 * u * q + r - 3.0 * P * P / rho) / tau;
}

/* ======================================================================= */
/* 14-moment system, Sec. 2.4                                               */
/* ======================================================================= */

/* Conserved densities: rho, rho u_i, rho u_i u_j + P_ij,
 * rho u_i u_j u_j + u_i P_jj + 2 u_j P_ij + Q_ijj,
 * rho u_i u_i u_j u_j + 2 u_i u_i P_jj + 4 u_i u_j P_ij + 4 u_i Q_ijj + R_iijj */
void or14_prim2cons(const real *Q, real *U) {
    real rho = Q[0], u[3] = {Q[1], Q[2], Q[3]};
    real P[3][3]; mat_from_prim(Q, P);
    real q[3] = {Q[10], Q[11], Q[12]}, R = Q[13];
    real u2 = 0.0, trP = trace3(P), uPu = 0.0, uq = 0.0;
    for (int i = 0; i < 3; ++i) { u2 += u[i] * u[i]; uq += u[i] * q[i]; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) uPu += u[i] * u[j] * P[i][j];
    U[0] = rho;
    for (int i = 0; i < 3; ++i) U[1 + i] = rho * u[i];
    int idx = 4;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) U[idx++] = rho * u[i] * u[j] + P[i][j];
    for (int i = 0; i < 3; ++i) {
        real uP = 0.0;
        for (int j = 0; j < 3; ++j) uP += u[j] * P[i][j];
        U[10 + i] = rho * u[i] * u2 + u[i] * trP + 2.0 * uP + q[i];
    }
    U[13] = rho * u2 * u2 + 2.0 * u2 * trP + 4.0 * uPu + 4.0 * uq + R;
}

void or14_cons2prim(const real *U, real *Q) {
    real rho = U[0];
    real u[3];
    for (int i = 0; i < 3; ++i) u[i] = U[1 + i] / rho;
    real P[3][3];
    int idx = 4;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            P[i][j] = U[idx++] - rho * u[i] * u[j];
            P[j][i] = P[i][j];
        }
    real u2 = 0.0, trP = trace3(P), uPu = 0.0;
    for (int i = 0; i < 3; ++i) u2 += u[i] * u[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) uPu += u[i] * u[j] * P[i][j];
    real q[3];
    for (int i = 0; i < 3; ++i) {
        real uP = 0.0;
        for (int j = 0; j < 3; ++j) uP += u[j] * P[i][j];
        q[i] = U[10 + i] - rho * u[i] * u2 - u[i] * trP - 2.0 * uP;
    }
    real uq = u[0] * q[0] + u[1] * q[1] + u[2] * q[2];
    real R = U[13] - rho * u2 * u2 - 2.0 * u2 * trP - 4.0 * uPu - 4.0 * uq;
    Q[0] = rho;
    for (int i = 0; i < 3; ++i) Q[1 + i] = u[i];
    Q[4] = P[0][0]; Q[5] = P[0][1]; Q[6] = P[0][2];
    Q[7] = P[1][1]; Q[8] = P[1][2]; Q[9] = P[2][2];
    for (int i = 0; i < 3; ++i) Q[10 + i] = q[i];
    Q[13] = R;
}

/* Dimensionless state of Eq. (dimensionless-variables), with the
 * hydrostatic pressure p = tr(P)/3 as the scale (Sec. 3.3). */
typedef struct {
    real rho, p, th;        /* density, hydrostatic pressure, p/rho */
    real P[3][3];           /* P*  */
    real q[3];              /* q*  */
    real R;                 /* R*  */
} dimless14;

static void to_dimless14(const real *Q, dimless14 *d) {
    real P[3][3]; mat_from_prim(Q, P);
    d->rho = Q[0];
    d->p = trace3(P) / 3.0;
    d->th = d->p / d->rho;
    real sq = d->rho * pow(d->th, 1.5);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) d->P[i][j] = P[i][j] / d->p;
    for (int i = 0; i < 3; ++i) d->q[i] = Q[10 + i] / sq;
    d->R = Q[13] / (d->rho * d->th * d->th);
}

/* Eq. (sigma-mapping-14mom) with rho* = 1. */
static real sigma14_dimless(const dimless14 *d) {
    real P2[3][3], Pi[3][3];
    matmul3((real (*)[3])d->P, (real (*)[3])d->P, P2);
    inv3((real (*)[3])d->P, Pi);
    real T = trace3(P2);                 /* P_ij P_ji */
    real trP = trace3((real (*)[3])d->P);
    real qPq = 0.0;                      /* Q_kii (P^-1)_kl Q_ljj */
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) qPq += d->q[k] * Pi[k][l] * d->q[l];
    real A = 2.0 * T + trP * trP - d->R;
    real X = 8.0 * T * qPq;
    return sigma_root(A, X, T);
}

real or14_sigma(const real *Q) {
    dimless14 d;
    to_dimless14(Q, &d);
    return sigma14_dimless(&d);
}

/* Eqs. (closure-14mom-Qijk-approx), (closure-14mom-Rijkk-approx),
 * (closure-14mom-Sijjkk-approx) with B, K and W as printed, evaluated with
 * rho* = 1 and the clamped sigma_bar (Appendix A), then re-dimensionalised:
 * Q = Q* rho th^(3/2), R = R* rho th^2, S = S* rho th^(5/2). */
void or14_closure(const real *Q, real sigma_lim,
                  real *Qt, real *Rt, real *S) {
    dimless14 d;
    to_dimless14(Q, &d);
    real sb = sigma_clamp(sigma14_dimless(&d), sigma_lim);
    real (*P)[3] = d.P;
    real P2[3][3], P3[3][3], P4[3][3], Pi[3][3];
    matmul3(P, P, P2);
    matmul3(P2, P, P3);
    matmul3(P3, P, P4);
    inv3(P, Pi);
    real trP = trace3(P), trP2 = trace3(P2), trP3 = trace3(P3);

    /* B_lm = 2 P_lm (P^2)_aa + 4 (P^3)_lm */
    real B[3][3], Bi[3][3];
    for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) B[l][m] = 2.0 * P[l][m] * trP2 + 4.0 * P3[l][m];
    inv3(B, Bi);

    /* K_ijkm = [2 P_il (P^2)_jk + 2 P_kl (P^2)_ij + 2 P_jl (P^2)_ik] B^-1_lm */
    real K[3][3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int m = 0; m < 3; ++m) {
                    real s = 0.0;
                    for (int l = 0; l < 3; ++l)
                        s += (2.0 * P[i][l] * P2[j][k] + 2.0 * P[k][l] * P2[i][j]
                              + 2.0 * P[j][l] * P2[i][k]) * Bi[l][m];
                    K[i][j][k][m] = s;
                }

    /* Q_ijk = K_ijkm Q_mnn  (Q_mnn = q_m) */
    real Qs[3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                real s = 0.0;
                for (int m = 0; m < 3; ++m) s += K[i][j][k][m] * d.q[m];
                Qs[i][j][k] = s;
            }

    /* R_ijkk = (1/sigma) Q_ijl (P^-1)_lm Q_mkk + [2(1-sigma) P_ik P_kj + P_ij P_kk]/rho */
    real Rs[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real s = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int m = 0; m < 3; ++m) s += Qs[i][j][l] * Pi[l][m] * d.q[m];
            Rs[i][j] = s / sb + (2.0 * (1.0 - sb) * P2[i][j] + P[i][j] * trP);
        }

    /* W_im = (1/rho)[2 P_il (P_aa)^3 + 12 P_il (P^3)_aa + 14 (P^2)_aa (P^2)_il
     *        + 20 P_aa (P^3)_il + 20 (P^4)_il - 2 (P^2)_aa P_bb P_il
     *        - 6 (P_aa)^2 (P^2)_il] B^-1_lm */
    real Wb[3][3], W[3][3];
    for (int i = 0; i < 3; ++i)
        for (int l = 0; l < 3; ++l)
            Wb[i][l] = 2.0 * P[i][l] * trP * trP * trP + 12.0 * P[i][l] * trP3
                     + 14.0 * trP2 * P2[i][l] + 20.0 * trP * P3[i][l]
                     + 20.0 * P4[i][l] - 2.0 * trP2 * trP * P[i][l]
                     - 6.0 * trP * trP * P2[i][l];
    matmul3(Wb, Bi, W);

    /* S_ijjkk = (1/sigma^2) P^-1_kn P^-1_lm Q_npp Q_mjj Q_ikl
     *         + 2 sigma^(1/2) P_jj Q_ikk / rho + (1 - sigma^(1/2)) W_im Q_mnn */
    real sqs = sqrt(sb);
    for (int i = 0; i < 3; ++i) {
        real s1 = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l)
                for (int n = 0; n < 3; ++n)
                    for (int m = 0; m < 3; ++m)
                        s1 += Pi[k][n] * Pi[l][m] * d.q[n] * d.q[m] * Qs[i][k][l];
        real s3 = 0.0;
        for (int m = 0; m < 3; ++m) s3 += W[i][m] * d.q[m];
        S[i] = s1 / (sb * sb) + 2.0 * sqs * trP * d.q[i] + (1.0 - sqs) * s3;
    }

    real sc3 = d.rho * pow(d.th, 1.5);
    real sc4 = d.rho * d.th * d.th;
    real sc5 = d.rho * pow(d.th, 2.5);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) Qt[i * 9 + j * 3 + k] = Qs[i][j][k] * sc3;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rt[i * 3 + j] = Rs[i][j] * sc4;
    for (int i = 0; i < 3; ++i) S[i] *= sc5;
}

/* x_k-fluxes of the 14-moment system (Sec. 2.4), k = dir, for given
 * closing moments; Q_kjj is the contraction of the supplied tensor. */
void or14_flux_given_closure(const real *Q, const real *Qt,
                             const real *Rt, const real *S, int dir,
                             real *F) {
    int k = dir;
    real rho = Q[0], u[3] = {Q[1], Q[2], Q[3]};
    real P[3][3]; mat_from_prim(Q, P);
    real R = Q[13];
    real u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    real trP = trace3(P);
#define QT(a, b, c) Qt[(a) * 9 + (b) * 3 + (c)]
#define RT(a, b) Rt[(a) * 3 + (b)]
    real Qc[3];                          /* Q_ijj */
    for (int i = 0; i < 3; ++i) Qc[i] = QT(i, 0, 0) + QT(i, 1, 1) + QT(i, 2, 2);

    F[0] = rho * u[k];
    for (int i = 0; i < 3; ++i) F[1 + i] = rho * u[i] * u[k] + P[i][k];
    int idx = 4;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j)
            F[idx++] = rho * u[i] * u[j] * u[k] + u[i] * P[j][k] + u[j] * P[i][k]
                     + u[k] * P[i][j] + QT(i, j, k);
    for (int i = 0; i < 3; ++i) {
        real s = rho * u[i] * u[k] * u2 + u[i] * u[k] * trP + u2 * P[i][k]
                 + u[i] * Qc[k] + u[k] * Qc[i] + RT(i, k);
        for (int j = 0; j < 3; ++j)
            s += 2.0 * u[i] * u[j] * P[j][k] + 2.0 * u[j] * u[k] * P[i][j]
               + 2.0 * u[j] * QT(i, j, k);
        F[10 + i] = s;
    }
    real s = rho * u[k] * u2 * u2 + 2.0 * u[k] * u2 * trP + 2.0 * u2 * Qc[k]
             + u[k] * R + S[k];
    for (int j = 0; j < 3; ++j) s += 4.0 * u2 * u[j] * P[j][k];
    for (int i = 0; i < 3; ++i) {
        s += 4.0 * u[i] * u[k] * Qc[i] + 4.0 * u[i] * RT(i, k);
        for (int j = 0; j < 3; ++j)
            s += 4.0 * u[i] * u[j] * u[k] * P[i][j] + 4.0 * u[i] * u[j] * QT(i, j, k);
    }
    F[13] = s;
#undef QT
#undef RT
}

void or14_flux(const real *Q, real sigma_lim, int dir, real *F) {
    real Qt[27], Rt[9], S[3];
    or14_closure(Q, sigma_lim, Qt, Rt, S);
    or14_flux_given_closure(Q, Qt, Rt, S, dir, F);
}

/* Eq. (14mom-approx-ws-equations) at a clamped sigma: dimensionless maximum
 * wave speed along direction d from (P*_dd, q*_d, transverse |q*|, sigma). */
real or14_lambda_star_max(real Pdd, real qd, real qperp, real sig) {
    real zeta = qd + sqrt(qperp * qperp) * (0.6 * Pdd * Pdd - 0.38 * Pdd + 0.35);
    real a = 1.4 * pow(Pdd, 1.1) * exp(-Pdd * Pdd);
    real b = 0.9 * Pdd * exp(-0.5 * pow(Pdd, 1.4));
    real E = 0.8 * sqrt((3.0 - 3.0 * sig) * Pdd);
    real C = sqrt((3.0 - 3.0 * sig) * Pdd);
    real B = 5.0 - 4.0 * sqrt(sig) + sqrt(10.0 - 16.0 * sqrt(sig) + 6.0 * sig);
    real Y = B + E * E - 2.0 * E * sqrt(B);
    real D0 = -0.8 * zeta * sig * C + 4.0 * sig * sig * Y + qperp * qperp / 10.0;
    return (a * sig + b) / (2.0 * sig) * hyp_bracket(zeta, D0) + E;
}

/* lambda_min* = -lambda_max*(-q_d*) with the other moments unchanged,
 * inflation k, lambda = u_d + lambda* sqrt(p/rho); other directions by
 * swapping indices (Sec. 5.1). */
void or14_wavespeeds(const real *Q, int dir, real sigma_lim, real k,
                     real *lmin, real *lmax) {
    dimless14 d;
    to_dimless14(Q, &d);
    real sb = sigma_clamp(sigma14_dimless(&d), sigma_lim);
    int e = (dir + 1) % 3, f = (dir + 2) % 3;
    real Pdd = d.P[dir][dir];
    real qd = d.q[dir];
    real qperp = sqrt(d.q[e] * d.q[e] + d.q[f] * d.q[f]);
    real lp = k * or14_lambda_star_max(Pdd, qd, qperp, sb);
    real lm = -k * or14_lambda_star_max(Pdd, -qd, qperp, sb);
    real c = sqrt(d.th);
    *lmax = Q[1 + dir] + lp * c;
    *lmin = Q[1 + dir] + lm * c;
}

/* BGK sources, Sec. 2.4: C_1 = C_i = 0, C_ij = -(P_ij - P delta_ij)/tau,
 * C_ijj = -(2 u_j P_ij + Q_ijj - 2 u_i P)/tau,
 * C_iijj = -[(4 u_i u_j P_ij + 4 u_i Q_ijj + R_iijj) - (4|u|^2 P + 15 P^2/rho)]/tau */
void or14_source(const real *Q, real tau, real *C) {
    real rho = Q[0], u[3] = {Q[1], Q[2], Q[3]};
    real P[3][3]; mat_from_prim(Q, P);
    real q[3] = {Q[10], Q[11], Q[12]}, R = Q[13];
    real p = trace3(P) / 3.0;
    for (int i = 0; i < 4; ++i) C[i] = 0.0;
    int idx = 4;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j)
            C[idx++] = -(P[i][j] - (i == j ? p : 0.0)) / tau;
    for (int i = 0; i < 3; ++i) {
        real uP = 0.0;
        for (int j = 0; j < 3; ++j) uP += u[j] * P[i][j];
        C[10 + i] = -(2.0 * uP + q[i] - 2.0 * u[i] * p) / tau;
    }
    real uPu = 0.0, uq = 0.0, u2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        uq += u[i] * q[i];
        u2 += u[i] * u[i];
        for (int j = 0; j < 3; ++j) uPu += u[i] * u[j] * P[i][j];
    }
    C[13] = -((4.0 * uPu + 4.0 * uq + R) - (4.0 * u2 * p + 15.0 * p * p / rho)) / tau;
}

/* Conversions of n cells (AoS, nf values per cell): plain loops over the
 * point functions above. */
void or_prim2cons_n(int nf, long n, const real *Q, real *U) {
    for (long c = 0; c < n; ++c) {
        if (nf == 5) or5_prim2cons(Q + c * 5, U + c * 5);
        else or14_prim2cons(Q + c * 14, U + c * 14);
    }
}

void or_cons2prim_n(int nf, long n, const real *U, real *Q) {
    for (long c = 0; c < n; ++c) {
        if (nf == 5) or5_cons2prim(U + c * 5, Q + c * 5);
        else or14_cons2prim(U + c * 14, Q + c * 14);
    }
}

/* ======================================================================= */
/* finite-volume scheme, Sec. 3                                             */
/* ======================================================================= */

static int nfields(const or_cfg *c) { return c->system == 5 ? 5 : 14; }

/* Reading (tau model): tau = tau_ref (rho_ref/rho) sqrt(T_ref/T), i.e.
 * tau = lambda / v_th with lambda proportional to 1/rho and
 * v_th = sqrt(8T/pi); T = P/rho (1D1V) or tr(P)/(3 rho) (3D3V). */
real or_tau(const or_cfg *c, const real *Q) {
    if (c->tau_model == OR_TAU_NONE) return INFINITY;
    if (c->tau_model == OR_TAU_CONST) return c->tau_ref;
    real T = (c->system == 5) ? Q[2] / Q[0] : (Q[4] + Q[7] + Q[9]) / (3.0 * Q[0]);
    return c->tau_ref * (c->rho_ref / Q[0]) * sqrt(c->T_ref / T);
}

static void prim2cons(const or_cfg *c, const real *Q, real *U) {
    if (c->system == 5) or5_prim2cons(Q, U); else or14_prim2cons(Q, U);
}
static void cons2prim(const or_cfg *c, const real *U, real *Q) {
    if (c->system == 5) or5_cons2prim(U, Q); else or14_cons2prim(U, Q);
}
static void pflux(const or_cfg *c, const real *Q, int dir, real *F) {
    if (c->system == 5) or5_flux(Q, c->sigma_lim, F);
    else or14_flux(Q, c->sigma_lim, dir, F);
}
static void wspeeds(const or_cfg *c, const real *Q, int dir, real *lmin,
                    real *lmax) {
    if (c->system == 5) or5_wavespeeds(Q, c->sigma_lim, c->k_ws, lmin, lmax);
    else or14_wavespeeds(Q, dir, c->sigma_lim, c->k_ws, lmin, lmax);
}
static void source(const or_cfg *c, const real *Q, real *C) {
    int nf = nfields(c);
    if (c->tau_model == OR_TAU_NONE) {
        for (int k = 0; k < nf; ++k) C[k] = 0.0;
        return;
    }
    real tau = or_tau(c, Q);
    if (c->system == 5) or5_source(Q, tau, C); else or14_source(Q, tau, C);
}

/* Primitive moments of the Maxwellian with the density, velocity and
 * pressure of Q: 5-moment (rho, u, P, 0, 3 P^2/rho); 14-moment
 * (rho, u, p delta_ij, 0, 15 p^2/rho), p = tr P / 3 (Sec. 2.3, 2.4: the
 * equilibrium moments the BGK source relaxes towards). */
static void maxwellian_prim(const or_cfg *c, const real *Q, real *QM) {
    if (c->system == 5) {
        QM[0] = Q[0]; QM[1] = Q[1]; QM[2] = Q[2]; QM[3] = 0.0;
        QM[4] = 3.0 * Q[2] * Q[2] / Q[0];
        return;
    }
    real p = (Q[4] + Q[7] + Q[9]) / 3.0;
    for (int k = 0; k < 14; ++k) QM[k] = 0.0;
    QM[0] = Q[0]; QM[1] = Q[1]; QM[2] = Q[2]; QM[3] = Q[3];
    QM[4] = p; QM[7] = p; QM[9] = p;
    QM[13] = 15.0 * p * p / Q[0];
}

/* Point-implicit BGK source over h (reading of the remark closing the
 * cost discussion of Sec. 4.3: below Kn ~ 1e-4 the source limits an
 * explicit step and a simple point-implicit treatment suffices).  After an
 * explicit stage V = U_base + h (-div F), solve dU/dt = -(U - U_M)/tau by
 * backward Euler over h.  The source leaves density, momentum and energy
 * unchanged, so U_M (the Maxwellian's conserved moments) and tau are V's,
 * and the implicit step is U = U_M + (V - U_M) / (1 + h/tau).  Density and
 * momentum are kept as they are (collision invariants). */
static void relax_cell(const or_cfg *c, real *U, real h) {
    if (c->tau_model == OR_TAU_NONE) return;
    int nf = nfields(c);
    real Q[14], QM[14], UM[14];
    cons2prim(c, U, Q);
    real tau = or_tau(c, Q);
    maxwellian_prim(c, Q, QM);
    prim2cons(c, QM, UM);
    real g = 1.0 / (1.0 + h / tau);
    int first = (c->system == 5) ? 2 : 4;
    for (int k = first; k < nf; ++k) U[k] = UM[k] + g * (U[k] - UM[k]);
}

/* HLL with Davis speeds S_L = min(lmin_L, lmin_R), S_R = max(lmax_L, lmax_R)
 * (reading: the paper names HLL, Sec. 3.1; the formula is the textbook one),
 * or Rusanov with s = max |lambda| over both states. */
static void face_flux(const or_cfg *c, const real *QL, const real *QR,
                      int dir, real *Fout) {
    int nf = nfields(c);
    real UL[14], UR[14], FL[14], FR[14];
    real lminL, lmaxL, lminR, lmaxR;
    prim2cons(c, QL, UL);
    prim2cons(c, QR, UR);
    pflux(c, QL, dir, FL);
    pflux(c, QR, dir, FR);
    wspeeds(c, QL, dir, &lminL, &lmaxL);
    wspeeds(c, QR, dir, &lminR, &lmaxR);
    if (c->flux == OR_FLUX_RUSANOV) {
        real s = fabs(lminL);
        if (fabs(lmaxL) > s) s = fabs(lmaxL);
        if (fabs(lminR) > s) s = fabs(lminR);
        if (fabs(lmaxR) > s) s = fabs(lmaxR);
        for (int k = 0; k < nf; ++k)
            Fout[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * s * (UR[k] - UL[k]);
        return;
    }
    real SL = lminL < lminR ? lminL : lminR;
    real SR = lmaxL > lmaxR ? lmaxL : lmaxR;
    if (SL >= 0.0) {
        for (int k = 0; k < nf; ++k) Fout[k] = FL[k];
    } else if (SR <= 0.0) {
        for (int k = 0; k < nf; ++k) Fout[k] = FR[k];
    } else {
        for (int k = 0; k < nf; ++k)
            Fout[k] = (SR * FL[k] - SL * FR[k] + SL * SR * (UR[k] - UL[k])) / (SR - SL);
    }
}

/* Flat-field test of the shared limiter (a reading: the paper states no
 * tolerance).  Field k of the stencil centred on Q is flat when
 * m = max(|dm|, |dp|) is within OR_FLAT_TOL times the field's natural scale
 * at Q, with theta = p / rho and p the mean pressure: rho (density),
 * sqrt(theta) (velocities), p (pressure tensor), p sqrt(theta) (heat
 * fluxes), p theta (fourth moment).  The comparisons are multiplied out
 * (rho, p > 0), with s = P for the 5-moment system and s = tr P = 3p for the
 * 14-moment one, so that no division or square root enters:
 *   m <= T rho;  m^2 rho <= T^2 p;  m <= T p;  m^2 rho <= T^2 p^3;
 *   m rho <= T p^2   (T = OR_FLAT_TOL, p written through s). */
#define OR_FLAT_TOL 1e-10
static int field_flat(const or_cfg *c, const real *Q, int k, real m) {
    real rho = Q[0];
    int cls;
    real s, cp, cv, ch, cr;
    if (c->system == 5) {
        s = Q[2];
        cp = OR_FLAT_TOL;
        cv = OR_FLAT_TOL * OR_FLAT_TOL;
        ch = OR_FLAT_TOL * OR_FLAT_TOL;
        cr = OR_FLAT_TOL;
        cls = k;
    } else {
        s = (Q[4] + Q[7]) + Q[9];
        cp = OR_FLAT_TOL / 3.0;
        cv = OR_FLAT_TOL * OR_FLAT_TOL / 3.0;
        ch = OR_FLAT_TOL * OR_FLAT_TOL / 27.0;
        cr = OR_FLAT_TOL / 9.0;
        cls = k == 0 ? 0 : k <= 3 ? 1 : k <= 9 ? 2 : k <= 12 ? 3 : 4;
    }
    switch (cls) {
    case 0: return m <= OR_FLAT_TOL * rho;
    case 1: return (m * m) * rho <= cv * s;
    case 2: return m <= cp * s;
    case 3: return (m * m) * rho <= ((ch * s) * s) * s;
    default: return m * rho <= (cr * s) * s;
    }
}

/* Shared most-stringent limiter (Sec. 3.2).  Reading, per primitive k with
 * dm = Q_i - Q_{i-1}, dp = Q_{i+1} - Q_i, c = (dm + dp)/2:
 *   phi_k = 1 if the field is flat across the stencil (both differences
 *           exactly zero, or field_flat: such differences are round-off of
 *           the conserved-to-primitive recovery -- a field that is uniform
 *           or zero in exact arithmetic must not limit the others, or the
 *           scheme drops to first order wherever round-off changes sign);
 *   phi_k = 0 if dm*dp <= 0;
 *   minmod(dm, dp)/c (minmod) or 2 dm dp/(dm^2 + dp^2) (van Albada) else;
 * phi = min_k phi_k and the slope of every field is phi * c_k. */
static real shared_phi(const or_cfg *c, const real *Qm, const real *Q0,
                         const real *Qp) {
    int nf = nfields(c);
    real phi = 1.0;
    for (int k = 0; k < nf; ++k) {
        real dm = Q0[k] - Qm[k], dp = Qp[k] - Q0[k];
        real m = fabs(dm) > fabs(dp) ? fabs(dm) : fabs(dp);
        real pk;
        if ((dm == 0.0 && dp == 0.0) || field_flat(c, Q0, k, m)) pk = 1.0;
        else if (dm * dp <= 0.0) pk = 0.0;
        else if (c->limiter == OR_LIM_VANALBADA) pk = 2.0 * dm * dp / (dm * dm + dp * dp);
        else {
            real cen = 0.5 * (dm + dp);
            real mm = fabs(dm) < fabs(dp) ? dm : dp;
            pk = mm / cen;
        }
        if (pk < phi) phi = pk;
    }
    return phi;
}

/* OR_VALUE(x): x with its derivative dropped (the identity in the plain
 * build; the derivative build defines it) */
#ifndef OR_VALUE
#define OR_VALUE(x) (x)
#endif

/* face state of cell Q0 on its side sgn (+1 right, -1 left) */
static void face_state(const or_cfg *c, const real *Qm, const real *Q0,
                       const real *Qp, real sgn, real *Qf) {
    int nf = nfields(c);
    if (c->order == 1) {
        for (int k = 0; k < nf; ++k) Qf[k] = Q0[k];
        return;
    }
    real phi = shared_phi(c, Qm, Q0, Qp);
    if (c->frozen_limiter) phi = OR_VALUE(phi);
    for (int k = 0; k < nf; ++k) {
        /* a field that is flat across the stencil keeps its cell value (its
         * slope phi * 0 vanishes; written out so that its derivative is the
         * zero slope as well, reading of Sec. 3.2 for the tangent) */
        if (Q0[k] - Qm[k] == 0.0 && Qp[k] - Q0[k] == 0.0) {
            Qf[k] = Q0[k];
            continue;
        }
        real cen = 0.5 * ((Q0[k] - Qm[k]) + (Qp[k] - Q0[k]));
        Qf[k] = Q0[k] + sgn * 0.5 * (phi * cen);
    }
}

/* ------------------------------------------------------------------ */
/* blocks                                                               */
/* ------------------------------------------------------------------ */

typedef struct {
    int i0, j0, w, h;     /* block interior in global cells */
    int mx, my;           /* margins                        */
    int W, H;             /* stored extent (w+2mx, h+2my)   */
    int nf;
    real *gp;           /* per-cell imposed primitive state of Dirichlet
                             ghosts (gp[cell*nf] is NaN where none)        */
} blk;

static real *cell(const blk *b, real *A, int i, int j) {
    return A + ((size_t)(j + b->my) * b->W + (size_t)(i + b->mx)) * b->nf;
}

static int side_is_boundary(const or_cfg *c, const blk *b, int s) {
    if (c->side[s].base_type == OR_BC_PERIODIC) return 0;   /* caller wraps */
    if (s == 0) return b->i0 == 0;
    if (s == 1) return b->i0 + b->w == c->nx;
    if (c->ny == 1) return 0;
    if (s == 2) return b->j0 == 0;
    return b->j0 + b->h == c->ny;
}

/* Ghost value for a cell of side s whose tangential centre coordinate is
 * xt, given the nearest interior cell value Uin (conserved).  Reading
 * (Sec. 6, inflow values imposed in the ghost cells; Sec. 3.2,
 * reconstruction of primitive variables): a Dirichlet ghost carries the
 * imposed primitive state itself, Gp; its conserved value Ug is stored too. */
static void ghost_value(const or_cfg *c, int s, real xt, const real *Uin,
                        real *Ug, real *Gp) {
    const or_side *sd = &c->side[s];
    int nf = nfields(c);
    for (int n = 0; n < sd->nspans; ++n)
        if (xt >= sd->span_lo[n] && xt <= sd->span_hi[n]) {
            prim2cons(c, sd->span_state[n], Ug);
            memcpy(Gp, sd->span_state[n], nf * sizeof(real));
            return;
        }
    if (sd->base_type == OR_BC_DIRICHLET) {
        prim2cons(c, sd->base_state, Ug);
        memcpy(Gp, sd->base_state, nf * sizeof(real));
        return;
    }
    for (int k = 0; k < nf; ++k) Ug[k] = Uin[k];          /* transmissive */
    Gp[0] = NAN;
}

/* Fill two ghost layers on every side of the block that is a domain
 * boundary (Sec. 6: inflow states imposed in ghost cells). */
static void fill_bc(const or_cfg *c, const blk *b, real *A) {
    real dx = (c->x1 - c->x0) / c->nx;
    real dy = (c->y1 - c->y0) / c->ny;
    for (int s = 0; s < 4; ++s) {
        if (!side_is_boundary(c, b, s)) continue;
        if (s < 2) {
            for (int j = -b->my; j < b->h + b->my; ++j) {
                real yt = c->y0 + ((real)(b->j0 + j) + 0.5) * dy;
                int iin = (s == 0) ? 0 : b->w - 1;
                for (int g = 1; g <= 2; ++g) {
                    int ig = (s == 0) ? -g : b->w - 1 + g;
                    ghost_value(c, s, yt, cell(b, A, iin, j), cell(b, A, ig, j),
                                cell(b, b->gp, ig, j));
                }
            }
        } else {
            for (int i = -b->mx; i < b->w + b->mx; ++i) {
                real xt = c->x0 + ((real)(b->i0 + i) + 0.5) * dx;
                int jin = (s == 2) ? 0 : b->h - 1;
                for (int g = 1; g <= 2; ++g) {
                    int jg = (s == 2) ? -g : b->h - 1 + g;
                    ghost_value(c, s, xt, cell(b, A, i, jin), cell(b, A, i, jg),
                                cell(b, b->gp, i, jg));
                }
            }
        }
    }
}

/* residual L = -sum_d (F_{d,+} - F_{d,-})/dx_d + C on cells [xa,xb) x [ya,yb)
 * (block-local), from the conserved block A (ghosts/margins valid). */
static void residual_region(const or_cfg *c, const blk *b, real *A,
                            int xa, int xb, int ya, int yb, real *L) {
    int nf = nfields(c);
    real dx = (c->x1 - c->x0) / c->nx;
    real dy = (c->y1 - c->y0) / c->ny;
    size_t ncell = (size_t)b->W * b->H;
    real *Qp = (real *)malloc(ncell * nf * sizeof(real));
    OR_PARALLEL_FOR
    for (size_t n = 0; n < ncell; ++n) {
        if (!isnan(b->gp[n * nf])) memcpy(Qp + n * nf, b->gp + n * nf, nf * sizeof(real));
        else cons2prim(c, A + n * nf, Qp + n * nf);
    }
    int rw = xb - xa;
    /* L[(j-ya)*rw + (i-xa)] */
    OR_PARALLEL_FOR
    for (int j = ya; j < yb; ++j)
        for (int i = xa; i < xb; ++i) {
            real *Lc = L + ((size_t)(j - ya) * rw + (i - xa)) * nf;
            real C[14];
            if (c->source_scheme == OR_SRC_POINT_IMPLICIT) {
                for (int k = 0; k < nf; ++k) C[k] = 0.0;
            } else {
                source(c, cell(b, Qp, i, j), C);
            }
            for (int k = 0; k < nf; ++k) Lc[k] = C[k];
        }
    int ndim = (c->ny == 1) ? 1 : 2;
    int rh = yb - ya;
    for (int d = 0; d < ndim; ++d) {
        real h = (d == 0) ? dx : dy;
        /* face s of a line lies between cells s-1 and s; a line of the
         * region has nfl faces (rw + 1 along x, rh + 1 along y), and there
         * are nl lines (rh rows, or rw columns).  All face fluxes first,
         * then the flux differences, line by line in face order. */
        int nfl = (d == 0) ? rw + 1 : rh + 1;
        int nl = (d == 0) ? rh : rw;
        real *F = (real *)malloc((size_t)nl * nfl * nf * sizeof(real));
        OR_PARALLEL_FOR
        for (long f = 0; f < (long)nl * nfl; ++f) {
            int l = (int)(f / nfl), s = (int)(f % nfl);
            real QL[14], QR[14];
            if (d == 0) {
                int j = ya + l, si = xa + s;
                face_state(c, cell(b, Qp, si - 2, j), cell(b, Qp, si - 1, j),
                           cell(b, Qp, si, j), +1.0, QL);
                face_state(c, cell(b, Qp, si - 1, j), cell(b, Qp, si, j),
                           cell(b, Qp, si + 1, j), -1.0, QR);
            } else {
                int i = xa + l, sj = ya + s;
                face_state(c, cell(b, Qp, i, sj - 2), cell(b, Qp, i, sj - 1),
                           cell(b, Qp, i, sj), +1.0, QL);
                face_state(c, cell(b, Qp, i, sj - 1), cell(b, Qp, i, sj),
                           cell(b, Qp, i, sj + 1), -1.0, QR);
            }
            face_flux(c, QL, QR, d, F + (size_t)f * nf);
        }
        OR_PARALLEL_FOR
        for (int l = 0; l < nl; ++l)
            for (int s = 1; s < nfl; ++s) {
                const real *Fr = F + ((size_t)l * nfl + s) * nf;
                const real *Fl = Fr - nf;
                /* cell s-1 of line l */
                real *Lc = (d == 0) ? L + ((size_t)l * rw + (s - 1)) * nf
                                    : L + ((size_t)(s - 1) * rw + l) * nf;
                for (int k = 0; k < nf; ++k) Lc[k] -= (Fr[k] - Fl[k]) / h;
            }
        free(F);
    }
    free(Qp);
}

static void blk_init(const or_cfg *c, blk *b, int i0, int j0, int w, int h) {
    b->i0 = i0; b->j0 = j0; b->w = w; b->h = h;
    b->mx = OR_MARGIN;
    b->my = (c->ny == 1) ? 0 : OR_MARGIN;
    b->W = w + 2 * b->mx;
    b->H = h + 2 * b->my;
    b->nf = nfields(c);
    size_t n = (size_t)b->W * b->H * b->nf;
    b->gp = (real *)malloc(n * sizeof(real));
    for (size_t k = 0; k < n; ++k) b->gp[k] = NAN;
}

int or_block_residual(const or_cfg *c, int i0, int j0, int w, int h,
                      const real *Ub, real *Lout) {
    blk b;
    blk_init(c, &b, i0, j0, w, h);
    size_t n = (size_t)b.W * b.H * b.nf;
    real *A = (real *)malloc(n * sizeof(real));
    memcpy(A, Ub, n * sizeof(real));
    fill_bc(c, &b, A);
    residual_region(c, &b, A, 0, w, 0, h, Lout);
    free(A);
    free(b.gp);
    return 0;
}

/* One step (forward Euler or midpoint RK2, Sec. 3):
 *   FE : U^{n+1} = U^n + dt L(U^n)
 *   RK2: U*      = U^n + dt/2 L(U^n),  U^{n+1} = U^n + dt L(U*)
 * With the point-implicit source, L is -div F and every stage result is
 * relaxed over its own step (dt, or dt/2 for U*) by relax_cell. */
int or_block_step(const or_cfg *c, int i0, int j0, int w, int h,
                  const real *Ub, real dt, real *Uout) {
    blk b;
    blk_init(c, &b, i0, j0, w, h);
    int nf = b.nf;
    size_t n = (size_t)b.W * b.H * nf;
    real *A = (real *)malloc(n * sizeof(real));
    memcpy(A, Ub, n * sizeof(real));
    fill_bc(c, &b, A);
    if (c->integrator == OR_FE) {
        real *L = (real *)malloc((size_t)w * h * nf * sizeof(real));
        residual_region(c, &b, A, 0, w, 0, h, L);
        OR_PARALLEL_FOR
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                real *Uc = cell(&b, A, i, j);
                real *Lc = L + ((size_t)j * w + i) * nf;
                real *Uo = Uout + ((size_t)j * w + i) * nf;
                for (int k = 0; k < nf; ++k) Uo[k] = Uc[k] + dt * Lc[k];
                if (c->source_scheme == OR_SRC_POINT_IMPLICIT) relax_cell(c, Uo, dt);
            }
        free(L);
        free(A);
        free(b.gp);
        return 0;
    }
    /* stage 1 on the interior plus 2 layers into every cut side */
    int xa = side_is_boundary(c, &b, 0) ? 0 : -2;
    int xb = side_is_boundary(c, &b, 1) ? w : w + 2;
    int ya = 0, yb = h;
    if (c->ny > 1) {
        ya = side_is_boundary(c, &b, 2) ? 0 : -2;
        yb = side_is_boundary(c, &b, 3) ? h : h + 2;
    }
    int rw = xb - xa, rh = yb - ya;
    real *L = (real *)malloc((size_t)rw * rh * nf * sizeof(real));
    residual_region(c, &b, A, xa, xb, ya, yb, L);
    real *S = (real *)malloc(n * sizeof(real));
    memcpy(S, A, n * sizeof(real));
    OR_PARALLEL_FOR
    for (int j = ya; j < yb; ++j)
        for (int i = xa; i < xb; ++i) {
            real *Uc = cell(&b, A, i, j);
            real *Sc = cell(&b, S, i, j);
            real *Lc = L + ((size_t)(j - ya) * rw + (i - xa)) * nf;
            for (int k = 0; k < nf; ++k) Sc[k] = Uc[k] + 0.5 * dt * Lc[k];
            if (c->source_scheme == OR_SRC_POINT_IMPLICIT) relax_cell(c, Sc, 0.5 * dt);
        }
    fill_bc(c, &b, S);
    real *L2 = (real *)malloc((size_t)w * h * nf * sizeof(real));
    residual_region(c, &b, S, 0, w, 0, h, L2);
    OR_PARALLEL_FOR
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            real *Uc = cell(&b, A, i, j);
            real *Lc = L2 + ((size_t)j * w + i) * nf;
            real *Uo = Uout + ((size_t)j * w + i) * nf;
            for (int k = 0; k < nf; ++k) Uo[k] = Uc[k] + dt * Lc[k];
            if (c->source_scheme == OR_SRC_POINT_IMPLICIT) relax_cell(c, Uo, dt);
        }
    free(L2);
    free(S);
    free(L);
    free(A);
    free(b.gp);
    return 0;
}

/* Reading (CFL in 2D): m = max over cells of sum_d max(|lmin_d|,|lmax_d|)/dx_d
 * at cell centres of U^n; dt = CFL/m. */
real or_max_rate(const or_cfg *c, const real *U) {
    int nf = nfields(c);
    real dx = (c->x1 - c->x0) / c->nx;
    real dy = (c->y1 - c->y0) / c->ny;
    int ndim = (c->ny == 1) ? 1 : 2;
    real m = 0.0;
    OR_PARALLEL_FOR_MAX(m)
    for (size_t n = 0; n < (size_t)c->nx * c->ny; ++n) {
        real Q[14];
        cons2prim(c, U + n * nf, Q);
        real r = 0.0;
        for (int d = 0; d < ndim; ++d) {
            real lmin, lmax;
            wspeeds(c, Q, d, &lmin, &lmax);
            real a = fabs(lmin) > fabs(lmax) ? fabs(lmin) : fabs(lmax);
            r += a / (d == 0 ? dx : dy);
        }
        if (r > m) m = r;
    }
    return m;
}

real or_dt(const or_cfg *c, const real *U, real t, real t_end) {
    real dt = c->cfl / or_max_rate(c, U);
    if (t + dt > t_end) dt = t_end - t;
    return dt;
}

/* Whole-grid step: copy into a block with margins; periodic sides wrap. */
int or_step(const or_cfg *c, real *U, real dt) {
    blk b;
    blk_init(c, &b, 0, 0, c->nx, c->ny);
    int nf = b.nf;
    size_t n = (size_t)b.W * b.H * nf;
    real *A = (real *)calloc(n, sizeof(real));
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
            memcpy(cell(&b, A, i, j), U + ((size_t)j * c->nx + i) * nf,
                   nf * sizeof(real));
    /* periodic wrap into the margins (all 4 layers) */
    if (c->side[0].base_type == OR_BC_PERIODIC)
        for (int j = 0; j < c->ny; ++j)
            for (int g = 1; g <= OR_MARGIN; ++g) {
                memcpy(cell(&b, A, -g, j), cell(&b, A, c->nx - g, j), nf * sizeof(real));
                memcpy(cell(&b, A, c->nx - 1 + g, j), cell(&b, A, g - 1, j),
                       nf * sizeof(real));
            }
    if (c->ny > 1 && c->side[2].base_type == OR_BC_PERIODIC)
        for (int i = -b.mx; i < c->nx + b.mx; ++i)
            for (int g = 1; g <= OR_MARGIN; ++g) {
                memcpy(cell(&b, A, i, -g), cell(&b, A, i, c->ny - g), nf * sizeof(real));
                memcpy(cell(&b, A, i, c->ny - 1 + g), cell(&b, A, i, g - 1),
                       nf * sizeof(real));
            }
    int rc = or_block_step(c, 0, 0, c->nx, c->ny, A, dt, U);
    free(A);
    free(b.gp);
    return rc;
}

int or_run(const or_cfg *c, real *U, real *t, real t_end, int max_steps,
           real *dt_hist) {
    int n = 0;
    while (n < max_steps && *t < t_end) {
        real dt = or_dt(c, U, *t, t_end);
        if (!(dt > 0.0)) break;
        or_step(c, U, dt);
        if (dt_hist) dt_hist[n] = dt;
        *t += dt;
        ++n;
    }
    return n;
}
