// mxe_physics.cuh -- device-side point physics of the 5- and 14-moment
// maximum-entropy systems with interpolative closure (Boccelli et al.,
// JCP 2024, arXiv 2401.15233), templated on the arithmetic type.
//
// What differs from a literal transcription of the paper (all algebraically
// identical):
//   * K_ijkm is never formed: Q_ijk = K_ijkm q_m = 2[w_i (P^2)_jk +
//     w_j (P^2)_ik + w_k (P^2)_ij] with w = P B^-1 q
//     (Eq. closure-14mom-Qijk-approx with K as printed).
//   * For a flux in direction k only the slice Q_kab (6 values), R_akjj
//     (3 values) and S_kiijj are evaluated; W enters only through its row k
//     contracted with B^-1 q.
//   * sigma uses the rationalised root X / (4T (sqrt(A^2+X) - A)) when A < 0,
//     and the wave-speed bracket zeta + sqrt(zeta^2 + D0) its rationalised form
//     when zeta < 0 (no cancellation); a negative discriminant is clamped.
//   * The 14-moment flux is written as u_k U + (central part) so that the
//     conserved face state is reused.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mxe {

// ---------------------------------------------------------------- math shims
template <class T> struct M;
template <> struct M<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return ::exp(x); }
    static __device__ __forceinline__ double log_(double x) { return ::log(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
};
template <> struct M<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return ::sqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
    static __device__ __forceinline__ float log_(float x) { return __logf(x); }
    static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
};

// Explicitly rounded operations (never fused into FMA by the compiler).
// Used where a result feeds a branch of the scheme (primitive recovery, the
// limiter, face reconstruction, the stage update) so that those values are
// rounded exactly as in the reference evaluation order.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

struct SchemeParams {
    double sigma_lim;    // Appendix A
    double k_ws;         // Sec. 5.1 inflation
    int    flux;         // 0 HLL, 1 Rusanov
    int    limiter;      // 0 minmod, 1 van Albada
    int    order;        // 1 or 2
};

struct RelaxParams {
    int    model;        // 0 none, 1 const, 2 hard-sphere-like
    double tau_ref, rho_ref, T_ref;
    int    implicit;     // 1: point-implicit source (relax after each stage)
};

// sigma_bar = min(max(sigma, sigma_lim), 1)   (Appendix A; upper clamp: reading)
template <class T>
__device__ __forceinline__ T clamp_sigma(T s, T slim) {
    s = s < slim ? slim : s;
    return s > T(1) ? T(1) : s;
}

// sigma = [A + sqrt(A^2 + X)] / (4 Tn), rationalised for A < 0.
template <class T>
__device__ __forceinline__ T sigma_root(T A, T X, T Tn) {
    T rt = M<T>::sqrt_(A * A + X);
    return A >= T(0) ? (A + rt) / (T(4) * Tn) : X / (T(4) * Tn * (rt - A));
}

// zeta + sqrt(zeta^2 + D0), discriminant clamped at 0, rationalised for zeta < 0.
template <class T>
__device__ __forceinline__ T hyp_bracket(T zeta, T D0) {
    T D = zeta * zeta + D0;
    if (D <= T(0)) return zeta;
    T rt = M<T>::sqrt_(D);
    return zeta >= T(0) ? zeta + rt : D0 / (rt - zeta);
}

// B = 5 - 4 sqrt(s) + sqrt(10 - 16 sqrt(s) + 6 s) and Y = B + E^2 - 2 E sqrt(B)
// of the wave-speed fits.  Double: as printed.  Float: the algebraically
// identical 10 - 16 r + 6 r^2 = 2 (5 - 3 r)(1 - r) (r = sqrt s) and
// Y = (sqrt B - E)^2, which keep their digits as sigma -> 1.
template <class T> struct WsTerms;
template <> struct WsTerms<double> {
    static __device__ __forceinline__ void get(double ssb, double sb, double E, double& B,
                                               double& Y) {
        B = 5.0 - 4.0 * ssb + ::sqrt(10.0 - 16.0 * ssb + 6.0 * sb);
        Y = B + E * E - 2.0 * E * ::sqrt(B);
    }
};
template <> struct WsTerms<float> {
    static __device__ __forceinline__ void get(float ssb, float sb, float E, float& B,
                                               float& Y) {
        B = 5.0f - 4.0f * ssb + ::sqrtf(2.0f * (5.0f - 3.0f * ssb) * (1.0f - ssb));
        float d = ::sqrtf(B) - E;
        Y = d * d;
    }
};

// =========================================================================
// 5-moment system (Sec. 2.3)
// =========================================================================
template <class T>
__device__ __forceinline__ void prim2cons5(const T* Q, T* U) {
    T rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * u * u + P;
    U[3] = rho * u * u * u + T(3) * u * P + q;
    U[4] = rho * u * u * u * u + T(6) * u * u * P + T(4) * u * q + r;
}

template <class T>
__device__ __forceinline__ void cons2prim5(const T* U, T* Q) {
    T rho = U[0];
    T u = U[1] / rho;
    T P = U[2] - rho * u * u;
    T q = U[3] - rho * u * u * u - T(3) * u * P;
    T r = U[4] - rho * u * u * u * u - T(6) * u * u * P - T(4) * u * q;
    Q[0] = rho; Q[1] = u; Q[2] = P; Q[3] = q; Q[4] = r;
}

// Primitive recovery with every operation explicitly rounded, in the order
// rho, u = U1/rho, P = U2 - (rho u) u, q = U3 - ((rho u) u) u - (3u) P,
// r = U4 - (((rho u) u) u) u - ((6u) u) P - (4u) q.
__device__ __forceinline__ void cons2prim5_rn(const double* U, double* Q) {
    double rho = U[0];
    double u = U[1] / rho;
    double ru = mul_rn(rho, u), ruu = mul_rn(ru, u), ruuu = mul_rn(ruu, u);
    double P = sub_rn(U[2], ruu);
    double q = sub_rn(sub_rn(U[3], ruuu), mul_rn(mul_rn(3.0, u), P));
    double r = sub_rn(sub_rn(sub_rn(U[4], mul_rn(ruuu, u)), mul_rn(mul_rn(mul_rn(6.0, u), u), P)),
                      mul_rn(mul_rn(4.0, u), q));
    Q[0] = rho; Q[1] = u; Q[2] = P; Q[3] = q; Q[4] = r;
}

// Baradaran fit, Eq. (ws-max-baradaran-orig), with shared E, C, Y.
template <class T>
__device__ __forceinline__ T lam5_star(T qs, T sb, T E, T C, T Y) {
    T D0 = T(-0.8) * qs * sb * C + T(4) * sb * sb * Y;
    return hyp_bracket(qs, D0) / (T(2) * sb) + E;
}

// Primitive moments of cons5(W) + dU from the increment alone (FP32 path;
// every term scales with the increment, see prim_increment14).
__device__ __forceinline__ void prim_increment5(const float* W, const float* dU, float* Wn) {
    float rho = W[0], u = W[1], P = W[2], q = W[3];
    float drho = dU[0];
    float rho1 = rho + drho;
    float du = (dU[1] - u * drho) / rho1;
    float u1 = u + du;
    float dP = dU[2] - drho * u * u - rho1 * (2.0f * u * du + du * du);
    float P1 = P + dP;
    float s = 2.0f * u * du + du * du;                      // u1^2 - u^2
    // G = rho u^3 + 3 u P
    float dG = drho * u * u * u + rho1 * du * (3.0f * u * u + 3.0f * u * du + du * du)
             + 3.0f * (du * P1 + u * dP);
    float dq = dU[3] - dG;
    float q1 = q + dq;
    // K = rho u^4 + 6 u^2 P + 4 u q
    float dK = drho * u * u * u * u + rho1 * s * (2.0f * u * u + s) + 6.0f * (s * P1 + u * u * dP)
             + 4.0f * (du * q1 + u * dq);
    Wn[0] = rho1; Wn[1] = u1; Wn[2] = P1; Wn[3] = q1;
    Wn[4] = W[4] + (dU[4] - dK);
}

// Raw sigma of Eq. (sigma-mapping-5mom) from the dimensionless q*, r*.
template <class T>
__device__ __forceinline__ T sigma5(T qs, T rs) {
    return sigma_root(T(3) - rs, T(8) * qs * qs, T(1));
}

// Face-state evaluation: conserved U, x-flux F (Eq. 5mom-sys-eqs with the
// closure of Eq. closure-1D1V-s-approx) and wave speeds.
template <class T>
__device__ __forceinline__ void face_eval5(const T* Q, T sigma_lim, T k_ws, T* U, T* F,
                                           T& lmin, T& lmax) {
    T rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    T th = P / rho;
    T sq = M<T>::sqrt_(th);
    T sc3 = rho * th * sq;
    T qs = q / sc3;
    T rs = r / (rho * th * th);
    T sb = clamp_sigma(sigma5(qs, rs), sigma_lim);
    T ssb = M<T>::sqrt_(sb);
    T ss = qs * qs * qs / (sb * sb) + (T(10) - T(8) * ssb) * qs;
    T s = ss * sc3 * th;
    prim2cons5(Q, U);
    F[0] = rho * u;
    F[1] = rho * u * u + P;
    F[2] = rho * u * u * u + T(3) * u * P + q;
    F[3] = rho * u * u * u * u + T(6) * u * u * P + T(4) * u * q + r;
    F[4] = rho * u * u * u * u * u + T(10) * u * u * u * P + T(10) * u * u * q + T(5) * u * r + s;
    T C = M<T>::sqrt_(T(3) - T(3) * sb);
    T E = T(0.8) * C;
    T B, Y;
    WsTerms<T>::get(ssb, sb, E, B, Y);
    lmax = u + k_ws * lam5_star(qs, sb, E, C, Y) * sq;
    lmin = u - k_ws * lam5_star(-qs, sb, E, C, Y) * sq;
}

template <class T>
__device__ __forceinline__ void face_eval5(const T* Q, const SchemeParams& sp, T* U, T* F,
                                           T& lmin, T& lmax) {
    T rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    T th = P / rho;
    T sq = M<T>::sqrt_(th);
    T sc3 = rho * th * sq;
    T qs = q / sc3;
    T rs = r / (rho * th * th);
    T sb = clamp_sigma(sigma5(qs, rs), T(sp.sigma_lim));
    T ssb = M<T>::sqrt_(sb);
    T ss = qs * qs * qs / (sb * sb) + (T(10) - T(8) * ssb) * qs;
    T s = ss * sc3 * th;
    prim2cons5(Q, U);
    F[0] = rho * u;
    F[1] = rho * u * u + P;
    F[2] = rho * u * u * u + T(3) * u * P + q;
    F[3] = rho * u * u * u * u + T(6) * u * u * P + T(4) * u * q + r;
    F[4] = rho * u * u * u * u * u + T(10) * u * u * u * P + T(10) * u * u * q + T(5) * u * r + s;
    T C = M<T>::sqrt_(T(3) - T(3) * sb);
    T E = T(0.8) * C;
    T B = T(5) - T(4) * ssb + M<T>::sqrt_(T(10) - T(16) * ssb + T(6) * sb);
    T Y = B + E * E - T(2) * E * M<T>::sqrt_(B);
    T k = T(sp.k_ws);
    lmax = u + k * lam5_star(qs, sb, E, C, Y) * sq;
    lmin = u - k * lam5_star(-qs, sb, E, C, Y) * sq;
}

template <class T>
__device__ __forceinline__ void rate5(const T* Q, const SchemeParams& sp, T& amax, T& sig_raw) {
    T rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    T th = P / rho;
    T sq = M<T>::sqrt_(th);
    T qs = q / (rho * th * sq);
    T rs = r / (rho * th * th);
    sig_raw = sigma5(qs, rs);
    T sb = clamp_sigma(sig_raw, T(sp.sigma_lim));
    T ssb = M<T>::sqrt_(sb);
    T C = M<T>::sqrt_(T(3) - T(3) * sb);
    T E = T(0.8) * C;
    T B = T(5) - T(4) * ssb + M<T>::sqrt_(T(10) - T(16) * ssb + T(6) * sb);
    T Y = B + E * E - T(2) * E * M<T>::sqrt_(B);
    T k = T(sp.k_ws);
    T lmax = u + k * lam5_star(qs, sb, E, C, Y) * sq;
    T lmin = u - k * lam5_star(-qs, sb, E, C, Y) * sq;
    T a = fabs(lmin), b = fabs(lmax);
    amax = a > b ? a : b;
}

// BGK source of Eq. (5mom-sys-eqs).
template <class T>
__device__ __forceinline__ void source5(const T* Q, T tau, T* C) {
    T rho = Q[0], u = Q[1], P = Q[2], q = Q[3], r = Q[4];
    C[0] = T(0); C[1] = T(0); C[2] = T(0);
    C[3] = -q / tau;
    C[4] = -(T(4) * u * q + r - T(3) * P * P / rho) / tau;
}

// =========================================================================
// 14-moment system (Sec. 2.4)
// Q = (rho, ux, uy, uz, Pxx, Pxy, Pxz, Pyy, Pyz, Pzz, qx, qy, qz, R)
// symmetric 3x3 stored as s[6] = (xx, xy, xz, yy, yz, zz)
// =========================================================================
__device__ __forceinline__ constexpr int sidx(int a, int b) {
    // index of (a,b) in the symmetric packing
    return a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5));
}

template <class T>
__device__ __forceinline__ void prim2cons14(const T* Q, T* U) {
    T rho = Q[0], ux = Q[1], uy = Q[2], uz = Q[3];
    T Pxx = Q[4], Pxy = Q[5], Pxz = Q[6], Pyy = Q[7], Pyz = Q[8], Pzz = Q[9];
    T u2 = ux * ux + uy * uy + uz * uz;
    T trP = Pxx + Pyy + Pzz;
    T Pux = Pxx * ux + Pxy * uy + Pxz * uz;
    T Puy = Pxy * ux + Pyy * uy + Pyz * uz;
    T Puz = Pxz * ux + Pyz * uy + Pzz * uz;
    T uPu = ux * Pux + uy * Puy + uz * Puz;
    T uq = ux * Q[10] + uy * Q[11] + uz * Q[12];
    U[0] = rho;
    U[1] = rho * ux; U[2] = rho * uy; U[3] = rho * uz;
    U[4] = rho * ux * ux + Pxx; U[5] = rho * ux * uy + Pxy; U[6] = rho * ux * uz + Pxz;
    U[7] = rho * uy * uy + Pyy; U[8] = rho * uy * uz + Pyz; U[9] = rho * uz * uz + Pzz;
    T e = rho * u2 + trP;
    U[10] = ux * e + T(2) * Pux + Q[10];
    U[11] = uy * e + T(2) * Puy + Q[11];
    U[12] = uz * e + T(2) * Puz + Q[12];
    U[13] = rho * u2 * u2 + T(2) * u2 * trP + T(4) * uPu + T(4) * uq + Q[13];
}

template <class T>
__device__ __forceinline__ void cons2prim14(const T* U, T* Q) {
    T rho = U[0];
    T ir = T(1) / rho;
    T ux = U[1] * ir, uy = U[2] * ir, uz = U[3] * ir;
    T Pxx = U[4] - rho * ux * ux, Pxy = U[5] - rho * ux * uy, Pxz = U[6] - rho * ux * uz;
    T Pyy = U[7] - rho * uy * uy, Pyz = U[8] - rho * uy * uz, Pzz = U[9] - rho * uz * uz;
    T u2 = ux * ux + uy * uy + uz * uz;
    T trP = Pxx + Pyy + Pzz;
    T Pux = Pxx * ux + Pxy * uy + Pxz * uz;
    T Puy = Pxy * ux + Pyy * uy + Pyz * uz;
    T Puz = Pxz * ux + Pyz * uy + Pzz * uz;
    T e = rho * u2 + trP;
    T qx = U[10] - ux * e - T(2) * Pux;
    T qy = U[11] - uy * e - T(2) * Puy;
    T qz = U[12] - uz * e - T(2) * Puz;
    T uPu = ux * Pux + uy * Puy + uz * Puz;
    T uq = ux * qx + uy * qy + uz * qz;
    T R = U[13] - rho * u2 * u2 - T(2) * u2 * trP - T(4) * uPu - T(4) * uq;
    Q[0] = rho; Q[1] = ux; Q[2] = uy; Q[3] = uz;
    Q[4] = Pxx; Q[5] = Pxy; Q[6] = Pxz; Q[7] = Pyy; Q[8] = Pyz; Q[9] = Pzz;
    Q[10] = qx; Q[11] = qy; Q[12] = qz; Q[13] = R;
}

// Primitive recovery with every operation explicitly rounded (sums in index
// order, products left to right):
//   u_i = U_i/rho, P_ij = E_ij - (rho u_i) u_j, |u|^2, tr P,
//   u.P.u = sum_i sum_j (u_i u_j) P_ij,
//   q_i = ((H_i - (rho u_i)|u|^2) - u_i tr P) - 2 (sum_j u_j P_ij),
//   R = (((E4 - (rho |u|^2)|u|^2) - (2|u|^2) tr P) - 4 u.P.u) - 4 u.q
__device__ __forceinline__ void cons2prim14_rn(const double* U, double* Q) {
    double rho = U[0];
    double u[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
    double P[3][3];
    int idx = 4;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            P[i][j] = sub_rn(U[idx++], mul_rn(mul_rn(rho, u[i]), u[j]));
            P[j][i] = P[i][j];
        }
    double u2 = add_rn(add_rn(mul_rn(u[0], u[0]), mul_rn(u[1], u[1])), mul_rn(u[2], u[2]));
    double trP = add_rn(add_rn(P[0][0], P[1][1]), P[2][2]);
    double uPu = mul_rn(mul_rn(u[0], u[0]), P[0][0]);
#pragma unroll
    for (int n = 1; n < 9; ++n) {
        int i = n / 3, j = n % 3;
        uPu = add_rn(uPu, mul_rn(mul_rn(u[i], u[j]), P[i][j]));
    }
    double q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double uP = add_rn(add_rn(mul_rn(u[0], P[i][0]), mul_rn(u[1], P[i][1])), mul_rn(u[2], P[i][2]));
        q[i] = sub_rn(sub_rn(sub_rn(U[10 + i], mul_rn(mul_rn(rho, u[i]), u2)), mul_rn(u[i], trP)),
                      mul_rn(2.0, uP));
    }
    double uq = add_rn(add_rn(mul_rn(u[0], q[0]), mul_rn(u[1], q[1])), mul_rn(u[2], q[2]));
    double R = sub_rn(sub_rn(sub_rn(sub_rn(U[13], mul_rn(mul_rn(rho, u2), u2)),
                                    mul_rn(mul_rn(2.0, u2), trP)),
                             mul_rn(4.0, uPu)),
                      mul_rn(4.0, uq));
    Q[0] = rho; Q[1] = u[0]; Q[2] = u[1]; Q[3] = u[2];
    Q[4] = P[0][0]; Q[5] = P[0][1]; Q[6] = P[0][2]; Q[7] = P[1][1]; Q[8] = P[1][2]; Q[9] = P[2][2];
    Q[10] = q[0]; Q[11] = q[1]; Q[12] = q[2]; Q[13] = R;
}

// symmetric products
template <class T>
__device__ __forceinline__ void sym_mul(const T* A, const T* B, T* C) {
    // C = A B for symmetric A, B whose product is symmetric (A, B commute:
    // both are polynomials in the same P)
    C[0] = A[0] * B[0] + A[1] * B[1] + A[2] * B[2];
    C[1] = A[0] * B[1] + A[1] * B[3] + A[2] * B[4];
    C[2] = A[0] * B[2] + A[1] * B[4] + A[2] * B[5];
    C[3] = A[1] * B[1] + A[3] * B[3] + A[4] * B[4];
    C[4] = A[1] * B[2] + A[3] * B[4] + A[4] * B[5];
    C[5] = A[2] * B[2] + A[4] * B[4] + A[5] * B[5];
}

template <class T>
__device__ __forceinline__ T sym_inv(const T* A, T* I) {
    T c00 = A[3] * A[5] - A[4] * A[4];
    T c01 = A[2] * A[4] - A[1] * A[5];
    T c02 = A[1] * A[4] - A[2] * A[3];
    T det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    T id = T(1) / det;
    I[0] = c00 * id;
    I[1] = c01 * id;
    I[2] = c02 * id;
    I[3] = (A[0] * A[5] - A[2] * A[2]) * id;
    I[4] = (A[1] * A[2] - A[0] * A[4]) * id;
    I[5] = (A[0] * A[3] - A[1] * A[1]) * id;
    return det;
}

template <class T>
__device__ __forceinline__ void sym_vec(const T* A, const T* v, T* o) {
    o[0] = A[0] * v[0] + A[1] * v[1] + A[2] * v[2];
    o[1] = A[1] * v[0] + A[3] * v[1] + A[4] * v[2];
    o[2] = A[2] * v[0] + A[4] * v[1] + A[5] * v[2];
}

// Dimensionless state and raw sigma (Eq. sigma-mapping-14mom with rho* = 1).
template <class T>
struct Dimless14 {
    T th, sq;          // p/rho, sqrt(p/rho)
    T Ps[6];           // P*
    T qs[3];           // q*
    T trPs, T2;        // tr P*, tr P*^2
    T Pi[6];           // P*^-1
    T y[3];            // P*^-1 q*
    T sig;             // raw sigma
    T det;             // det P* (<= 1 since tr P* = 3; small = ill-conditioned)
};

template <class T>
__device__ __forceinline__ void dimless14(const T* Q, Dimless14<T>& d) {
    T rho = Q[0];
    T p = (Q[4] + Q[7] + Q[9]) / T(3);
    T ip = T(1) / p;
    d.th = p / rho;
    d.sq = M<T>::sqrt_(d.th);
    T isc3 = T(1) / (rho * d.th * d.sq);
#pragma unroll
    for (int n = 0; n < 6; ++n) d.Ps[n] = Q[4 + n] * ip;
#pragma unroll
    for (int n = 0; n < 3; ++n) d.qs[n] = Q[10 + n] * isc3;
    T Rs = Q[13] / (rho * d.th * d.th);
    d.trPs = d.Ps[0] + d.Ps[3] + d.Ps[5];
    d.T2 = d.Ps[0] * d.Ps[0] + d.Ps[3] * d.Ps[3] + d.Ps[5] * d.Ps[5]
         + T(2) * (d.Ps[1] * d.Ps[1] + d.Ps[2] * d.Ps[2] + d.Ps[4] * d.Ps[4]);
    d.det = sym_inv(d.Ps, d.Pi);
    sym_vec(d.Pi, d.qs, d.y);
    T qPq = d.qs[0] * d.y[0] + d.qs[1] * d.y[1] + d.qs[2] * d.y[2];
    T A = T(2) * d.T2 + d.trPs * d.trPs - Rs;
    T X = T(8) * d.T2 * qPq;
    d.sig = sigma_root(A, X, d.T2);
}

// Eq. (14mom-approx-ws-equations): lambda*_max and lambda*_min along k.
template <class T, int K>
__device__ __forceinline__ void lam14_star(const Dimless14<T>& d, T sb, T& lp, T& lm) {
    constexpr int E1 = (K + 1) % 3, E2 = (K + 2) % 3;
    T Pkk = d.Ps[sidx(K, K)];
    T qd = d.qs[K];
    T qperp = M<T>::sqrt_(d.qs[E1] * d.qs[E1] + d.qs[E2] * d.qs[E2]);
    T lP = M<T>::log_(Pkk);
    T a = T(1.4) * M<T>::exp_(T(1.1) * lP - Pkk * Pkk);
    T b = T(0.9) * Pkk * M<T>::exp_(T(-0.5) * M<T>::exp_(T(1.4) * lP));
    T ssb = M<T>::sqrt_(sb);
    T C = M<T>::sqrt_((T(3) - T(3) * sb) * Pkk);
    T E = T(0.8) * C;
    T B, Y;
    WsTerms<T>::get(ssb, sb, E, B, Y);
    T al = qperp * (T(0.6) * Pkk * Pkk - T(0.38) * Pkk + T(0.35));
    T base = T(4) * sb * sb * Y + qperp * qperp / T(10);
    T pre = (a * sb + b) / (T(2) * sb);
    T zp = qd + al;
    T zm = -qd + al;
    lp = pre * hyp_bracket(zp, T(-0.8) * zp * sb * C + base) + E;
    lm = -(pre * hyp_bracket(zm, T(-0.8) * zm * sb * C + base) + E);
}

// Closure slice for direction K, dimensional: Qk[6] = Q_Kab (sym packing),
// Rk[3] = R_aKjj, Sk = S_Kiijj (Eqs. closure-14mom-Qijk/Rijkk/Sijjkk).
template <class T, int K>
__device__ __forceinline__ void closure14_slice(const T* Q, const Dimless14<T>& d, T sb,
                                                T* Qk, T* Rk, T& Sk) {
    const T* Ps = d.Ps;
    T P2[6], P3[6];
    sym_mul(Ps, Ps, P2);
    sym_mul(P2, Ps, P3);
    T trP3 = P3[0] + P3[3] + P3[5];
    T Bm[6], Bi[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) Bm[n] = T(2) * Ps[n] * d.T2 + T(4) * P3[n];
    sym_inv(Bm, Bi);
    T v[3], w[3];
    sym_vec(Bi, d.qs, v);        // B^-1 q*
    sym_vec(Ps, v, w);           // w = P* B^-1 q*
    // Q_Kab = 2 [w_K (P^2)_ab + w_a (P^2)_Kb + w_b (P^2)_Ka]
    T Qs[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
            Qs[sidx(a, b)] = T(2) * (w[K] * P2[sidx(a, b)] + w[a] * P2[sidx(K, b)]
                                     + w[b] * P2[sidx(K, a)]);
    T isb = T(1) / sb;
    // R_aKjj = (1/sigma) Q_aKl y_l + 2(1-sigma) (P^2)_aK + P_aK tr P
    T Rs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T s = Qs[sidx(a, 0)] * d.y[0] + Qs[sidx(a, 1)] * d.y[1] + Qs[sidx(a, 2)] * d.y[2];
        Rs[a] = s * isb + T(2) * (T(1) - sb) * P2[sidx(a, K)] + Ps[sidx(a, K)] * d.trPs;
    }
    // S_K = (1/sigma^2) y_a y_b Q_Kab + 2 sqrt(sigma) trP q_K + (1 - sqrt(sigma)) (W q)_K
    T yQy = Qs[0] * d.y[0] * d.y[0] + Qs[3] * d.y[1] * d.y[1] + Qs[5] * d.y[2] * d.y[2]
          + T(2) * (Qs[1] * d.y[0] * d.y[1] + Qs[2] * d.y[0] * d.y[2] + Qs[4] * d.y[1] * d.y[2]);
    // row K of the W bracket (before B^-1), contracted with v = B^-1 q*
    T t = d.trPs, t2 = t * t;
    T c1 = T(2) * t2 * t + T(12) * trP3 - T(2) * d.T2 * t;     // coefficient of P
    T c2 = T(14) * d.T2 - T(6) * t2;                             // of P^2
    T c3 = T(20) * t;                                            // of P^3
    T Wq = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T P4Ka = P2[sidx(K, 0)] * P2[sidx(0, a)] + P2[sidx(K, 1)] * P2[sidx(1, a)]
               + P2[sidx(K, 2)] * P2[sidx(2, a)];
        T m = c1 * Ps[sidx(K, a)] + c2 * P2[sidx(K, a)] + c3 * P3[sidx(K, a)] + T(20) * P4Ka;
        Wq += m * v[a];
    }
    T ssb = M<T>::sqrt_(sb);
    T Ss = yQy * isb * isb + T(2) * ssb * t * d.qs[K] + (T(1) - ssb) * Wq;
    // re-dimensionalise
    T rho = Q[0];
    T sc3 = rho * d.th * d.sq, sc4 = rho * d.th * d.th, sc5 = sc4 * d.sq;
#pragma unroll
    for (int n = 0; n < 6; ++n) Qk[n] = Qs[n] * sc3;
#pragma unroll
    for (int a = 0; a < 3; ++a) Rk[a] = Rs[a] * sc4;
    Sk = Ss * sc5;
}

// k-flux of the 14-moment system for given closing slice, written as
// u_k U + central part (the paper's expanded fluxes, regrouped).
template <class T, int K>
__device__ __forceinline__ void flux14(const T* Q, const T* U, const T* Qk, const T* Rk, T Sk,
                                       T* F) {
    T u[3] = {Q[1], Q[2], Q[3]};
    const T* P = Q + 4;                       // sym packing
    const T* q = Q + 10;
    T uk = u[K];
    T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T Pu[3];
    sym_vec(P, u, Pu);
    T Qu[3];                                  // (Q_K u)_a = Q_Kab u_b
    sym_vec(Qk, u, Qu);
#pragma unroll
    for (int n = 0; n < 14; ++n) F[n] = uk * U[n];
#pragma unroll
    for (int i = 0; i < 3; ++i) F[1 + i] += P[sidx(i, K)];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
            F[4 + sidx(i, j)] += u[i] * P[sidx(j, K)] + u[j] * P[sidx(i, K)] + Qk[sidx(i, j)];
    T g = T(2) * Pu[K] + q[K];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        F[10 + i] += u[i] * g + u2 * P[sidx(i, K)] + T(2) * Qu[i] + Rk[i];
    T uQu = u[0] * Qu[0] + u[1] * Qu[1] + u[2] * Qu[2];
    T uR = u[0] * Rk[0] + u[1] * Rk[1] + u[2] * Rk[2];
    F[13] += T(4) * u2 * Pu[K] + T(2) * u2 * q[K] + T(4) * uQu + T(4) * uR + Sk;
}

// Conserved state, k-flux and wave speeds of one face state.
template <class T, int K>
__device__ __forceinline__ void face_eval14(const T* Q, T sigma_lim, T k_ws, T* U, T* F,
                                            T& lmin, T& lmax) {
    Dimless14<T> d;
    dimless14(Q, d);
    T sb = clamp_sigma(d.sig, sigma_lim);
    T Qk[6], Rk[3], Sk;
    closure14_slice<T, K>(Q, d, sb, Qk, Rk, Sk);
    prim2cons14(Q, U);
    flux14<T, K>(Q, U, Qk, Rk, Sk, F);
    T lp, lm;
    lam14_star<T, K>(d, sb, lp, lm);
    lmax = Q[1 + K] + k_ws * lp * d.sq;
    lmin = Q[1 + K] + k_ws * lm * d.sq;
}

// The same, also returning the raw sigma and det P* of the state (the
// conditioning of its closure).
template <class T, int K>
__device__ __forceinline__ void face_eval14(const T* Q, T sigma_lim, T k_ws, T* U, T* F,
                                            T& lmin, T& lmax, T& sig, T& det) {
    Dimless14<T> d;
    dimless14(Q, d);
    T sb = clamp_sigma(d.sig, sigma_lim);
    T Qk[6], Rk[3], Sk;
    closure14_slice<T, K>(Q, d, sb, Qk, Rk, Sk);
    prim2cons14(Q, U);
    flux14<T, K>(Q, U, Qk, Rk, Sk, F);
    T lp, lm;
    lam14_star<T, K>(d, sb, lp, lm);
    lmax = Q[1 + K] + k_ws * lp * d.sq;
    lmin = Q[1 + K] + k_ws * lm * d.sq;
    sig = d.sig;
    det = d.det;
}

template <class T, int K>
__device__ __forceinline__ void face_eval14(const T* Q, const SchemeParams& sp, T* U, T* F,
                                            T& lmin, T& lmax) {
    face_eval14<T, K>(Q, T(sp.sigma_lim), T(sp.k_ws), U, F, lmin, lmax);
}

// CFL contribution max(|lmin|,|lmax|) along K and the raw sigma.
template <class T, int K>
__device__ __forceinline__ T amax14(const T* Q, const Dimless14<T>& d, T sigma_lim, T k_ws) {
    T sb = clamp_sigma(d.sig, sigma_lim);
    T lp, lm;
    lam14_star<T, K>(d, sb, lp, lm);
    T lmax = Q[1 + K] + k_ws * lp * d.sq;
    T lmin = Q[1 + K] + k_ws * lm * d.sq;
    T a = fabs(lmin), b = fabs(lmax);
    return a > b ? a : b;
}

template <class T, int K>
__device__ __forceinline__ T amax14(const T* Q, const Dimless14<T>& d, const SchemeParams& sp) {
    return amax14<T, K>(Q, d, T(sp.sigma_lim), T(sp.k_ws));
}

// Primitive moments of cons(W) + dU from the increment alone (FP32 path):
// every term below is proportional to the increment, so nothing of the size
// of the bulk-motion contributions (rho u^4 against R at high Mach number)
// is cancelled.  Algebraically W' = prim(cons(W) + dU) exactly.
__device__ __forceinline__ void prim_increment14(const float* W, const float* dU, float* Wn) {
    float rho = W[0];
    float u[3] = {W[1], W[2], W[3]};
    const float* P = W + 4;
    const float* q = W + 10;
    float drho = dU[0];
    float rho1 = rho + drho;
    float ir1 = 1.0f / rho1;
    float du[3], u1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        du[i] = (dU[1 + i] - u[i] * drho) * ir1;
        u1[i] = u[i] + du[i];
    }
    float dP[6];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b)
            dP[sidx(a, b)] = dU[4 + sidx(a, b)] - drho * u[a] * u[b]
                           - rho1 * (u[a] * du[b] + du[a] * u[b] + du[a] * du[b]);
    float P1[6];
#pragma unroll
    for (int n = 0; n < 6; ++n) P1[n] = P[n] + dP[n];
    float trP1 = P1[0] + P1[3] + P1[5];
    float dtr = dP[0] + dP[3] + dP[5];
    float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    float s = 2.0f * (u[0] * du[0] + u[1] * du[1] + u[2] * du[2])
            + (du[0] * du[0] + du[1] * du[1] + du[2] * du[2]);
    float Pdu[3], dPu1[3], Pu[3];
    sym_vec(P, du, Pdu);
    sym_vec(dP, u1, dPu1);
    sym_vec(P, u, Pu);
    float q1[3], dq[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float dG = drho * u[i] * u2 + rho1 * (du[i] * u2 + u1[i] * s) + du[i] * trP1 + u[i] * dtr
                 + 2.0f * (dPu1[i] + Pdu[i]);
        dq[i] = dU[10 + i] - dG;
        q1[i] = q[i] + dq[i];
    }
    float u1dPu1 = u1[0] * dPu1[0] + u1[1] * dPu1[1] + u1[2] * dPu1[2];
    float duPu = du[0] * Pu[0] + du[1] * Pu[1] + du[2] * Pu[2];
    float duPdu = du[0] * Pdu[0] + du[1] * Pdu[1] + du[2] * Pdu[2];
    float dK = drho * u2 * u2 + rho1 * s * (2.0f * u2 + s) + 2.0f * (s * trP1 + u2 * dtr)
             + 4.0f * (u1dPu1 + 2.0f * duPu + duPdu)
             + 4.0f * (du[0] * q1[0] + du[1] * q1[1] + du[2] * q1[2]
                       + u[0] * dq[0] + u[1] * dq[1] + u[2] * dq[2]);
    Wn[0] = rho1;
    Wn[1] = u1[0]; Wn[2] = u1[1]; Wn[3] = u1[2];
#pragma unroll
    for (int n = 0; n < 6; ++n) Wn[4 + n] = P1[n];
    Wn[10] = q1[0]; Wn[11] = q1[1]; Wn[12] = q1[2];
    Wn[13] = W[13] + (dU[13] - dK);
}

// BGK sources of Sec. 2.4.
template <class T>
__device__ __forceinline__ void source14(const T* Q, T tau, T* C) {
    T rho = Q[0], ux = Q[1], uy = Q[2], uz = Q[3];
    T Pxx = Q[4], Pxy = Q[5], Pxz = Q[6], Pyy = Q[7], Pyz = Q[8], Pzz = Q[9];
    T p = (Pxx + Pyy + Pzz) / T(3);
    C[0] = T(0); C[1] = T(0); C[2] = T(0); C[3] = T(0);
    C[4] = -(Pxx - p) / tau; C[5] = -Pxy / tau; C[6] = -Pxz / tau;
    C[7] = -(Pyy - p) / tau; C[8] = -Pyz / tau; C[9] = -(Pzz - p) / tau;
    T Pux = Pxx * ux + Pxy * uy + Pxz * uz;
    T Puy = Pxy * ux + Pyy * uy + Pyz * uz;
    T Puz = Pxz * ux + Pyz * uy + Pzz * uz;
    C[10] = -(T(2) * Pux + Q[10] - T(2) * ux * p) / tau;
    C[11] = -(T(2) * Puy + Q[11] - T(2) * uy * p) / tau;
    C[12] = -(T(2) * Puz + Q[12] - T(2) * uz * p) / tau;
    T uPu = ux * Pux + uy * Puy + uz * Puz;
    T uq = ux * Q[10] + uy * Q[11] + uz * Q[12];
    T u2 = ux * ux + uy * uy + uz * uz;
    C[13] = -((T(4) * uPu + T(4) * uq + Q[13]) - (T(4) * u2 * p + T(15) * p * p / rho)) / tau;
}

template <class T>
__device__ __forceinline__ T tau_of(const RelaxParams& rp, const T* Q, int system) {
    if (rp.model == 1) return T(rp.tau_ref);
    T Tt = system == 5 ? Q[2] / Q[0] : (Q[4] + Q[7] + Q[9]) / (T(3) * Q[0]);
    return T(rp.tau_ref) * (T(rp.rho_ref) / Q[0]) * M<T>::sqrt_(T(rp.T_ref) / Tt);
}

// ---------------------------------------------------------------- point-implicit BGK
// Point-implicit source (the closing remark of Sec. 4.3): after an explicit
// stage V = U_base + h (-div F), backward Euler for dU/dt = -(U - U_M)/tau
// over h.  The source keeps density, momentum and energy, so the Maxwellian
// U_M (Sec. 2.3 / 2.4: same density, velocity and pressure) and tau are V's
// and the step is U = U_M + (V - U_M) / (1 + h/tau) for every moment but
// density and momentum.  Conserved form, FP64 (Q = primitives of U, tau
// from Q), each operation rounded on its own as in the plain evaluation.
__device__ __forceinline__ void relax5_cons(double* U, const double* Q, double tau, double h) {
    double QM[5] = {Q[0], Q[1], Q[2], 0.0, 3.0 * Q[2] * Q[2] / Q[0]};
    double UM[5];
    prim2cons5(QM, UM);
    double g = 1.0 / (1.0 + h / tau);
#pragma unroll
    for (int k = 2; k < 5; ++k) U[k] = add_rn(UM[k], mul_rn(g, sub_rn(U[k], UM[k])));
}

__device__ __forceinline__ void relax14_cons(double* U, const double* Q, double tau, double h) {
    double p = (Q[4] + Q[7] + Q[9]) / 3.0;
    double QM[14] = {Q[0], Q[1], Q[2], Q[3], p, 0.0, 0.0, p, 0.0, p, 0.0, 0.0, 0.0,
                     15.0 * p * p / Q[0]};
    double UM[14];
    prim2cons14(QM, UM);
    double g = 1.0 / (1.0 + h / tau);
#pragma unroll
    for (int k = 4; k < 14; ++k) U[k] = add_rn(UM[k], mul_rn(g, sub_rn(U[k], UM[k])));
}

// The same relaxation in primitive form (FP32 mixed path): rho, u and p are
// kept, P <- p I + g (P - p I), q <- g q, R <- R_M + g (R - R_M),
// g = 1 / (1 + h/tau), R_M = 15 p^2 / rho.  N receives U - U_M of the state
// before relaxing, in conserved form: prim2cons is linear in (rho, P, q, R)
// at fixed u, so U - U_M = prim2cons(0, u, P - p I, q, R - R_M), evaluated
// without the cancellation of a difference of conserved vectors.
template <class T>
__device__ __forceinline__ void relax14_prim(T* W, T g, T* N) {
    T p = (W[4] + W[7] + W[9]) / T(3);
    T RM = T(15) * p * p / W[0];
    T D[14] = {T(0), W[1], W[2], W[3], W[4] - p, W[5], W[6], W[7] - p, W[8], W[9] - p,
               W[10], W[11], W[12], W[13] - RM};
    prim2cons14(D, N);
    W[4] = p + g * D[4]; W[5] = g * D[5]; W[6] = g * D[6];
    W[7] = p + g * D[7]; W[8] = g * D[8]; W[9] = p + g * D[9];
    W[10] = g * D[10]; W[11] = g * D[11]; W[12] = g * D[12];
    W[13] = RM + g * D[13];
}

// ---------------------------------------------------------------- limiter
// Shared most-stringent limiter (Sec. 3.2): phi = min_k phi_k with
// phi_k = 1 (flat: |dm| and |dp| both within the field's tolerance, or both
// zero), 0 (dm dp <= 0), min(|dm|,|dp|)/(|dm+dp|/2) (minmod) or
// 2 dm dp/(dm^2 + dp^2) (van Albada).
//
// The flat-field test is a reading (the paper states no tolerance): a
// field that is uniform or zero in exact arithmetic carries round-off from
// the conserved-to-primitive recovery, and letting the random signs of
// those differences zero the shared limiter drops the scheme to first order
// wherever one field is uniform.  Field k is flat when m = max(|dm|, |dp|)
// is within T = 1e-10 times its natural scale at the centre cell (theta =
// p / rho, p the mean pressure): rho; sqrt(theta) (velocities); p (pressure
// tensor); p sqrt(theta) (heat fluxes); p theta (fourth moment).  The
// comparisons are multiplied out so that no division or square root enters,
// with s = P (5-moment) or s = tr P = 3p (14-moment):
//   m <= T rho;  m^2 rho <= T^2 p;  m <= T p;  m^2 rho <= T^2 p^3;  m rho <= T p^2.
// The FP32 primitives of the mixed path take the same test and also count
// a field as flat when m <= 2^-20 |Q_i,k| (8 to 16 FP32 ulps of the centre
// value): in a uniform non-zero field the FP32 flux differences leave a
// random walk of a few ulps in the FP64 state, which the natural-scale bound
// alone would let through.  The factor is the smallest power of two at
// which the mixed path stays second order on a density wave at uniform
// velocity and pressure (2^-21, 2^-22 and 2^-24 measured first order); a
// larger one also treats shallow genuine extrema as flat, which showed as
// error on long near-collisionless runs (2^-16: 1.4e-4 density L1 on the
// 4096-cell Sod tube at Kn = 10 to t = 0.2, against 3.8e-5 with 2^-20).
template <class T>
struct FlatConst;
template <>
struct FlatConst<double> {
    static constexpr double tol = 1e-10;
};
template <>
struct FlatConst<float> {
    static constexpr float tol = 1e-10f;
};
constexpr float FLAT_REL_F32 = 9.5367431640625e-07f;   // 2^-20

// scale class of field k in the 5-field, planar 10-field and general
// 14-field primitive layouts: 0 rho, 1 velocity, 2 pressure tensor,
// 3 heat flux, 4 fourth moment
template <int NF>
__host__ __device__ constexpr int flat_class(int k) {
    return NF == 5 ? k
         : NF == 10 ? (k == 0 ? 0 : k <= 2 ? 1 : k <= 6 ? 2 : k <= 8 ? 3 : 4)
                    : (k == 0 ? 0 : k <= 3 ? 1 : k <= 9 ? 2 : k <= 12 ? 3 : 4);
}

// density and pressure measure s of the stencil's centre cell
template <class T>
struct FlatRef {
    T rho, s;
};

// FlatRef of the primitive cell whose field k sits at w[k * fs]
template <int NF, class T>
__device__ __forceinline__ FlatRef<T> flat_ref(const T* w, int fs) {
    T s;
    if (NF == 5) s = w[2 * fs];
    else if (NF == 10) s = add_rn(add_rn(w[3 * fs], w[5 * fs]), w[6 * fs]);
    else s = add_rn(add_rn(w[4 * fs], w[7 * fs]), w[9 * fs]);
    return FlatRef<T>{w[0], s};
}

// the flat test of field k (compile-time index) with m = max(|dm|, |dp|)
template <int NF, class T>
__device__ __forceinline__ bool field_flat(const FlatRef<T>& f, int k, T m) {
    constexpr T t = FlatConst<T>::tol;
    constexpr T cp = NF == 5 ? t : t / T(3);
    constexpr T cv = NF == 5 ? t * t : t * t / T(3);
    constexpr T ch = NF == 5 ? t * t : t * t / T(27);
    constexpr T cr = NF == 5 ? t : t / T(9);
    switch (flat_class<NF>(k)) {
    case 0: return m <= mul_rn(t, f.rho);
    case 1: return mul_rn(mul_rn(m, m), f.rho) <= mul_rn(cv, f.s);
    case 2: return m <= mul_rn(cp, f.s);
    case 3: return mul_rn(mul_rn(m, m), f.rho) <= mul_rn(mul_rn(mul_rn(ch, f.s), f.s), f.s);
    default: return mul_rn(m, f.rho) <= mul_rn(mul_rn(cr, f.s), f.s);
    }
}

template <class T>
__device__ __forceinline__ T abs_max(T a, T b) {
    return fmax(fabs(a), fabs(b));
}

// phi_k without the flat-field test (1 only when dm = dp = 0)
template <class T>
__device__ __forceinline__ T phi_field(T dm, T dp, int lim) {
    if (mul_rn(dm, dp) > T(0)) {
        if (lim == 1)
            return mul_rn(mul_rn(T(2), dm), dp) / add_rn(mul_rn(dm, dm), mul_rn(dp, dp));
        T am = fabs(dm), ap = fabs(dp);
        T mn = am < ap ? am : ap;
        return mn / mul_rn(T(0.5), add_rn(am, ap));
    }
    return (dm == T(0) && dp == T(0)) ? T(1) : T(0);
}

// phi = min(phi, phi_k) for field k (compile-time index) of the stencil
// centred on the cell fr.  A flat field has phi_k = 1, which never lowers
// phi, so the flat test runs only where phi_k without it would: the result
// is the min over all fields either way.
template <int NF, class T>
__device__ __forceinline__ void phi_accumulate(T& phi, T dm, T dp, int lim, const FlatRef<T>& fr,
                                               int k) {
    const T pk = phi_field(dm, dp, lim);
    if (pk < phi && !field_flat<NF>(fr, k, abs_max(dm, dp))) phi = pk;
}

// MUSCL face value Q0 + sgn/2 (phi c) with the central difference
// c = ((Q0 - Qm) + (Qp - Q0))/2, explicitly rounded.
template <class T>
__device__ __forceinline__ T muscl_face(T qm, T q0, T qp, T phi, T half_sgn) {
    T cen = mul_rn(T(0.5), add_rn(sub_rn(q0, qm), sub_rn(qp, q0)));
    return add_rn(q0, mul_rn(half_sgn, mul_rn(phi, cen)));
}

}  // namespace mxe
