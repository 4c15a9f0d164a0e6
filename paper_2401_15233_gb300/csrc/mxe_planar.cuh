// mxe_planar.cuh -- 14-moment point physics for planar states.
//
// When the state and every boundary state are mirror-symmetric in z (all
// of u_z, P_xz, P_yz, q_z exactly zero) the 14-moment system keeps them zero
// for all time: their fluxes and sources are odd in z.  The 2D crossed jets
// are such a flow.  The functions below evaluate the same method on the ten
// remaining moments with the pressure tensor block-diagonal (2x2 in x-y
// plus P_zz):
//   compact primitives  (rho, ux, uy, Pxx, Pxy, Pyy, Pzz, qx, qy, R)
//   compact conserved   (rho, rho ux, rho uy, Exx, Exy, Eyy, Ezz, Hx, Hy, E4)
// Every formula is the general one (Sec. 2.4 closure, Sec. 5 wave speeds)
// with the vanishing terms removed; K is the flux direction (0 = x, 1 = y)
// and O the other in-plane direction.
#pragma once
#include "mxe_physics.cuh"

namespace mxe {

constexpr int NP = 10;
// position of each compact field in the 14-field layout
__host__ __device__ constexpr int planar_field(int k) {
    return k < 3 ? k : (k == 3 ? 4 : (k == 4 ? 5 : (k == 5 ? 7 : (k == 6 ? 9 : (k == 7 ? 10 : (k == 8 ? 11 : 13))))));
}

template <class T>
__device__ __forceinline__ void prim2cons_p(const T* Q, T* U) {
    T rho = Q[0], ux = Q[1], uy = Q[2];
    T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    T u2 = ux * ux + uy * uy;
    T trP = Pxx + Pyy + Pzz;
    T Pux = Pxx * ux + Pxy * uy;
    T Puy = Pxy * ux + Pyy * uy;
    T uPu = ux * Pux + uy * Puy;
    T uq = ux * Q[7] + uy * Q[8];
    T e = rho * u2 + trP;
    U[0] = rho;
    U[1] = rho * ux; U[2] = rho * uy;
    U[3] = rho * ux * ux + Pxx; U[4] = rho * ux * uy + Pxy; U[5] = rho * uy * uy + Pyy;
    U[6] = Pzz;
    U[7] = ux * e + T(2) * Pux + Q[7];
    U[8] = uy * e + T(2) * Puy + Q[8];
    U[9] = rho * u2 * u2 + T(2) * u2 * trP + T(4) * uPu + T(4) * uq + Q[9];
}

// Primitive recovery with one reciprocal of rho and contractible arithmetic
// (the FP64 re-sync of the mixed path, whose result is rounded to FP32; each
// cancelling difference E - m u is one fused operation).
template <class T>
__device__ __forceinline__ void cons2prim_p(const T* U, T* Q) {
    T rho = U[0];
    T ir = T(1) / rho;
    T ux = U[1] * ir, uy = U[2] * ir;
    T Pxx = U[3] - U[1] * ux, Pxy = U[4] - U[1] * uy, Pyy = U[5] - U[2] * uy, Pzz = U[6];
    T u2 = ux * ux + uy * uy;
    T trP = Pxx + Pyy + Pzz;
    T uPx = ux * Pxx + uy * Pxy, uPy = ux * Pxy + uy * Pyy;
    T uPu = ux * uPx + uy * uPy;
    T e = rho * u2 + trP;
    T qx = U[7] - ux * e - T(2) * uPx;
    T qy = U[8] - uy * e - T(2) * uPy;
    T uq = ux * qx + uy * qy;
    Q[0] = rho; Q[1] = ux; Q[2] = uy; Q[3] = Pxx; Q[4] = Pxy; Q[5] = Pyy; Q[6] = Pzz;
    Q[7] = qx; Q[8] = qy;
    Q[9] = U[9] - rho * u2 * u2 - T(2) * u2 * trP - T(4) * uPu - T(4) * uq;
}

// FP64 primitive recovery rounded exactly like the general evaluation order
// (the vanishing terms it adds are exact zeros).
__device__ __forceinline__ void cons2prim_p_rn(const double* U, double* Q) {
    double rho = U[0];
    double ux = U[1] / rho, uy = U[2] / rho;
    double Pxx = sub_rn(U[3], mul_rn(mul_rn(rho, ux), ux));
    double Pxy = sub_rn(U[4], mul_rn(mul_rn(rho, ux), uy));
    double Pyy = sub_rn(U[5], mul_rn(mul_rn(rho, uy), uy));
    double Pzz = U[6];
    double u2 = add_rn(mul_rn(ux, ux), mul_rn(uy, uy));
    double trP = add_rn(add_rn(Pxx, Pyy), Pzz);
    double uPu = mul_rn(mul_rn(ux, ux), Pxx);
    uPu = add_rn(uPu, mul_rn(mul_rn(ux, uy), Pxy));
    uPu = add_rn(uPu, mul_rn(mul_rn(uy, ux), Pxy));
    uPu = add_rn(uPu, mul_rn(mul_rn(uy, uy), Pyy));
    double uPx = add_rn(mul_rn(ux, Pxx), mul_rn(uy, Pxy));
    double uPy = add_rn(mul_rn(ux, Pxy), mul_rn(uy, Pyy));
    double qx = sub_rn(sub_rn(sub_rn(U[7], mul_rn(mul_rn(rho, ux), u2)), mul_rn(ux, trP)),
                       mul_rn(2.0, uPx));
    double qy = sub_rn(sub_rn(sub_rn(U[8], mul_rn(mul_rn(rho, uy), u2)), mul_rn(uy, trP)),
                       mul_rn(2.0, uPy));
    double uq = add_rn(mul_rn(ux, qx), mul_rn(uy, qy));
    double R = sub_rn(sub_rn(sub_rn(sub_rn(U[9], mul_rn(mul_rn(rho, u2), u2)),
                                    mul_rn(mul_rn(2.0, u2), trP)),
                             mul_rn(4.0, uPu)),
                      mul_rn(4.0, uq));
    Q[0] = rho; Q[1] = ux; Q[2] = uy; Q[3] = Pxx; Q[4] = Pxy; Q[5] = Pyy; Q[6] = Pzz;
    Q[7] = qx; Q[8] = qy; Q[9] = R;
}

template <class T>
struct DimlessP {
    T th, sq;
    T a, b, d, f;          // P* = [[a b 0][b d 0][0 0 f]]
    T qx, qy;              // q*
    T trPs, T2;
    T ia, ib, id, ifz;     // P*^-1 (2x2 block + zz)
    T yx, yy;              // P*^-1 q*
    T sig, det;
};

template <class T>
__device__ __forceinline__ void dimless_p(const T* Q, DimlessP<T>& g) {
    T rho = Q[0];
    T p = (Q[3] + Q[5] + Q[6]) / T(3);
    T ip = T(1) / p;
    g.th = p / rho;
    g.sq = M<T>::sqrt_(g.th);
    T isc3 = T(1) / (rho * g.th * g.sq);
    g.a = Q[3] * ip; g.b = Q[4] * ip; g.d = Q[5] * ip; g.f = Q[6] * ip;
    g.qx = Q[7] * isc3; g.qy = Q[8] * isc3;
    T Rs = Q[9] / (rho * g.th * g.th);
    g.trPs = g.a + g.d + g.f;
    g.T2 = g.a * g.a + g.d * g.d + g.f * g.f + T(2) * (g.b * g.b);
    T det2 = g.a * g.d - g.b * g.b;
    T i2 = T(1) / det2;
    g.ia = g.d * i2; g.ib = -g.b * i2; g.id = g.a * i2;
    g.ifz = T(1) / g.f;
    g.det = det2 * g.f;
    g.yx = g.ia * g.qx + g.ib * g.qy;
    g.yy = g.ib * g.qx + g.id * g.qy;
    T qPq = g.qx * g.yx + g.qy * g.yy;
    T A = T(2) * g.T2 + g.trPs * g.trPs - Rs;
    T X = T(8) * g.T2 * qPq;
    g.sig = sigma_root(A, X, g.T2);
}

// Eq. (14mom-approx-ws-equations) along K with q_perp = |q*_O|.
template <class T, int K>
__device__ __forceinline__ void lam_p(const DimlessP<T>& g, T sb, T& lp, T& lm) {
    T Pkk = K == 0 ? g.a : g.d;
    T qd = K == 0 ? g.qx : g.qy;
    T qperp = fabs(K == 0 ? g.qy : g.qx);
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

// Closure slice along K (dimensional): QK = (Q_KKK, Q_KKO, Q_KOO, Q_Kzz),
// RK = (R_KKjj, R_OKjj), SK = S_Kiijj.
template <class T, int K>
__device__ __forceinline__ void closure_p(const T* Q, const DimlessP<T>& g, T sb, T* QK, T* RK,
                                          T& SK) {
    const T a = g.a, b = g.b, d = g.d, f = g.f;
    T P2xx = a * a + b * b, P2xy = b * (a + d), P2yy = b * b + d * d, P2zz = f * f;
    T P3xx = P2xx * a + P2xy * b, P3xy = P2xx * b + P2xy * d, P3yy = P2xy * b + P2yy * d;
    T P3zz = P2zz * f;
    T trP3 = P3xx + P3yy + P3zz;
    T Bxx = T(2) * a * g.T2 + T(4) * P3xx;
    T Bxy = T(2) * b * g.T2 + T(4) * P3xy;
    T Byy = T(2) * d * g.T2 + T(4) * P3yy;
    T iB = T(1) / (Bxx * Byy - Bxy * Bxy);
    T vx = (Byy * g.qx - Bxy * g.qy) * iB;
    T vy = (Bxx * g.qy - Bxy * g.qx) * iB;
    T wx = a * vx + b * vy, wy = b * vx + d * vy;
    // in-plane components along K and O
    T wK = K == 0 ? wx : wy, wO = K == 0 ? wy : wx;
    T vK = K == 0 ? vx : vy, vO = K == 0 ? vy : vx;
    T yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    T P2KK = K == 0 ? P2xx : P2yy, P2OO = K == 0 ? P2yy : P2xx;
    T P3KK = K == 0 ? P3xx : P3yy;
    T PKK = K == 0 ? a : d;
    T qK = K == 0 ? g.qx : g.qy;
    T QKKK = T(6) * wK * P2KK;
    T QKKO = T(4) * wK * P2xy + T(2) * wO * P2KK;
    T QKOO = T(2) * wK * P2OO + T(4) * wO * P2xy;
    T QKzz = T(2) * wK * P2zz;
    T isb = T(1) / sb;
    T RKK = (QKKK * yK + QKKO * yO) * isb + T(2) * (T(1) - sb) * P2KK + PKK * g.trPs;
    T ROK = (QKKO * yK + QKOO * yO) * isb + T(2) * (T(1) - sb) * P2xy + b * g.trPs;
    T yQy = QKKK * yK * yK + T(2) * QKKO * yK * yO + QKOO * yO * yO;
    T t = g.trPs, t2 = t * t;
    T c1 = T(2) * t2 * t + T(12) * trP3 - T(2) * g.T2 * t;
    T c2 = T(14) * g.T2 - T(6) * t2;
    T c3 = T(20) * t;
    // row K of the W bracket against v (P^4 = P^2 P^2)
    T P4KK = P2KK * P2KK + P2xy * P2xy;
    T P4KO = P2xy * (P2xx + P2yy);
    T mKK = c1 * PKK + c2 * P2KK + c3 * P3KK + T(20) * P4KK;
    T mKO = c1 * b + c2 * P2xy + c3 * P3xy + T(20) * P4KO;
    T Wq = mKK * vK + mKO * vO;
    T ssb = M<T>::sqrt_(sb);
    T Ss = yQy * isb * isb + T(2) * ssb * t * qK + (T(1) - ssb) * Wq;
    T rho = Q[0];
    T sc3 = rho * g.th * g.sq, sc4 = rho * g.th * g.th, sc5 = sc4 * g.sq;
    QK[0] = QKKK * sc3; QK[1] = QKKO * sc3; QK[2] = QKOO * sc3; QK[3] = QKzz * sc3;
    RK[0] = RKK * sc4; RK[1] = ROK * sc4;
    SK = Ss * sc5;
}

// K-flux of the compact system: u_K U + central part.
template <class T, int K>
__device__ __forceinline__ void flux_p(const T* Q, const T* U, const T* QK, const T* RK, T SK,
                                       T* F) {
    T ux = Q[1], uy = Q[2];
    T uK = K == 0 ? ux : uy, uO = K == 0 ? uy : ux;
    T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5];
    T PKK = K == 0 ? Pxx : Pyy, POO = K == 0 ? Pyy : Pxx;
    T qK = Q[7 + K];
    T u2 = ux * ux + uy * uy;
    T PuK = PKK * uK + Pxy * uO;                  // (P u)_K
    // (Q_K u)_a for a = K, O: Q_Kab u_b
    T QuK = QK[0] * uK + QK[1] * uO;
    T QuO = QK[1] * uK + QK[2] * uO;
#pragma unroll
    for (int n = 0; n < NP; ++n) F[n] = uK * U[n];
    // momentum
    F[1] += K == 0 ? Pxx : Pxy;
    F[2] += K == 0 ? Pxy : Pyy;
    // second moments: u_i P_jK + u_j P_iK + Q_ijK
    T PxK = K == 0 ? Pxx : Pxy, PyK = K == 0 ? Pxy : Pyy;
    T QxxK = K == 0 ? QK[0] : QK[2];              // Q_xxK
    T QxyK = QK[1];                               // Q_xyK = Q_KKO for both K
    T QyyK = K == 0 ? QK[2] : QK[0];
    F[3] += T(2) * ux * PxK + QxxK;
    F[4] += ux * PyK + uy * PxK + QxyK;
    F[5] += T(2) * uy * PyK + QyyK;
    F[6] += QK[3];
    // third moments: u_i (2 (Pu)_K + q_K) + |u|^2 P_iK + 2 (Q_K u)_i + R_iK
    T gK = T(2) * PuK + qK;
    T QuX = K == 0 ? QuK : QuO, QuY = K == 0 ? QuO : QuK;
    T RxK = K == 0 ? RK[0] : RK[1], RyK = K == 0 ? RK[1] : RK[0];
    F[7] += ux * gK + u2 * PxK + T(2) * QuX + RxK;
    F[8] += uy * gK + u2 * PyK + T(2) * QuY + RyK;
    T uQu = uK * QuK + uO * QuO;
    T uR = uK * RK[0] + uO * RK[1];
    F[9] += T(4) * u2 * PuK + T(2) * u2 * qK + T(4) * uQu + T(4) * uR + SK;
}

template <class T, int K>
__device__ __forceinline__ void face_eval_p(const T* Q, T sigma_lim, T k_ws, T* U, T* F, T& lmin,
                                            T& lmax) {
    DimlessP<T> g;
    dimless_p(Q, g);
    T sb = clamp_sigma(g.sig, sigma_lim);
    T QK[4], RK[2], SK;
    closure_p<T, K>(Q, g, sb, QK, RK, SK);
    prim2cons_p(Q, U);
    flux_p<T, K>(Q, U, QK, RK, SK, F);
    T lp, lm;
    lam_p<T, K>(g, sb, lp, lm);
    lmax = Q[1 + K] + k_ws * lp * g.sq;
    lmin = Q[1 + K] + k_ws * lm * g.sq;
}

// The same, also returning the raw sigma and det P* of the state.
template <class T, int K>
__device__ __forceinline__ void face_eval_p(const T* Q, T sigma_lim, T k_ws, T* U, T* F, T& lmin,
                                            T& lmax, T& sig, T& det) {
    DimlessP<T> g;
    dimless_p(Q, g);
    T sb = clamp_sigma(g.sig, sigma_lim);
    T QK[4], RK[2], SK;
    closure_p<T, K>(Q, g, sb, QK, RK, SK);
    prim2cons_p(Q, U);
    flux_p<T, K>(Q, U, QK, RK, SK, F);
    T lp, lm;
    lam_p<T, K>(g, sb, lp, lm);
    lmax = Q[1 + K] + k_ws * lp * g.sq;
    lmin = Q[1 + K] + k_ws * lm * g.sq;
    sig = g.sig;
    det = g.det;
}

template <class T, int K>
__device__ __forceinline__ T amax_p(const T* Q, const DimlessP<T>& g, T sigma_lim, T k_ws) {
    T sb = clamp_sigma(g.sig, sigma_lim);
    T lp, lm;
    lam_p<T, K>(g, sb, lp, lm);
    T lmax = Q[1 + K] + k_ws * lp * g.sq;
    T lmin = Q[1 + K] + k_ws * lm * g.sq;
    T x = fabs(lmin), y = fabs(lmax);
    return x > y ? x : y;
}

template <class T>
__device__ __forceinline__ void source_p(const T* Q, T tau, T* C) {
    T rho = Q[0], ux = Q[1], uy = Q[2];
    T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    T p = (Pxx + Pyy + Pzz) / T(3);
    C[0] = T(0); C[1] = T(0); C[2] = T(0);
    C[3] = -(Pxx - p) / tau; C[4] = -Pxy / tau; C[5] = -(Pyy - p) / tau; C[6] = -(Pzz - p) / tau;
    T Pux = Pxx * ux + Pxy * uy;
    T Puy = Pxy * ux + Pyy * uy;
    C[7] = -(T(2) * Pux + Q[7] - T(2) * ux * p) / tau;
    C[8] = -(T(2) * Puy + Q[8] - T(2) * uy * p) / tau;
    T uPu = ux * Pux + uy * Puy;
    T uq = ux * Q[7] + uy * Q[8];
    T u2 = ux * ux + uy * uy;
    C[9] = -((T(4) * uPu + T(4) * uq + Q[9]) - (T(4) * u2 * p + T(15) * p * p / rho)) / tau;
}

template <class T>
__device__ __forceinline__ T tau_p(int model, T tau_ref, T rho_ref, T T_ref, const T* Q) {
    if (model == 1) return tau_ref;
    T Tt = (Q[3] + Q[5] + Q[6]) / (T(3) * Q[0]);
    return tau_ref * (rho_ref / Q[0]) * M<T>::sqrt_(T_ref / Tt);
}

// Point-implicit relaxation (see relax14_cons / relax14_prim) of the
// compact state: the Maxwellian is (rho, ux, uy, p, 0, p, p, 0, 0, 15 p^2/rho).
__device__ __forceinline__ void relax_p_cons(double* U, const double* Q, double tau, double h) {
    double p = (Q[3] + Q[5] + Q[6]) / 3.0;
    double QM[NP] = {Q[0], Q[1], Q[2], p, 0.0, p, p, 0.0, 0.0, 15.0 * p * p / Q[0]};
    double UM[NP];
    prim2cons_p(QM, UM);
    double g = 1.0 / (1.0 + h / tau);
#pragma unroll
    for (int k = 3; k < NP; ++k) U[k] = add_rn(UM[k], mul_rn(g, sub_rn(U[k], UM[k])));
}

template <class T>
__device__ __forceinline__ void relax_p_prim(T* W, T g, T* N) {
    T p = (W[3] + W[5] + W[6]) / T(3);
    T RM = T(15) * p * p / W[0];
    T D[NP] = {T(0), W[1], W[2], W[3] - p, W[4], W[5] - p, W[6] - p, W[7], W[8], W[9] - RM};
    prim2cons_p(D, N);
    W[3] = p + g * D[3]; W[4] = g * D[4]; W[5] = p + g * D[5]; W[6] = p + g * D[6];
    W[7] = g * D[7]; W[8] = g * D[8];
    W[9] = RM + g * D[9];
}

// Primitive moments of cons(W) + dU from the increment (see
// prim_increment14): every term scales with the increment.
__device__ __forceinline__ void prim_increment_p(const float* W, const float* dU, float* Wn) {
    float rho = W[0], ux = W[1], uy = W[2];
    float Pxx = W[3], Pxy = W[4], Pyy = W[5], Pzz = W[6];
    float drho = dU[0];
    float rho1 = rho + drho;
    float ir1 = 1.0f / rho1;
    float dux = (dU[1] - ux * drho) * ir1, duy = (dU[2] - uy * drho) * ir1;
    float ux1 = ux + dux, uy1 = uy + duy;
    float dPxx = dU[3] - drho * ux * ux - rho1 * (2.0f * ux * dux + dux * dux);
    float dPxy = dU[4] - drho * ux * uy - rho1 * (ux * duy + dux * uy + dux * duy);
    float dPyy = dU[5] - drho * uy * uy - rho1 * (2.0f * uy * duy + duy * duy);
    float dPzz = dU[6];
    float Pxx1 = Pxx + dPxx, Pxy1 = Pxy + dPxy, Pyy1 = Pyy + dPyy, Pzz1 = Pzz + dPzz;
    float trP1 = Pxx1 + Pyy1 + Pzz1;
    float dtr = dPxx + dPyy + dPzz;
    float u2 = ux * ux + uy * uy;
    float s = 2.0f * (ux * dux + uy * duy) + (dux * dux + duy * duy);
    float Pdux = Pxx * dux + Pxy * duy, Pduy = Pxy * dux + Pyy * duy;
    float dPu1x = dPxx * ux1 + dPxy * uy1, dPu1y = dPxy * ux1 + dPyy * uy1;
    float Pux = Pxx * ux + Pxy * uy, Puy = Pxy * ux + Pyy * uy;
    float dGx = drho * ux * u2 + rho1 * (dux * u2 + ux1 * s) + dux * trP1 + ux * dtr
              + 2.0f * (dPu1x + Pdux);
    float dGy = drho * uy * u2 + rho1 * (duy * u2 + uy1 * s) + duy * trP1 + uy * dtr
              + 2.0f * (dPu1y + Pduy);
    float dqx = dU[7] - dGx, dqy = dU[8] - dGy;
    float qx1 = W[7] + dqx, qy1 = W[8] + dqy;
    float u1dPu1 = ux1 * dPu1x + uy1 * dPu1y;
    float duPu = dux * Pux + duy * Puy;
    float duPdu = dux * Pdux + duy * Pduy;
    float dK = drho * u2 * u2 + rho1 * s * (2.0f * u2 + s) + 2.0f * (s * trP1 + u2 * dtr)
             + 4.0f * (u1dPu1 + 2.0f * duPu + duPdu)
             + 4.0f * (dux * qx1 + duy * qy1 + ux * dqx + uy * dqy);
    Wn[0] = rho1; Wn[1] = ux1; Wn[2] = uy1;
    Wn[3] = Pxx1; Wn[4] = Pxy1; Wn[5] = Pyy1; Wn[6] = Pzz1;
    Wn[7] = qx1; Wn[8] = qy1;
    Wn[9] = W[9] + (dU[9] - dK);
}

}  // namespace mxe
