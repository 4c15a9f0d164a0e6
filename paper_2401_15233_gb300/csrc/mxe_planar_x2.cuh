// mxe_planar_x2.cuh -- the planar 14-moment face-state evaluation of
// mxe_planar.cuh for two face states at once, in packed FP32 (f32x2).
//
// Both face states of a face (left in lane x, right in lane y) go through
// the same closure, flux and wave-speed arithmetic.  GB300 issues one
// packed FFMA2/FADD2/FMUL2 for two FP32 operations at the FP32 pipe's full
// rate, so an issue-bound stage kernel executes about half the FP32
// arithmetic instructions for the pair.  Transcendentals, divisions,
// comparisons and selects stay per lane.  The formulas are those of
// dimless_p / closure_p / prim2cons_p / flux_p / lam_p (Sec. 2.4 closure,
// Eqs. closure-14mom-Qijk/Rijkk/Sijjkk; Sec. 5 wave speeds, Eq.
// 14mom-approx-ws-equations), regrouped into fused multiply-adds; the
// results agree with the scalar FP32 path to FP32 rounding.
#pragma once
#include "mxe_planar.cuh"

namespace mxe {
namespace x2 {

using v2 = float2;

__device__ __forceinline__ v2 S(float a) { return make_float2(a, a); }
__device__ __forceinline__ v2 add(v2 a, v2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ v2 mul(v2 a, v2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ v2 fma(v2 a, v2 b, v2 c) { return __ffma2_rn(a, b, c); }
// a - b
__device__ __forceinline__ v2 sub(v2 a, v2 b) { return __ffma2_rn(b, S(-1.0f), a); }
__device__ __forceinline__ v2 neg(v2 a) { return __fmul2_rn(a, S(-1.0f)); }

// per-lane operations (no packed form)
__device__ __forceinline__ v2 rcp(v2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
__device__ __forceinline__ v2 sqrt_(v2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
__device__ __forceinline__ v2 rsqrt_(v2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ v2 ex2(v2 a) { return make_float2(exp2f(a.x), exp2f(a.y)); }
__device__ __forceinline__ v2 lg2(v2 a) { return make_float2(__log2f(a.x), __log2f(a.y)); }
__device__ __forceinline__ v2 abs_(v2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ v2 div_(v2 a, v2 b) {
    return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}

constexpr float LOG2E = 1.4426950408889634f;

// Dimensionless state (scaled by p = tr P / 3, Sec. 3.3) of two face states.
struct DimX2 {
    v2 tr, p, th, sq;       // tr P, p = tr P / 3, theta = p / rho, sqrt theta
    v2 a, b, d, f;          // P* = [[a b 0][b d 0][0 0 f]]
    v2 bb;                  // b^2
    v2 qx, qy;              // q*
    v2 trPs, T2;
    v2 yx, yy;              // P*^-1 q* (in-plane)
    v2 sig, det;
};

// sigma = [A + sqrt(A^2 + X)] / (4 T), rationalised for A < 0.
__device__ __forceinline__ v2 sigma_root_x2(v2 A, v2 X, v2 T2) {
    v2 rt = sqrt_(fma(A, A, X));
    v2 fT = mul(T2, S(4.0f));
    v2 s1 = add(A, rt);                // A >= 0
    v2 dn = mul(fT, sub(rt, A));       // A < 0
    return div_(make_float2(A.x >= 0.0f ? s1.x : X.x, A.y >= 0.0f ? s1.y : X.y),
                make_float2(A.x >= 0.0f ? fT.x : dn.x, A.y >= 0.0f ? fT.y : dn.y));
}

__device__ __forceinline__ void dimless_x2(const v2* Q, DimX2& g) {
    v2 rho = Q[0];
    g.tr = add(add(Q[3], Q[5]), Q[6]);
    g.p = mul(g.tr, S(1.0f / 3.0f));
    v2 ip = rcp(g.p), ir = rcp(rho);
    g.th = mul(g.p, ir);
    v2 rsq = rsqrt_(g.th);
    g.sq = mul(g.th, rsq);
    v2 isc3 = mul(ip, rsq);                           // 1 / (rho th sqrt th)
    g.a = mul(Q[3], ip); g.b = mul(Q[4], ip); g.d = mul(Q[5], ip); g.f = mul(Q[6], ip);
    g.qx = mul(Q[7], isc3); g.qy = mul(Q[8], isc3);
    v2 nRs = mul(mul(Q[9], neg(rho)), mul(ip, ip));   // -R / (rho th^2)
    g.trPs = add(add(g.a, g.d), g.f);
    g.bb = mul(g.b, g.b);
    g.T2 = fma(g.a, g.a, fma(g.d, g.d, fma(g.f, g.f, add(g.bb, g.bb))));
    v2 det2 = fma(g.a, g.d, neg(g.bb));
    v2 i2 = rcp(det2);
    v2 ia = mul(g.d, i2), ib = mul(neg(g.b), i2), id = mul(g.a, i2);
    g.det = mul(det2, g.f);
    g.yx = fma(ia, g.qx, mul(ib, g.qy));
    g.yy = fma(ib, g.qx, mul(id, g.qy));
    v2 qPq = fma(g.qx, g.yx, mul(g.qy, g.yy));
    v2 A = fma(g.trPs, g.trPs, fma(g.T2, S(2.0f), nRs));
    v2 X = mul(mul(g.T2, S(8.0f)), qPq);
    g.sig = sigma_root_x2(A, X, g.T2);
}

__device__ __forceinline__ v2 clamp_sigma_x2(v2 s, float slim) {
    return make_float2(fminf(fmaxf(s.x, slim), 1.0f), fminf(fmaxf(s.y, slim), 1.0f));
}

// Closure slice along K (dimensional): QK = (Q_KKK, Q_KKO, Q_KOO, Q_Kzz),
// RK = (R_KKjj, R_OKjj), SK = S_Kiijj (see closure_p).
template <int K>
__device__ __forceinline__ void closure_x2(const DimX2& g, v2 sb, v2 isb, v2 ssb, v2* QK, v2* RK,
                                           v2& SK) {
    const v2 a = g.a, b = g.b, d = g.d, f = g.f;
    v2 P2xx = fma(a, a, g.bb), P2xy = mul(b, add(a, d)), P2yy = fma(d, d, g.bb), P2zz = mul(f, f);
    v2 P3xx = fma(P2xx, a, mul(P2xy, b)), P3xy = fma(P2xx, b, mul(P2xy, d));
    v2 P3yy = fma(P2xy, b, mul(P2yy, d));
    v2 trP3 = fma(P2zz, f, add(P3xx, P3yy));
    v2 T2x2 = add(g.T2, g.T2);
    v2 Bxx = fma(a, T2x2, mul(P3xx, S(4.0f)));
    v2 Bxy = fma(b, T2x2, mul(P3xy, S(4.0f)));
    v2 Byy = fma(d, T2x2, mul(P3yy, S(4.0f)));
    v2 nBxy = neg(Bxy);
    v2 iB = rcp(fma(Bxy, nBxy, mul(Bxx, Byy)));
    v2 vx = mul(fma(Byy, g.qx, mul(nBxy, g.qy)), iB);
    v2 vy = mul(fma(Bxx, g.qy, mul(nBxy, g.qx)), iB);
    v2 wx = fma(a, vx, mul(b, vy)), wy = fma(b, vx, mul(d, vy));
    const v2 wK = K == 0 ? wx : wy, wO = K == 0 ? wy : wx;
    const v2 vK = K == 0 ? vx : vy, vO = K == 0 ? vy : vx;
    const v2 yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    const v2 P2KK = K == 0 ? P2xx : P2yy, P2OO = K == 0 ? P2yy : P2xx;
    const v2 P3KK = K == 0 ? P3xx : P3yy, P3KO = P3xy;
    const v2 PKK = K == 0 ? a : d;
    const v2 qK = K == 0 ? g.qx : g.qy;
    v2 w2K = add(wK, wK), w2O = add(wO, wO);
    v2 QKKK = mul(mul(wK, P2KK), S(6.0f));
    v2 QKKO = mul(fma(w2K, P2xy, mul(wO, P2KK)), S(2.0f));
    v2 QKOO = mul(fma(wK, P2OO, mul(w2O, P2xy)), S(2.0f));
    v2 QKzz = mul(w2K, P2zz);
    v2 omsb2 = fma(sb, S(-2.0f), S(2.0f));           // 2 (1 - sigma)
    v2 t1 = fma(QKKK, yK, mul(QKKO, yO));
    v2 t2 = fma(QKKO, yK, mul(QKOO, yO));
    v2 RKK = fma(t1, isb, fma(omsb2, P2KK, mul(PKK, g.trPs)));
    v2 ROK = fma(t2, isb, fma(omsb2, P2xy, mul(b, g.trPs)));
    v2 yQy = fma(yK, t1, mul(yO, t2));
    v2 t = g.trPs, tt = mul(t, t);
    v2 c1 = fma(add(t, t), sub(tt, g.T2), mul(trP3, S(12.0f)));
    v2 c2 = fma(g.T2, S(14.0f), mul(tt, S(-6.0f)));
    v2 c3 = mul(t, S(20.0f));
    v2 P4KK = fma(P2KK, P2KK, mul(P2xy, P2xy));
    v2 P4KO = mul(P2xy, add(P2xx, P2yy));
    v2 mKK = fma(c1, PKK, fma(c2, P2KK, fma(c3, P3KK, mul(P4KK, S(20.0f)))));
    v2 mKO = fma(c1, b, fma(c2, P2xy, fma(c3, P3KO, mul(P4KO, S(20.0f)))));
    v2 Wq = fma(mKK, vK, mul(mKO, vO));
    v2 Ss = fma(yQy, mul(isb, isb), fma(add(ssb, ssb), mul(t, qK), mul(sub(S(1.0f), ssb), Wq)));
    v2 sc3 = mul(g.p, g.sq), sc4 = mul(g.p, g.th);
    v2 sc5 = mul(sc4, g.sq);
    QK[0] = mul(QKKK, sc3); QK[1] = mul(QKKO, sc3); QK[2] = mul(QKOO, sc3); QK[3] = mul(QKzz, sc3);
    RK[0] = mul(RKK, sc4); RK[1] = mul(ROK, sc4);
    SK = mul(Ss, sc5);
}

// Conserved face state of the compact primitives; also returns |u|^2, P u.
__device__ __forceinline__ void prim2cons_x2(const v2* Q, v2 trP, v2* U, v2& u2, v2& Pux,
                                             v2& Puy) {
    v2 rho = Q[0], ux = Q[1], uy = Q[2];
    v2 Pxx = Q[3], Pxy = Q[4], Pyy = Q[5];
    u2 = fma(ux, ux, mul(uy, uy));
    Pux = fma(Pxx, ux, mul(Pxy, uy));
    Puy = fma(Pxy, ux, mul(Pyy, uy));
    v2 uPu = fma(ux, Pux, mul(uy, Puy));
    v2 uq = fma(ux, Q[7], mul(uy, Q[8]));
    v2 e = fma(rho, u2, trP);
    U[0] = rho;
    U[1] = mul(rho, ux); U[2] = mul(rho, uy);
    U[3] = fma(U[1], ux, Pxx); U[4] = fma(U[1], uy, Pxy); U[5] = fma(U[2], uy, Pyy);
    U[6] = Q[6];
    U[7] = fma(ux, e, fma(Pux, S(2.0f), Q[7]));
    U[8] = fma(uy, e, fma(Puy, S(2.0f), Q[8]));
    U[9] = fma(mul(rho, u2), u2, fma(add(u2, u2), trP, fma(add(uPu, uq), S(4.0f), Q[9])));
}

// K-flux of the compact system, u_K U + central part (see flux_p).
template <int K>
__device__ __forceinline__ void flux_x2(const v2* Q, const v2* U, v2 u2, v2 Pux, v2 Puy,
                                        const v2* QK, const v2* RK, v2 SK, v2* F) {
    const v2 ux = Q[1], uy = Q[2];
    const v2 uK = K == 0 ? ux : uy, uO = K == 0 ? uy : ux;
    const v2 Pxy = Q[4];
    const v2 PxK = K == 0 ? Q[3] : Pxy, PyK = K == 0 ? Pxy : Q[5];
    const v2 qK = Q[7 + K];
    const v2 PuK = K == 0 ? Pux : Puy;
    v2 QuK = fma(QK[0], uK, mul(QK[1], uO));
    v2 QuO = fma(QK[1], uK, mul(QK[2], uO));
    const v2 QxxK = K == 0 ? QK[0] : QK[2];
    const v2 QxyK = QK[1];
    const v2 QyyK = K == 0 ? QK[2] : QK[0];
    F[0] = mul(uK, U[0]);
    F[1] = fma(uK, U[1], PxK);
    F[2] = fma(uK, U[2], PyK);
    F[3] = fma(uK, U[3], fma(add(ux, ux), PxK, QxxK));
    F[4] = fma(uK, U[4], fma(ux, PyK, fma(uy, PxK, QxyK)));
    F[5] = fma(uK, U[5], fma(add(uy, uy), PyK, QyyK));
    F[6] = fma(uK, U[6], QK[3]);
    v2 gK = fma(PuK, S(2.0f), qK);
    const v2 QuX = K == 0 ? QuK : QuO, QuY = K == 0 ? QuO : QuK;
    const v2 RxK = K == 0 ? RK[0] : RK[1], RyK = K == 0 ? RK[1] : RK[0];
    F[7] = fma(uK, U[7], fma(ux, gK, fma(u2, PxK, fma(QuX, S(2.0f), RxK))));
    F[8] = fma(uK, U[8], fma(uy, gK, fma(u2, PyK, fma(QuY, S(2.0f), RyK))));
    v2 uQu = fma(uK, QuK, mul(uO, QuO));
    v2 uR = fma(uK, RK[0], mul(uO, RK[1]));
    F[9] = fma(uK, U[9], fma(u2, fma(PuK, S(4.0f), add(qK, qK)), fma(add(uQu, uR), S(4.0f), SK)));
}

// zeta + sqrt(zeta^2 + D0), discriminant clamped at 0, rationalised for zeta < 0.
__device__ __forceinline__ float hyp1(float z, float D0, float D, float rt) {
    return z >= 0.0f ? z + rt : (D > 0.0f ? __fdividef(D0, rt - z) : z);
}
__device__ __forceinline__ v2 hyp_x2(v2 z, v2 D0) {
    v2 D = fma(z, z, D0);
    v2 rt = sqrt_(make_float2(fmaxf(D.x, 0.0f), fmaxf(D.y, 0.0f)));
    return make_float2(hyp1(z.x, D0.x, D.x, rt.x), hyp1(z.y, D0.y, D.y, rt.y));
}

// Eq. (14mom-approx-ws-equations) for two (P*_kk, q*_k, |q*_perp|) triples
// at once: the dimensionless lambda*_max (lp) and lambda*_min (lm).
__device__ __forceinline__ void lam_core_x2(v2 Pkk, v2 qd, v2 qperp, v2 sb, v2 isb, v2 ssb,
                                            v2& lp, v2& lm) {
    v2 l2 = lg2(Pkk);
    v2 Pkk2 = mul(Pkk, Pkk);
    v2 a = mul(ex2(fma(Pkk2, S(-LOG2E), mul(l2, S(1.1f)))), S(1.4f));
    v2 b = mul(mul(Pkk, S(0.9f)), ex2(mul(ex2(mul(l2, S(1.4f))), S(-0.5f * LOG2E))));
    v2 C = sqrt_(mul(fma(sb, S(-3.0f), S(3.0f)), Pkk));
    v2 E = mul(C, S(0.8f));
    // B = 5 - 4 r + sqrt(2 (5 - 3 r)(1 - r)), Y = (sqrt B - E)^2, r = sqrt(sigma)
    v2 B = add(fma(ssb, S(-4.0f), S(5.0f)),
               sqrt_(mul(mul(fma(ssb, S(-3.0f), S(5.0f)), sub(S(1.0f), ssb)), S(2.0f))));
    v2 dd = sub(sqrt_(B), E);
    v2 Y = mul(dd, dd);
    v2 al = mul(qperp, fma(Pkk2, S(0.6f), fma(Pkk, S(-0.38f), S(0.35f))));
    v2 base = fma(mul(sb, sb), mul(Y, S(4.0f)), mul(mul(qperp, qperp), S(0.1f)));
    v2 pre = mul(fma(a, sb, b), mul(isb, S(0.5f)));
    v2 zp = add(qd, al), zm = sub(al, qd);
    v2 m08 = mul(mul(sb, C), S(-0.8f));
    lp = fma(pre, hyp_x2(zp, fma(zp, m08, base)), E);
    lm = neg(fma(pre, hyp_x2(zm, fma(zm, m08, base)), E));
}

// The same along K for two face states, q_perp = |q*_O|.
template <int K>
__device__ __forceinline__ void lam_x2(const DimX2& g, v2 sb, v2 isb, v2 ssb, v2& lp, v2& lm) {
    lam_core_x2(K == 0 ? g.a : g.d, K == 0 ? g.qx : g.qy, abs_(K == 0 ? g.qy : g.qx), sb, isb,
                ssb, lp, lm);
}

// CFL rates max(|lambda_min|, |lambda_max|) of one cell state in x and y
// (the two directions as the lanes of one wave-speed evaluation).
__device__ __forceinline__ void rates_x2(const float* Q, float sigma_lim, float k_ws, float& ax,
                                         float& ay) {
    DimlessP<float> g;
    dimless_p(Q, g);
    const float sb = clamp_sigma(g.sig, sigma_lim);
    v2 lp, lm;
    lam_core_x2(make_float2(g.a, g.d), make_float2(g.qx, g.qy),
                make_float2(fabsf(g.qy), fabsf(g.qx)), S(sb), S(1.0f / sb), S(sqrtf(sb)), lp, lm);
    const v2 u = make_float2(Q[1], Q[2]);
    const v2 ks = S(k_ws * g.sq);
    const v2 hi = fma(lp, ks, u), lo = fma(lm, ks, u);
    ax = fmaxf(fabsf(lo.x), fabsf(hi.x));
    ay = fmaxf(fabsf(lo.y), fabsf(hi.y));
}

// Both face states of a face: conserved U, K-flux F, wave speeds, and the
// raw sigma and det P* (the conditioning the mixed policy checks).
template <int K>
__device__ __forceinline__ void face_eval_x2(const v2* Q, float sigma_lim, float k_ws, v2* U,
                                             v2* F, v2& lmin, v2& lmax, v2& sig, v2& det) {
    DimX2 g;
    dimless_x2(Q, g);
    v2 sb = clamp_sigma_x2(g.sig, sigma_lim);
    v2 rsb = rsqrt_(sb);
    v2 isb = mul(rsb, rsb), ssb = mul(sb, rsb);       // 1/sigma, sqrt(sigma)
    v2 QK[4], RK[2], SK;
    closure_x2<K>(g, sb, isb, ssb, QK, RK, SK);
    v2 u2, Pux, Puy;
    prim2cons_x2(Q, g.tr, U, u2, Pux, Puy);
    flux_x2<K>(Q, U, u2, Pux, Puy, QK, RK, SK, F);
    v2 lp, lm;
    lam_x2<K>(g, sb, isb, ssb, lp, lm);
    const v2 uK = Q[1 + K];
    v2 ks = mul(g.sq, S(k_ws));
    lmax = fma(lp, ks, uK);
    lmin = fma(lm, ks, uK);
    sig = g.sig;
    det = g.det;
}

}  // namespace x2
}  // namespace mxe
