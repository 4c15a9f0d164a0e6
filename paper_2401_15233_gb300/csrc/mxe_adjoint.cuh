// mxe_adjoint.cuh -- hand-written reverse mode (discrete adjoint) of the
// planar 14-moment point physics in FP64: primitive recovery, the
// interpolative closure (Sec. 2.4), the K-flux, the wave-speed fit
// (Sec. 5), the BGK source with its local relaxation time, and the HLL /
// Rusanov face flux (Sec. 3.1).
//
// Every *_bwd function recomputes the primal intermediates it needs with the
// forward formulas of mxe_planar.cuh, then propagates adjoints in reverse
// order: given the adjoints of a function's outputs it ADDS the adjoints of
// its inputs.  Branches follow the primal: a clamp that is active has
// derivative zero, min/max/minmod differentiate the selected argument,
// |x| has derivative sign(x) (0 at 0).
#pragma once
#include "mxe_planar.cuh"

namespace mxe {
namespace adj {

// Adjoint of DimlessP's fields that the closure and wave speeds use.
template <class T>
struct DimlessBar {
    T th, sq, a, b, d, f, qx, qy, trPs, T2, yx, yy, sig;
    __device__ __forceinline__ void zero() {
        th = sq = a = b = d = f = qx = qy = trPs = T2 = yx = yy = sig = T(0.0);
    }
};

// sigma = (A + rt)/(4 Tn) for A >= 0, X / (4 Tn (rt - A)) otherwise,
// rt = sqrt(A^2 + X)
template <class T>
__device__ __forceinline__ void sigma_root_bwd(T A, T X, T Tn, T sbar,
                                               T& Ab, T& Xb, T& Tnb) {
    if (sbar == T(0.0)) return;
    const T rt = M<T>::sqrt_(A * A + X);
    T rtb;
    if (A >= T(0.0)) {
        const T den = T(4.0) * Tn;
        const T sig = (A + rt) / den;
        Ab += sbar / den;
        rtb = sbar / den;
        Tnb -= sbar * sig / Tn;
    } else {
        const T D = T(4.0) * Tn * (rt - A);
        const T sig = X / D;
        Xb += sbar / D;
        const T Db = -sbar * sig / D;
        Tnb += Db * T(4.0) * (rt - A);
        rtb = Db * T(4.0) * Tn;
        Ab -= Db * T(4.0) * Tn;
    }
    if (rt > T(0.0)) {
        Ab += rtb * A / rt;
        Xb += rtb * T(0.5) / rt;
    }
}

// Reverse of dimless_p: adjoints gb of the fields of g -> adds to Qb.
template <class T>
__device__ __forceinline__ void dimless_p_bwd(const T* Q, const DimlessP<T>& g,
                                              DimlessBar<T> gb, T* Qb) {
    const T rho = Q[0];
    const T p = (Q[3] + Q[5] + Q[6]) / T(3.0);
    const T ip = T(1.0) / p;
    const T isc3 = T(1.0) / (rho * g.th * g.sq);
    const T Rs = Q[9] / (rho * g.th * g.th);
    const T det2 = g.a * g.d - g.b * g.b;
    const T i2 = T(1.0) / det2;
    const T qPq = g.qx * g.yx + g.qy * g.yy;
    const T A = T(2.0) * g.T2 + g.trPs * g.trPs - Rs;
    const T X = T(8.0) * g.T2 * qPq;
    // sigma
    T Ab = T(0.0), Xb = T(0.0);
    sigma_root_bwd(A, X, g.T2, gb.sig, Ab, Xb, gb.T2);
    gb.T2 += T(2.0) * Ab;
    gb.trPs += T(2.0) * g.trPs * Ab;
    T Rsb = -Ab;
    gb.T2 += T(8.0) * qPq * Xb;
    const T qPqb = T(8.0) * g.T2 * Xb;
    gb.qx += g.yx * qPqb;
    gb.yx += g.qx * qPqb;
    gb.qy += g.yy * qPqb;
    gb.yy += g.qy * qPqb;
    // y = P*^-1 q* with the 2x2 block inverse (ia, ib, id)
    const T iab = gb.yx * g.qx;
    const T ibb = gb.yx * g.qy + gb.yy * g.qx;
    const T idb = gb.yy * g.qy;
    gb.qx += gb.yx * g.ia + gb.yy * g.ib;
    gb.qy += gb.yx * g.ib + gb.yy * g.id;
    gb.d += iab * i2;
    gb.b -= ibb * i2;
    gb.a += idb * i2;
    const T i2b = iab * g.d - ibb * g.b + idb * g.a;
    const T det2b = -i2b * i2 * i2;
    gb.a += det2b * g.d;
    gb.d += det2b * g.a;
    gb.b -= T(2.0) * g.b * det2b;
    // T2 = a^2 + d^2 + f^2 + 2 b^2, trPs = a + d + f
    gb.a += T(2.0) * g.a * gb.T2 + gb.trPs;
    gb.d += T(2.0) * g.d * gb.T2 + gb.trPs;
    gb.f += T(2.0) * g.f * gb.T2 + gb.trPs;
    gb.b += T(4.0) * g.b * gb.T2;
    // Rs = Q9 / (rho th^2)
    T rhob = T(0.0);
    {
        const T den = rho * g.th * g.th;
        Qb[9] += Rsb / den;
        const T denb = -Rsb * Rs / den;
        rhob += denb * g.th * g.th;
        gb.th += denb * T(2.0) * rho * g.th;
    }
    // q* = q isc3, isc3 = 1/(rho th sq)
    Qb[7] += gb.qx * isc3;
    Qb[8] += gb.qy * isc3;
    {
        const T isc3b = gb.qx * Q[7] + gb.qy * Q[8];
        const T denb = -isc3b * isc3 * isc3;
        rhob += denb * g.th * g.sq;
        gb.th += denb * rho * g.sq;
        gb.sq += denb * rho * g.th;
    }
    // P* = P ip
    Qb[3] += gb.a * ip;
    Qb[4] += gb.b * ip;
    Qb[5] += gb.d * ip;
    Qb[6] += gb.f * ip;
    const T ipb = gb.a * Q[3] + gb.b * Q[4] + gb.d * Q[5] + gb.f * Q[6];
    // sq = sqrt(th), th = p / rho, ip = 1/p
    gb.th += gb.sq * T(0.5) / g.sq;
    T pb = gb.th / rho - ipb * ip * ip;
    rhob -= gb.th * g.th / rho;
    Qb[3] += pb / T(3.0);
    Qb[5] += pb / T(3.0);
    Qb[6] += pb / T(3.0);
    Qb[0] += rhob;
}

// zeta + sqrt(zeta^2 + D0) (clamped, rationalised): adjoint hb -> zb, D0b
template <class T>
__device__ __forceinline__ void hyp_bracket_bwd(T z, T D0, T hb, T& zb,
                                                T& D0b) {
    const T D = z * z + D0;
    if (D <= T(0.0)) {
        zb += hb;
        return;
    }
    const T rt = M<T>::sqrt_(D);
    T rtb;
    if (z >= T(0.0)) {
        zb += hb;
        rtb = hb;
    } else {
        const T den = rt - z;
        const T h = D0 / den;
        D0b += hb / den;
        const T denb = -hb * h / den;
        rtb = denb;
        zb -= denb;
    }
    const T Db = rtb * T(0.5) / rt;
    zb += T(2.0) * z * Db;
    D0b += Db;
}

// Intermediates of lam_p<K>.
template <class T>
struct LamP {
    T Pkk, qo, qperp, lP, ea, a_, e1, eb, b_, ssb, C, E, sR10, sB, Y, poly, base, pre;
    T zp, zm, D0p, D0m, hp, hm, lp, lm;
};

// lam_p<K> keeping its intermediates (same formulas, same order).
template <class T, int K>
__device__ __forceinline__ void lam_p_fwd(const DimlessP<T>& g, T sb, LamP<T>& L) {
    L.Pkk = K == 0 ? g.a : g.d;
    const T qd = K == 0 ? g.qx : g.qy;
    L.qo = K == 0 ? g.qy : g.qx;
    L.qperp = fabs(L.qo);
    L.lP = M<T>::log_(L.Pkk);
    L.ea = M<T>::exp_(T(1.1) * L.lP - L.Pkk * L.Pkk);
    L.a_ = T(1.4) * L.ea;
    L.e1 = M<T>::exp_(T(1.4) * L.lP);
    L.eb = M<T>::exp_(-T(0.5) * L.e1);
    L.b_ = T(0.9) * L.Pkk * L.eb;
    L.ssb = M<T>::sqrt_(sb);
    L.C = M<T>::sqrt_((T(3.0) - T(3.0) * sb) * L.Pkk);
    L.E = T(0.8) * L.C;
    // the forward's forms: printed in FP64; in FP32 the identical
    // 2 (5 - 3r)(1 - r) and (sqrt B - E)^2, which cannot round below zero
    if (sizeof(T) == 8)
        L.sR10 = M<T>::sqrt_(T(10.0) - T(16.0) * L.ssb + T(6.0) * sb);
    else
        L.sR10 = M<T>::sqrt_(T(2.0) * (T(5.0) - T(3.0) * L.ssb) * (T(1.0) - L.ssb));
    const T B = T(5.0) - T(4.0) * L.ssb + L.sR10;
    L.sB = M<T>::sqrt_(B);
    if (sizeof(T) == 8) {
        L.Y = B + L.E * L.E - T(2.0) * L.E * L.sB;
    } else {
        const T dd = L.sB - L.E;
        L.Y = dd * dd;
    }
    L.poly = T(0.6) * L.Pkk * L.Pkk - T(0.38) * L.Pkk + T(0.35);
    const T al = L.qperp * L.poly;
    L.base = T(4.0) * sb * sb * L.Y + L.qperp * L.qperp / T(10.0);
    L.pre = (L.a_ * sb + L.b_) / (T(2.0) * sb);
    L.zp = qd + al;
    L.zm = -qd + al;
    L.D0p = -T(0.8) * L.zp * sb * L.C + L.base;
    L.D0m = -T(0.8) * L.zm * sb * L.C + L.base;
    L.hp = hyp_bracket(L.zp, L.D0p);
    L.hm = hyp_bracket(L.zm, L.D0m);
    L.lp = L.pre * L.hp + L.E;
    L.lm = -(L.pre * L.hm + L.E);
}

// Reverse of lam_p<K> from its intermediates: adjoints lpb, lmb of (lp, lm)
// -> gb (a or d, qx, qy), sbb.
template <class T, int K>
__device__ __forceinline__ void lam_p_rev(const LamP<T>& L, T sb, T lpb, T lmb,
                                          DimlessBar<T>& gb, T& sbb) {
    const T Pkk = L.Pkk;
    const T preb = lpb * L.hp - lmb * L.hm;
    const T hpb = lpb * L.pre, hmb = -lmb * L.pre;
    T Eb = lpb - lmb;
    T zpb = T(0.0), zmb = T(0.0), D0pb = T(0.0), D0mb = T(0.0);
    hyp_bracket_bwd(L.zp, L.D0p, hpb, zpb, D0pb);
    hyp_bracket_bwd(L.zm, L.D0m, hmb, zmb, D0mb);
    T Cb = T(0.0);
    const T baseb = D0pb + D0mb;
    zpb += -T(0.8) * sb * L.C * D0pb;
    zmb += -T(0.8) * sb * L.C * D0mb;
    sbb += -T(0.8) * L.C * (L.zp * D0pb + L.zm * D0mb);
    Cb += -T(0.8) * sb * (L.zp * D0pb + L.zm * D0mb);
    const T qdb = zpb - zmb;
    const T alb = zpb + zmb;
    // pre = a_/2 + b_/(2 sb)
    const T a_b = T(0.5) * preb;
    const T b_b = preb / (T(2.0) * sb);
    sbb -= preb * L.b_ / (T(2.0) * sb * sb);
    // base = 4 sb^2 Y + qperp^2/10
    sbb += T(8.0) * sb * L.Y * baseb;
    const T Yb = T(4.0) * sb * sb * baseb;
    T qperpb = L.qperp / T(5.0) * baseb;
    // al = qperp poly(Pkk)
    qperpb += alb * L.poly;
    T Pkkb = alb * L.qperp * (T(1.2) * Pkk - T(0.38));
    // Y = B + E^2 - 2 E sqrt(B)
    const T Bb = Yb * (T(1.0) - L.E / L.sB);
    Eb += Yb * (T(2.0) * L.E - T(2.0) * L.sB);
    // B = 5 - 4 ssb + sqrt(R10), R10 = 10 - 16 ssb + 6 sb
    T ssbb = -T(4.0) * Bb;
    if (L.sR10 > T(0.0)) {
        const T R10b = Bb * T(0.5) / L.sR10;
        ssbb -= T(16.0) * R10b;
        sbb += T(6.0) * R10b;
    }
    // E = T(0.8) C, C = sqrt((3 - 3 sb) Pkk)
    Cb += T(0.8) * Eb;
    if (L.C > T(0.0)) {
        const T vb = Cb * T(0.5) / L.C;
        sbb -= T(3.0) * Pkk * vb;
        Pkkb += (T(3.0) - T(3.0) * sb) * vb;
    }
    sbb += ssbb * T(0.5) / L.ssb;
    // b_ = T(0.9) Pkk exp(-T(0.5) exp(T(1.4) lP)), a_ = T(1.4) exp(T(1.1) lP - Pkk^2)
    Pkkb += T(0.9) * L.eb * b_b;
    const T ebb = T(0.9) * Pkk * b_b;
    const T e1b = -T(0.5) * ebb * L.eb;
    T lPb = T(1.4) * e1b * L.e1;
    const T eab = T(1.4) * a_b;
    lPb += T(1.1) * eab * L.ea;
    Pkkb -= T(2.0) * Pkk * eab * L.ea;
    Pkkb += lPb / Pkk;
    const T sgn = L.qo > T(0.0) ? T(1.0) : (L.qo < T(0.0) ? -T(1.0) : T(0.0));
    if (K == 0) {
        gb.a += Pkkb;
        gb.qx += qdb;
        gb.qy += qperpb * sgn;
    } else {
        gb.d += Pkkb;
        gb.qy += qdb;
        gb.qx += qperpb * sgn;
    }
}

// Reverse of lam_p<K> (recomputing its intermediates).
template <class T, int K>
__device__ __forceinline__ void lam_p_bwd(const DimlessP<T>& g, T sb, T lpb,
                                          T lmb, DimlessBar<T>& gb, T& sbb) {
    LamP<T> L;
    lam_p_fwd<T, K>(g, sb, L);
    lam_p_rev<T, K>(L, sb, lpb, lmb, gb, sbb);
}

// Intermediates of closure_p<K> (recomputed for the reverse sweep).
template <class T>
struct CloP {
    T P2xx, P2xy, P2yy, P2zz, P3xx, P3xy, P3yy, trP3;
    T Bxx, Bxy, Byy, iB, vx, vy, wx, wy;
    T QKKK, QKKO, QKOO, QKzz, isb, RKK, ROK, yQy;
    T c1, c2, c3, P4KK, P4KO, mKK, mKO, Wq, ssb, Ss, sc3, sc4, sc5;
};

// Forward closure_p<K> keeping its intermediates; outputs QK, RK, SK as in
// closure_p.
template <class T, int K>
__device__ __forceinline__ void closure_p_fwd(const T* Q, const DimlessP<T>& g,
                                              T sb, CloP<T>& c, T* QK, T* RK,
                                              T& SK) {
    const T a = g.a, b = g.b, d = g.d, f = g.f;
    c.P2xx = a * a + b * b; c.P2xy = b * (a + d); c.P2yy = b * b + d * d; c.P2zz = f * f;
    c.P3xx = c.P2xx * a + c.P2xy * b; c.P3xy = c.P2xx * b + c.P2xy * d;
    c.P3yy = c.P2xy * b + c.P2yy * d;
    const T P3zz = c.P2zz * f;
    c.trP3 = c.P3xx + c.P3yy + P3zz;
    c.Bxx = T(2.0) * a * g.T2 + T(4.0) * c.P3xx;
    c.Bxy = T(2.0) * b * g.T2 + T(4.0) * c.P3xy;
    c.Byy = T(2.0) * d * g.T2 + T(4.0) * c.P3yy;
    c.iB = T(1.0) / (c.Bxx * c.Byy - c.Bxy * c.Bxy);
    c.vx = (c.Byy * g.qx - c.Bxy * g.qy) * c.iB;
    c.vy = (c.Bxx * g.qy - c.Bxy * g.qx) * c.iB;
    c.wx = a * c.vx + b * c.vy; c.wy = b * c.vx + d * c.vy;
    const T wK = K == 0 ? c.wx : c.wy, wO = K == 0 ? c.wy : c.wx;
    const T vK = K == 0 ? c.vx : c.vy, vO = K == 0 ? c.vy : c.vx;
    const T yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    const T P2KK = K == 0 ? c.P2xx : c.P2yy, P2OO = K == 0 ? c.P2yy : c.P2xx;
    const T P3KK = K == 0 ? c.P3xx : c.P3yy;
    const T PKK = K == 0 ? a : d;
    const T qK = K == 0 ? g.qx : g.qy;
    c.QKKK = T(6.0) * wK * P2KK;
    c.QKKO = T(4.0) * wK * c.P2xy + T(2.0) * wO * P2KK;
    c.QKOO = T(2.0) * wK * P2OO + T(4.0) * wO * c.P2xy;
    c.QKzz = T(2.0) * wK * c.P2zz;
    c.isb = T(1.0) / sb;
    c.RKK = (c.QKKK * yK + c.QKKO * yO) * c.isb + T(2.0) * (T(1.0) - sb) * P2KK + PKK * g.trPs;
    c.ROK = (c.QKKO * yK + c.QKOO * yO) * c.isb + T(2.0) * (T(1.0) - sb) * c.P2xy + b * g.trPs;
    c.yQy = c.QKKK * yK * yK + T(2.0) * c.QKKO * yK * yO + c.QKOO * yO * yO;
    const T t = g.trPs, t2 = t * t;
    c.c1 = T(2.0) * t2 * t + T(12.0) * c.trP3 - T(2.0) * g.T2 * t;
    c.c2 = T(14.0) * g.T2 - T(6.0) * t2;
    c.c3 = T(20.0) * t;
    c.P4KK = P2KK * P2KK + c.P2xy * c.P2xy;
    c.P4KO = c.P2xy * (c.P2xx + c.P2yy);
    c.mKK = c.c1 * PKK + c.c2 * P2KK + c.c3 * P3KK + T(20.0) * c.P4KK;
    c.mKO = c.c1 * b + c.c2 * c.P2xy + c.c3 * c.P3xy + T(20.0) * c.P4KO;
    c.Wq = c.mKK * vK + c.mKO * vO;
    c.ssb = M<T>::sqrt_(sb);
    c.Ss = c.yQy * c.isb * c.isb + T(2.0) * c.ssb * t * qK + (T(1.0) - c.ssb) * c.Wq;
    const T rho = Q[0];
    c.sc3 = rho * g.th * g.sq; c.sc4 = rho * g.th * g.th; c.sc5 = c.sc4 * g.sq;
    QK[0] = c.QKKK * c.sc3; QK[1] = c.QKKO * c.sc3; QK[2] = c.QKOO * c.sc3; QK[3] = c.QKzz * c.sc3;
    RK[0] = c.RKK * c.sc4; RK[1] = c.ROK * c.sc4;
    SK = c.Ss * c.sc5;
}

// Reverse of closure_p<K>: adjoints (QKb, RKb, SKb) -> gb, sbb, Qb[0].
template <class T, int K>
__device__ __forceinline__ void closure_p_bwd(const T* Q, const DimlessP<T>& g,
                                              T sb, const CloP<T>& c, const T* QKb,
                                              const T* RKb, T SKb, DimlessBar<T>& gb,
                                              T& sbb, T* Qb) {
    const T a = g.a, b = g.b, d = g.d, f = g.f;
    const T wK = K == 0 ? c.wx : c.wy, wO = K == 0 ? c.wy : c.wx;
    const T vK = K == 0 ? c.vx : c.vy, vO = K == 0 ? c.vy : c.vx;
    const T yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    const T P2KK = K == 0 ? c.P2xx : c.P2yy, P2OO = K == 0 ? c.P2yy : c.P2xx;
    const T P3KK = K == 0 ? c.P3xx : c.P3yy;
    const T PKK = K == 0 ? a : d;
    const T qK = K == 0 ? g.qx : g.qy;
    const T t = g.trPs, t2 = t * t;
    const T rho = Q[0];
    // re-dimensionalisation
    const T Ssb = SKb * c.sc5;
    T sc5b = SKb * c.Ss;
    const T RKKb = RKb[0] * c.sc4, ROKb = RKb[1] * c.sc4;
    T sc4b = RKb[0] * c.RKK + RKb[1] * c.ROK;
    T QKKKb = QKb[0] * c.sc3, QKKOb = QKb[1] * c.sc3, QKOOb = QKb[2] * c.sc3;
    const T QKzzb = QKb[3] * c.sc3;
    const T sc3b = QKb[0] * c.QKKK + QKb[1] * c.QKKO + QKb[2] * c.QKOO + QKb[3] * c.QKzz;
    sc4b += sc5b * g.sq;
    gb.sq += sc5b * c.sc4;
    Qb[0] += sc4b * g.th * g.th + sc3b * g.th * g.sq;
    gb.th += sc4b * T(2.0) * rho * g.th + sc3b * rho * g.sq;
    gb.sq += sc3b * rho * g.th;
    // Ss = yQy isb^2 + 2 ssb t qK + (1 - ssb) Wq
    T yQyb = Ssb * c.isb * c.isb;
    T isbb = Ssb * c.yQy * T(2.0) * c.isb;
    const T ssbb = Ssb * (T(2.0) * t * qK - c.Wq);
    T tb = Ssb * T(2.0) * c.ssb * qK;
    T qKb = Ssb * T(2.0) * c.ssb * t;
    const T Wqb = Ssb * (T(1.0) - c.ssb);
    sbb += ssbb * T(0.5) / c.ssb;
    // Wq = mKK vK + mKO vO
    const T mKKb = Wqb * vK, mKOb = Wqb * vO;
    T vKb = Wqb * c.mKK, vOb = Wqb * c.mKO;
    // mKO = c1 b + c2 P2xy + c3 P3xy + 20 P4KO; mKK = c1 PKK + c2 P2KK + c3 P3KK + 20 P4KK
    T c1b = mKOb * b + mKKb * PKK;
    T c2b = mKOb * c.P2xy + mKKb * P2KK;
    T c3b = mKOb * c.P3xy + mKKb * P3KK;
    T bb = mKOb * c.c1;
    T P2xyb = mKOb * c.c2;
    T P3xyb = mKOb * c.c3;
    const T P4KOb = T(20.0) * mKOb;
    T PKKb = mKKb * c.c1;
    T P2KKb = mKKb * c.c2;
    T P3KKb = mKKb * c.c3;
    const T P4KKb = T(20.0) * mKKb;
    // P4KO = P2xy (P2xx + P2yy); P4KK = P2KK^2 + P2xy^2
    P2xyb += P4KOb * (c.P2xx + c.P2yy) + T(2.0) * c.P2xy * P4KKb;
    T P2xxb = P4KOb * c.P2xy, P2yyb = P4KOb * c.P2xy;
    P2KKb += T(2.0) * P2KK * P4KKb;
    // c3 = 20 t; c2 = 14 T2 - 6 t^2; c1 = 2 t^3 + 12 trP3 - 2 T2 t
    tb += T(20.0) * c3b;
    T T2b = T(14.0) * c2b - T(2.0) * t * c1b;
    tb += -T(12.0) * t * c2b + (T(6.0) * t2 - T(2.0) * g.T2) * c1b;
    T trP3b = T(12.0) * c1b;
    // yQy = QKKK yK^2 + 2 QKKO yK yO + QKOO yO^2
    QKKKb += yQyb * yK * yK;
    QKKOb += yQyb * T(2.0) * yK * yO;
    QKOOb += yQyb * yO * yO;
    T yKb = yQyb * (T(2.0) * c.QKKK * yK + T(2.0) * c.QKKO * yO);
    T yOb = yQyb * (T(2.0) * c.QKKO * yK + T(2.0) * c.QKOO * yO);
    // ROK = (QKKO yK + QKOO yO) isb + 2 (1 - sb) P2xy + b trPs
    QKKOb += ROKb * yK * c.isb;
    QKOOb += ROKb * yO * c.isb;
    yKb += ROKb * c.QKKO * c.isb;
    yOb += ROKb * c.QKOO * c.isb;
    isbb += ROKb * (c.QKKO * yK + c.QKOO * yO);
    sbb -= T(2.0) * c.P2xy * ROKb;
    P2xyb += T(2.0) * (T(1.0) - sb) * ROKb;
    bb += t * ROKb;
    tb += b * ROKb;
    // RKK = (QKKK yK + QKKO yO) isb + 2 (1 - sb) P2KK + PKK trPs
    QKKKb += RKKb * yK * c.isb;
    QKKOb += RKKb * yO * c.isb;
    yKb += RKKb * c.QKKK * c.isb;
    yOb += RKKb * c.QKKO * c.isb;
    isbb += RKKb * (c.QKKK * yK + c.QKKO * yO);
    sbb -= T(2.0) * P2KK * RKKb;
    P2KKb += T(2.0) * (T(1.0) - sb) * RKKb;
    PKKb += t * RKKb;
    tb += PKK * RKKb;
    sbb -= isbb * c.isb * c.isb;
    // Q_K.. = w P^2 combinations
    T wKb = T(2.0) * c.P2zz * QKzzb + T(2.0) * P2OO * QKOOb + T(4.0) * c.P2xy * QKKOb +
                 T(6.0) * P2KK * QKKKb;
    T wOb = T(4.0) * c.P2xy * QKOOb + T(2.0) * P2KK * QKKOb;
    T P2zzb = T(2.0) * wK * QKzzb;
    T P2OOb = T(2.0) * wK * QKOOb;
    P2xyb += T(4.0) * wO * QKOOb + T(4.0) * wK * QKKOb;
    P2KKb += T(2.0) * wO * QKKOb + T(6.0) * wK * QKKKb;
    // map K/O selections back to x/y
    T wxb, wyb, vxb, vyb;
    if (K == 0) {
        wxb = wKb; wyb = wOb; vxb = vKb; vyb = vOb;
        gb.yx += yKb; gb.yy += yOb;
        P2xxb += P2KKb; P2yyb += P2OOb;
        gb.a += PKKb; gb.qx += qKb;
    } else {
        wxb = wOb; wyb = wKb; vxb = vOb; vyb = vKb;
        gb.yy += yKb; gb.yx += yOb;
        P2yyb += P2KKb; P2xxb += P2OOb;
        gb.d += PKKb; gb.qy += qKb;
    }
    T P3xxb = K == 0 ? P3KKb : T(0.0), P3yyb = K == 0 ? T(0.0) : P3KKb;
    gb.trPs += tb;
    gb.b += bb;
    // w = P* v (2x2 block)
    gb.a += wxb * c.vx;
    gb.b += wxb * c.vy + wyb * c.vx;
    gb.d += wyb * c.vy;
    vxb += wxb * a + wyb * b;
    vyb += wxb * b + wyb * d;
    // v = B^-1 q* (2x2): vx = (Byy qx - Bxy qy) iB, vy = (Bxx qy - Bxy qx) iB
    const T nxb = vxb * c.iB, nyb = vyb * c.iB;
    const T iBb = vxb * (c.Byy * g.qx - c.Bxy * g.qy) + vyb * (c.Bxx * g.qy - c.Bxy * g.qx);
    T Byyb = nxb * g.qx, Bxxb = nyb * g.qy;
    T Bxyb = -(nxb * g.qy + nyb * g.qx);
    gb.qx += nxb * c.Byy - nyb * c.Bxy;
    gb.qy += -nxb * c.Bxy + nyb * c.Bxx;
    const T detBb = -iBb * c.iB * c.iB;
    Bxxb += detBb * c.Byy;
    Byyb += detBb * c.Bxx;
    Bxyb -= T(2.0) * c.Bxy * detBb;
    // B = 2 P* T2 + 4 P*^3 (2x2 block)
    gb.a += T(2.0) * g.T2 * Bxxb;
    gb.b += T(2.0) * g.T2 * Bxyb;
    gb.d += T(2.0) * g.T2 * Byyb;
    T2b += T(2.0) * (a * Bxxb + b * Bxyb + d * Byyb);
    P3xxb += T(4.0) * Bxxb + trP3b;
    P3xyb += T(4.0) * Bxyb;
    P3yyb += T(4.0) * Byyb + trP3b;
    const T P3zzb = trP3b;
    gb.T2 += T2b;
    // P^3 = P^2 P
    P2zzb += P3zzb * f;
    gb.f += P3zzb * c.P2zz;
    P2xyb += P3yyb * b + P3xyb * d + P3xxb * b;
    gb.b += P3yyb * c.P2xy + P3xyb * c.P2xx + P3xxb * c.P2xy;
    P2yyb += P3yyb * d;
    gb.d += P3yyb * c.P2yy + P3xyb * c.P2xy;
    P2xxb += P3xyb * b + P3xxb * a;
    gb.a += P3xxb * c.P2xx;
    // P^2
    gb.f += T(2.0) * f * P2zzb;
    gb.b += T(2.0) * b * P2yyb + (a + d) * P2xyb + T(2.0) * b * P2xxb;
    gb.d += T(2.0) * d * P2yyb + b * P2xyb;
    gb.a += b * P2xyb + T(2.0) * a * P2xxb;
}

// Reverse of flux_p<K>: Fb -> Qb (primitives used directly), Ub (adjoint of
// the conserved vector the flux carries), QKb, RKb, SKb.
template <class T, int K>
__device__ __forceinline__ void flux_p_bwd(const T* Q, const T* U, const T* QK,
                                           const T* RK, const T* Fb, T* Qb,
                                           T* Ub, T* QKb, T* RKb, T& SKb) {
    const T ux = Q[1], uy = Q[2];
    const T uK = K == 0 ? ux : uy, uO = K == 0 ? uy : ux;
    const T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5];
    const T PKK = K == 0 ? Pxx : Pyy;
    const T qK = Q[7 + K];
    const T u2 = ux * ux + uy * uy;
    const T PuK = PKK * uK + Pxy * uO;
    const T QuK = QK[0] * uK + QK[1] * uO;
    const T QuO = QK[1] * uK + QK[2] * uO;
    const T PxK = K == 0 ? Pxx : Pxy, PyK = K == 0 ? Pxy : Pyy;
    const T gK = T(2.0) * PuK + qK;
    T uKb = T(0.0), uOb = T(0.0), uxb = T(0.0), uyb = T(0.0), u2b = T(0.0);
#pragma unroll
    for (int n = 0; n < NP; ++n) {
        Ub[n] += uK * Fb[n];
        uKb += Fb[n] * U[n];
    }
    // energy-like moment
    u2b += Fb[9] * (T(4.0) * PuK + T(2.0) * qK);
    T PuKb = T(4.0) * u2 * Fb[9];
    T qKb = T(2.0) * u2 * Fb[9];
    const T uQub = T(4.0) * Fb[9], uRb = T(4.0) * Fb[9];
    SKb += Fb[9];
    uKb += uRb * RK[0] + uQub * QuK;
    uOb += uRb * RK[1] + uQub * QuO;
    T RK0b = uRb * uK, RK1b = uRb * uO;
    T QuKb = uQub * uK, QuOb = uQub * uO;
    // third moments
    uyb += Fb[8] * gK;
    uxb += Fb[7] * gK;
    const T gKb = uy * Fb[8] + ux * Fb[7];
    u2b += Fb[8] * PyK + Fb[7] * PxK;
    T PyKb = u2 * Fb[8], PxKb = u2 * Fb[7];
    const T QuYb = T(2.0) * Fb[8], QuXb = T(2.0) * Fb[7];
    if (K == 0) {
        QuKb += QuXb; QuOb += QuYb;
        RK0b += Fb[7]; RK1b += Fb[8];
    } else {
        QuOb += QuXb; QuKb += QuYb;
        RK1b += Fb[7]; RK0b += Fb[8];
    }
    PuKb += T(2.0) * gKb;
    qKb += gKb;
    // second moments
    T QK0b = T(0.0), QK1b = T(0.0), QK2b = T(0.0);
    const T QK3b = Fb[6];
    uyb += T(2.0) * PyK * Fb[5];
    PyKb += T(2.0) * uy * Fb[5];
    const T QyyKb = Fb[5];
    uxb += PyK * Fb[4];
    PyKb += ux * Fb[4];
    uyb += PxK * Fb[4];
    PxKb += uy * Fb[4];
    QK1b += Fb[4];
    uxb += T(2.0) * PxK * Fb[3];
    PxKb += T(2.0) * ux * Fb[3];
    const T QxxKb = Fb[3];
    if (K == 0) { QK0b += QxxKb; QK2b += QyyKb; } else { QK2b += QxxKb; QK0b += QyyKb; }
    // momentum and the P_iK of the second moments
    T Pxxb = T(0.0), Pxyb = T(0.0), Pyyb = T(0.0);
    if (K == 0) {
        Pxxb += Fb[1] + PxKb;
        Pxyb += Fb[2] + PyKb;
    } else {
        Pxyb += Fb[1] + PxKb;
        Pyyb += Fb[2] + PyKb;
    }
    // (Q_K u), (P u)_K
    QK0b += QuKb * uK;
    QK1b += QuKb * uO + QuOb * uK;
    QK2b += QuOb * uO;
    uKb += QuKb * QK[0] + QuOb * QK[1] + PuKb * PKK;
    uOb += QuKb * QK[1] + QuOb * QK[2] + PuKb * Pxy;
    const T PKKb = PuKb * uK;
    Pxyb += PuKb * uO;
    if (K == 0) Pxxb += PKKb; else Pyyb += PKKb;
    uxb += T(2.0) * ux * u2b + (K == 0 ? uKb : uOb);
    uyb += T(2.0) * uy * u2b + (K == 0 ? uOb : uKb);
    Qb[1] += uxb;
    Qb[2] += uyb;
    Qb[3] += Pxxb;
    Qb[4] += Pxyb;
    Qb[5] += Pyyb;
    Qb[7 + K] += qKb;
    QKb[0] += QK0b; QKb[1] += QK1b; QKb[2] += QK2b; QKb[3] += QK3b;
    RKb[0] += RK0b; RKb[1] += RK1b;
}

// Reverse of prim2cons_p: Ub -> Qb.
template <class T>
__device__ __forceinline__ void prim2cons_p_bwd(const T* Q, const T* Ub, T* Qb) {
    const T rho = Q[0], ux = Q[1], uy = Q[2];
    const T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const T qx = Q[7], qy = Q[8];
    const T u2 = ux * ux + uy * uy;
    const T trP = Pxx + Pyy + Pzz;
    const T Pux = Pxx * ux + Pxy * uy, Puy = Pxy * ux + Pyy * uy;
    const T e = rho * u2 + trP;
    T rhob = Ub[0], uxb = T(0.0), uyb = T(0.0), u2b = T(0.0), trPb = T(0.0);
    T Pxxb = Ub[3], Pxyb = Ub[4], Pyyb = Ub[5], Pzzb = Ub[6];
    T qxb = Ub[7], qyb = Ub[8];
    // U9 = rho u2^2 + 2 u2 trP + 4 uPu + 4 uq + R
    rhob += Ub[9] * u2 * u2;
    u2b += Ub[9] * (T(2.0) * rho * u2 + T(2.0) * trP);
    trPb += T(2.0) * u2 * Ub[9];
    const T uPub = T(4.0) * Ub[9], uqb = T(4.0) * Ub[9];
    // U7, U8 = u_i e + 2 (P u)_i + q_i
    uyb += Ub[8] * e;
    uxb += Ub[7] * e;
    const T eb = Ub[8] * uy + Ub[7] * ux;
    T Puyb = T(2.0) * Ub[8], Puxb = T(2.0) * Ub[7];
    // second moments rho u_i u_j + P_ij
    rhob += Ub[5] * uy * uy + Ub[4] * ux * uy + Ub[3] * ux * ux + Ub[2] * uy + Ub[1] * ux;
    uyb += T(2.0) * rho * uy * Ub[5] + rho * ux * Ub[4] + rho * Ub[2];
    uxb += rho * uy * Ub[4] + T(2.0) * rho * ux * Ub[3] + rho * Ub[1];
    // e = rho u2 + trP
    rhob += eb * u2;
    u2b += eb * rho;
    trPb += eb;
    // uq, uPu
    uxb += uqb * qx + uPub * Pux;
    uyb += uqb * qy + uPub * Puy;
    qxb += uqb * ux;
    qyb += uqb * uy;
    Puxb += uPub * ux;
    Puyb += uPub * uy;
    // P u
    Pxyb += Puyb * ux + Puxb * uy;
    Pyyb += Puyb * uy;
    Pxxb += Puxb * ux;
    uxb += Puyb * Pxy + Puxb * Pxx;
    uyb += Puyb * Pyy + Puxb * Pxy;
    Pxxb += trPb; Pyyb += trPb; Pzzb += trPb;
    uxb += T(2.0) * ux * u2b;
    uyb += T(2.0) * uy * u2b;
    Qb[0] += rhob; Qb[1] += uxb; Qb[2] += uyb;
    Qb[3] += Pxxb; Qb[4] += Pxyb; Qb[5] += Pyyb; Qb[6] += Pzzb;
    Qb[7] += qxb; Qb[8] += qyb; Qb[9] += Ub[9];
}

// Reverse of face_eval_p<K>: adjoints of (U, F, lmin, lmax) of one face
// state -> Qb (added).
template <class T, int K>
__device__ __forceinline__ void face_eval_p_bwd(const T* Q, T sl, T kw,
                                                const T* Ubar_in, const T* Fb,
                                                T lminb, T lmaxb, T* Qb) {
    DimlessP<T> g;
    dimless_p(Q, g);
    const T sb = clamp_sigma(g.sig, sl);
    CloP<T> c;
    T QK[4], RK[2], SK;
    closure_p_fwd<T, K>(Q, g, sb, c, QK, RK, SK);
    T U[NP];
    prim2cons_p(Q, U);
    T lp, lm;
    lam_p<T, K>(g, sb, lp, lm);
    DimlessBar<T> gb;
    gb.zero();
    T sbb = T(0.0);
    // lmax = u_K + k lp sq, lmin = u_K + k lm sq
    Qb[1 + K] += lmaxb + lminb;
    gb.sq += kw * (lmaxb * lp + lminb * lm);
    const T lpb = lmaxb * kw * g.sq, lmb = lminb * kw * g.sq;
    // flux
    T Ub[NP];
#pragma unroll
    for (int n = 0; n < NP; ++n) Ub[n] = Ubar_in[n];
    T QKb[4] = {T(0.0), T(0.0), T(0.0), T(0.0)}, RKb[2] = {T(0.0), T(0.0)}, SKb = T(0.0);
    flux_p_bwd<T, K>(Q, U, QK, RK, Fb, Qb, Ub, QKb, RKb, SKb);
    prim2cons_p_bwd(Q, Ub, Qb);
    closure_p_bwd<T, K>(Q, g, sb, c, QKb, RKb, SKb, gb, sbb, Qb);
    lam_p_bwd<T, K>(g, sb, lpb, lmb, gb, sbb);
    if (!(g.sig < sl) && !(g.sig > T(1.0))) gb.sig += sbb;
    dimless_p_bwd(Q, g, gb, Qb);
}

// One face state evaluated once and reversed: the primal outputs (U, F,
// lmin, lmax) are handed to `outadj`, which returns their adjoints (the
// numerical-flux reverse needs both states of the face); the reverse then
// reuses the primal intermediates.  Adds to Qb.
template <class T, int K, class OutAdj>
__device__ __forceinline__ void face_side_adj(const T* Q, T sl, T kw,
                                              OutAdj&& outadj, T* Qb) {
    DimlessP<T> g;
    dimless_p(Q, g);
    const T sb = clamp_sigma(g.sig, sl);
    CloP<T> c;
    T QK[4], RK[2], SK;
    closure_p_fwd<T, K>(Q, g, sb, c, QK, RK, SK);
    T U[NP], F[NP];
    prim2cons_p(Q, U);
    flux_p<T, K>(Q, U, QK, RK, SK, F);
    LamP<T> L;
    lam_p_fwd<T, K>(g, sb, L);
    const T lmax = Q[1 + K] + kw * L.lp * g.sq;
    const T lmin = Q[1 + K] + kw * L.lm * g.sq;
    T Ub[NP], Fb[NP], lminb, lmaxb;
    outadj(U, F, lmin, lmax, Ub, Fb, lminb, lmaxb);
    DimlessBar<T> gb;
    gb.zero();
    T sbb = T(0.0);
    Qb[1 + K] += lmaxb + lminb;
    gb.sq += kw * (lmaxb * L.lp + lminb * L.lm);
    const T lpb = lmaxb * kw * g.sq, lmb = lminb * kw * g.sq;
    T QKb[4] = {T(0.0), T(0.0), T(0.0), T(0.0)}, RKb[2] = {T(0.0), T(0.0)}, SKb = T(0.0);
    flux_p_bwd<T, K>(Q, U, QK, RK, Fb, Qb, Ub, QKb, RKb, SKb);
    prim2cons_p_bwd(Q, Ub, Qb);
    closure_p_bwd<T, K>(Q, g, sb, c, QKb, RKb, SKb, gb, sbb, Qb);
    lam_p_rev<T, K>(L, sb, lpb, lmb, gb, sbb);
    if (!(g.sig < sl) && !(g.sig > T(1.0))) gb.sig += sbb;
    dimless_p_bwd(Q, g, gb, Qb);
}

// Reverse of source_p with the local relaxation time tau_p: W = adjoint of
// the source vector C -> Qb; returns the adjoint of tau_ref.
template <class T>
__device__ __forceinline__ T source_p_bwd(int model, T tau_ref, T rho_ref,
                                               T T_ref, const T* Q, const T* W,
                                               T* Qb) {
    const T rho = Q[0], ux = Q[1], uy = Q[2];
    const T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const T qx = Q[7], qy = Q[8], R = Q[9];
    const T tau = tau_p(model, tau_ref, rho_ref, T_ref, Q);
    const T p = (Pxx + Pyy + Pzz) / T(3.0);
    const T Pux = Pxx * ux + Pxy * uy, Puy = Pxy * ux + Pyy * uy;
    const T uPu = ux * Pux + uy * Puy, uq = ux * qx + uy * qy, u2 = ux * ux + uy * uy;
    // C_k = -N_k / tau
    const T N[10] = {T(0.0), T(0.0), T(0.0), Pxx - p, Pxy, Pyy - p, Pzz - p,
                          T(2.0) * Pux + qx - T(2.0) * ux * p, T(2.0) * Puy + qy - T(2.0) * uy * p,
                          (T(4.0) * uPu + T(4.0) * uq + R) - (T(4.0) * u2 * p + T(15.0) * p * p / rho)};
    T WN = T(0.0);
#pragma unroll
    for (int k = 3; k < NP; ++k) WN += W[k] * N[k];
    const T itau = T(1.0) / tau;
    const T taub = WN * itau * itau;
    T n[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) n[k] = -W[k] * itau;
    T rhob = T(0.0), uxb = T(0.0), uyb = T(0.0), pb = T(0.0), u2b = T(0.0);
    T Pxxb = n[3], Pxyb = n[4], Pyyb = n[5], Pzzb = n[6];
    pb -= n[3] + n[5] + n[6];
    T qxb = n[7], qyb = n[8], Rb = n[9];
    const T uPub = T(4.0) * n[9], uqb = T(4.0) * n[9];
    u2b -= T(4.0) * p * n[9];
    pb -= (T(4.0) * u2 + T(30.0) * p / rho) * n[9];
    rhob += T(15.0) * p * p / (rho * rho) * n[9];
    T Puxb = T(2.0) * n[7], Puyb = T(2.0) * n[8];
    uxb -= T(2.0) * p * n[7];
    uyb -= T(2.0) * p * n[8];
    pb -= T(2.0) * ux * n[7] + T(2.0) * uy * n[8];
    uxb += uqb * qx + uPub * Pux;
    uyb += uqb * qy + uPub * Puy;
    qxb += uqb * ux;
    qyb += uqb * uy;
    Puxb += uPub * ux;
    Puyb += uPub * uy;
    Pxyb += Puyb * ux + Puxb * uy;
    Pyyb += Puyb * uy;
    Pxxb += Puxb * ux;
    uxb += Puyb * Pxy + Puxb * Pxx;
    uyb += Puyb * Pyy + Puxb * Pxy;
    uxb += T(2.0) * ux * u2b;
    uyb += T(2.0) * uy * u2b;
    T tau_refb;
    if (model == 1) {
        tau_refb = taub;
    } else {
        // tau = tau_ref (rho_ref / rho) sqrt(T_ref / T), T = tr P / (3 rho)
        const T Tt = (Pxx + Pyy + Pzz) / (T(3.0) * rho);
        const T Tb = -taub * tau / (T(2.0) * Tt);
        rhob += -taub * tau / rho - Tb * Tt / rho;
        const T trb = Tb / (T(3.0) * rho);
        Pxxb += trb; Pyyb += trb; Pzzb += trb;
        tau_refb = taub * tau / tau_ref;
    }
    Pxxb += pb / T(3.0); Pyyb += pb / T(3.0); Pzzb += pb / T(3.0);
    Qb[0] += rhob; Qb[1] += uxb; Qb[2] += uyb;
    Qb[3] += Pxxb; Qb[4] += Pxyb; Qb[5] += Pyyb; Qb[6] += Pzzb;
    Qb[7] += qxb; Qb[8] += qyb; Qb[9] += Rb;
    return tau_refb;
}

// Reverse of the planar primitive recovery Q = prim(U): Qb -> Ub (added).
template <class T>
__device__ __forceinline__ void cons2prim_p_bwd(const T* Q, const T* Qbar, T* Ub) {
    const T rho = Q[0], ux = Q[1], uy = Q[2];
    const T Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const T qx = Q[7], qy = Q[8];
    const T u2 = ux * ux + uy * uy, trP = Pxx + Pyy + Pzz;
    T rhob = Qbar[0], uxb = Qbar[1], uyb = Qbar[2];
    T Pxxb = Qbar[3], Pxyb = Qbar[4], Pyyb = Qbar[5], Pzzb = Qbar[6];
    T qxb = Qbar[7], qyb = Qbar[8];
    const T Rb = Qbar[9];
    // R = U9 - rho u2^2 - 2 u2 trP - 4 uPu - 4 uq
    Ub[9] += Rb;
    rhob -= Rb * u2 * u2;
    T u2b = -Rb * (T(2.0) * rho * u2 + T(2.0) * trP);
    T trPb = -T(2.0) * u2 * Rb;
    const T uPub = -T(4.0) * Rb, uqb = -T(4.0) * Rb;
    uxb += uqb * qx;
    qxb += uqb * ux;
    uyb += uqb * qy;
    qyb += uqb * uy;
    uxb += uPub * (T(2.0) * ux * Pxx + T(2.0) * uy * Pxy);
    uyb += uPub * (T(2.0) * ux * Pxy + T(2.0) * uy * Pyy);
    Pxxb += uPub * ux * ux;
    Pxyb += T(2.0) * uPub * ux * uy;
    Pyyb += uPub * uy * uy;
    // q_i = U_i - rho u_i u2 - u_i trP - 2 (P u)_i
    Ub[7] += qxb;
    Ub[8] += qyb;
    rhob -= qxb * ux * u2 + qyb * uy * u2;
    uxb -= qxb * (rho * u2 + trP + T(2.0) * Pxx) + T(2.0) * qyb * Pxy;
    uyb -= qyb * (rho * u2 + trP + T(2.0) * Pyy) + T(2.0) * qxb * Pxy;
    u2b -= qxb * rho * ux + qyb * rho * uy;
    trPb -= qxb * ux + qyb * uy;
    Pxxb -= T(2.0) * qxb * ux;
    Pxyb -= T(2.0) * qxb * uy + T(2.0) * qyb * ux;
    Pyyb -= T(2.0) * qyb * uy;
    Pxxb += trPb; Pyyb += trPb; Pzzb += trPb;
    uxb += T(2.0) * ux * u2b;
    uyb += T(2.0) * uy * u2b;
    // P_ij = U_ij - rho u_i u_j
    Ub[6] += Pzzb;
    Ub[5] += Pyyb;
    Ub[4] += Pxyb;
    Ub[3] += Pxxb;
    rhob -= Pyyb * uy * uy + Pxyb * ux * uy + Pxxb * ux * ux;
    uyb -= T(2.0) * rho * uy * Pyyb + rho * ux * Pxyb;
    uxb -= rho * uy * Pxyb + T(2.0) * rho * ux * Pxxb;
    // u_i = U_i / rho
    Ub[2] += uyb / rho;
    Ub[1] += uxb / rho;
    rhob -= (uyb * uy + uxb * ux) / rho;
    Ub[0] += rhob;
}

// Shared limiter with its selected field and the partial derivatives of
// phi_{k*} with respect to dm and dp (zero when no field sets phi).
template <class T>
struct PhiAdj {
    T phi, ddm, ddp;
    int ks;
};

// Shared limiter from the stencil differences dm = q0 - qm, dp = qp - q0.
// A flat field (the flat test against the centre cell fr) has phi_k = 1 and
// never sets phi.
template <class T, int NF>
__device__ __forceinline__ PhiAdj<T> phi_adj_d(const T* dm, const T* dp, int lim,
                                               const FlatRef<T>& fr) {
    PhiAdj<T> r{T(1.0), T(0.0), T(0.0), -1};
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const T pk = phi_field(dm[k], dp[k], lim);
        if (pk < r.phi && !field_flat<NF>(fr, k, abs_max(dm[k], dp[k]))) {
            r.phi = pk;
            r.ks = k;
            if (mul_rn(dm[k], dp[k]) > T(0.0)) {
                if (lim == 1) {
                    const T s = dm[k] * dm[k] + dp[k] * dp[k];
                    r.ddm = T(2.0) * dp[k] * (dp[k] * dp[k] - dm[k] * dm[k]) / (s * s);
                    r.ddp = T(2.0) * dm[k] * (dm[k] * dm[k] - dp[k] * dp[k]) / (s * s);
                } else {
                    const T am = fabs(dm[k]), ap = fabs(dp[k]), s = am + ap;
                    const T sm = dm[k] > T(0.0) ? T(1.0) : T(-1.0);
                    const T sp = dp[k] > T(0.0) ? T(1.0) : T(-1.0);
                    if (am < ap) {
                        r.ddm = sm * T(2.0) * ap / (s * s);
                        r.ddp = -sp * T(2.0) * am / (s * s);
                    } else {
                        r.ddp = sp * T(2.0) * am / (s * s);
                        r.ddm = -sm * T(2.0) * ap / (s * s);
                    }
                }
            } else {
                r.ddm = r.ddp = T(0.0);      // constant branch
            }
        }
    }
    return r;
}

template <class T, int NF>
__device__ __forceinline__ PhiAdj<T> phi_adj(const T* qm, const T* q0, const T* qp, int lim) {
    T dm[NF], dp[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dm[k] = q0[k] - qm[k];
        dp[k] = qp[k] - q0[k];
    }
    return phi_adj_d<T, NF>(dm, dp, lim, flat_ref<NF>(q0, 1));
}

// Reverse of the MUSCL face value qf = q0 + hs (phi cen), cen = (dm + dp)/2,
// phi = phi_{k*}(dm, dp), dm = q0 - qm, dp = qp - q0: adjoint qfb ->
// contributions to the three stencil cells.  A field that is flat across the
// stencil (both differences exactly zero) has the zero slope, whose
// derivative is zero (the same choice as the oracle's tangent): a
// perturbation of a flat stencil is limited, not passed on with phi = 1.
template <class T, int NF>
__device__ __forceinline__ void muscl_bwd_d(const T* dm, const T* dp, const PhiAdj<T>& ph, T hs,
                                            const T* qfb, T* bm, T* b0, T* bp) {
    T phib = T(0.0);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        b0[k] += qfb[k];
        if (dm[k] == T(0.0) && dp[k] == T(0.0)) continue;
        const T cen = T(0.5) * (dm[k] + dp[k]);
        const T cb = hs * ph.phi * qfb[k];
        bm[k] -= T(0.5) * cb;
        bp[k] += T(0.5) * cb;
        phib += hs * cen * qfb[k];
    }
    if (ph.ks >= 0) {
        const T dmb = phib * ph.ddm, dpb = phib * ph.ddp;
#pragma unroll
        for (int k = 0; k < NF; ++k)
            if (k == ph.ks) {
                b0[k] += dmb - dpb;
                bm[k] -= dmb;
                bp[k] += dpb;
            }
    }
}

template <class T, int NF>
__device__ __forceinline__ void muscl_bwd(const T* qm, const T* q0, const T* qp,
                                          const PhiAdj<T>& ph, T hs, const T* qfb, T* bm, T* b0,
                                          T* bp) {
    T dm[NF], dp[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dm[k] = q0[k] - qm[k];
        dp[k] = qp[k] - q0[k];
    }
    muscl_bwd_d<T, NF>(dm, dp, ph, hs, qfb, bm, b0, bp);
}

}  // namespace adj
}  // namespace mxe
