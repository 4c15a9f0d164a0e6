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
struct DimlessBar {
    double th, sq, a, b, d, f, qx, qy, trPs, T2, yx, yy, sig;
    __device__ __forceinline__ void zero() {
        th = sq = a = b = d = f = qx = qy = trPs = T2 = yx = yy = sig = 0.0;
    }
};

// sigma = (A + rt)/(4 Tn) for A >= 0, X / (4 Tn (rt - A)) otherwise,
// rt = sqrt(A^2 + X)
__device__ __forceinline__ void sigma_root_bwd(double A, double X, double Tn, double sbar,
                                               double& Ab, double& Xb, double& Tnb) {
    if (sbar == 0.0) return;
    const double rt = ::sqrt(A * A + X);
    double rtb;
    if (A >= 0.0) {
        const double den = 4.0 * Tn;
        const double sig = (A + rt) / den;
        Ab += sbar / den;
        rtb = sbar / den;
        Tnb -= sbar * sig / Tn;
    } else {
        const double D = 4.0 * Tn * (rt - A);
        const double sig = X / D;
        Xb += sbar / D;
        const double Db = -sbar * sig / D;
        Tnb += Db * 4.0 * (rt - A);
        rtb = Db * 4.0 * Tn;
        Ab -= Db * 4.0 * Tn;
    }
    if (rt > 0.0) {
        Ab += rtb * A / rt;
        Xb += rtb * 0.5 / rt;
    }
}

// Reverse of dimless_p: adjoints gb of the fields of g -> adds to Qb.
__device__ __forceinline__ void dimless_p_bwd(const double* Q, const DimlessP<double>& g,
                                              DimlessBar gb, double* Qb) {
    const double rho = Q[0];
    const double p = (Q[3] + Q[5] + Q[6]) / 3.0;
    const double ip = 1.0 / p;
    const double isc3 = 1.0 / (rho * g.th * g.sq);
    const double Rs = Q[9] / (rho * g.th * g.th);
    const double det2 = g.a * g.d - g.b * g.b;
    const double i2 = 1.0 / det2;
    const double qPq = g.qx * g.yx + g.qy * g.yy;
    const double A = 2.0 * g.T2 + g.trPs * g.trPs - Rs;
    const double X = 8.0 * g.T2 * qPq;
    // sigma
    double Ab = 0.0, Xb = 0.0;
    sigma_root_bwd(A, X, g.T2, gb.sig, Ab, Xb, gb.T2);
    gb.T2 += 2.0 * Ab;
    gb.trPs += 2.0 * g.trPs * Ab;
    double Rsb = -Ab;
    gb.T2 += 8.0 * qPq * Xb;
    const double qPqb = 8.0 * g.T2 * Xb;
    gb.qx += g.yx * qPqb;
    gb.yx += g.qx * qPqb;
    gb.qy += g.yy * qPqb;
    gb.yy += g.qy * qPqb;
    // y = P*^-1 q* with the 2x2 block inverse (ia, ib, id)
    const double iab = gb.yx * g.qx;
    const double ibb = gb.yx * g.qy + gb.yy * g.qx;
    const double idb = gb.yy * g.qy;
    gb.qx += gb.yx * g.ia + gb.yy * g.ib;
    gb.qy += gb.yx * g.ib + gb.yy * g.id;
    gb.d += iab * i2;
    gb.b -= ibb * i2;
    gb.a += idb * i2;
    const double i2b = iab * g.d - ibb * g.b + idb * g.a;
    const double det2b = -i2b * i2 * i2;
    gb.a += det2b * g.d;
    gb.d += det2b * g.a;
    gb.b -= 2.0 * g.b * det2b;
    // T2 = a^2 + d^2 + f^2 + 2 b^2, trPs = a + d + f
    gb.a += 2.0 * g.a * gb.T2 + gb.trPs;
    gb.d += 2.0 * g.d * gb.T2 + gb.trPs;
    gb.f += 2.0 * g.f * gb.T2 + gb.trPs;
    gb.b += 4.0 * g.b * gb.T2;
    // Rs = Q9 / (rho th^2)
    double rhob = 0.0;
    {
        const double den = rho * g.th * g.th;
        Qb[9] += Rsb / den;
        const double denb = -Rsb * Rs / den;
        rhob += denb * g.th * g.th;
        gb.th += denb * 2.0 * rho * g.th;
    }
    // q* = q isc3, isc3 = 1/(rho th sq)
    Qb[7] += gb.qx * isc3;
    Qb[8] += gb.qy * isc3;
    {
        const double isc3b = gb.qx * Q[7] + gb.qy * Q[8];
        const double denb = -isc3b * isc3 * isc3;
        rhob += denb * g.th * g.sq;
        gb.th += denb * rho * g.sq;
        gb.sq += denb * rho * g.th;
    }
    // P* = P ip
    Qb[3] += gb.a * ip;
    Qb[4] += gb.b * ip;
    Qb[5] += gb.d * ip;
    Qb[6] += gb.f * ip;
    const double ipb = gb.a * Q[3] + gb.b * Q[4] + gb.d * Q[5] + gb.f * Q[6];
    // sq = sqrt(th), th = p / rho, ip = 1/p
    gb.th += gb.sq * 0.5 / g.sq;
    double pb = gb.th / rho - ipb * ip * ip;
    rhob -= gb.th * g.th / rho;
    Qb[3] += pb / 3.0;
    Qb[5] += pb / 3.0;
    Qb[6] += pb / 3.0;
    Qb[0] += rhob;
}

// zeta + sqrt(zeta^2 + D0) (clamped, rationalised): adjoint hb -> zb, D0b
__device__ __forceinline__ void hyp_bracket_bwd(double z, double D0, double hb, double& zb,
                                                double& D0b) {
    const double D = z * z + D0;
    if (D <= 0.0) {
        zb += hb;
        return;
    }
    const double rt = ::sqrt(D);
    double rtb;
    if (z >= 0.0) {
        zb += hb;
        rtb = hb;
    } else {
        const double den = rt - z;
        const double h = D0 / den;
        D0b += hb / den;
        const double denb = -hb * h / den;
        rtb = denb;
        zb -= denb;
    }
    const double Db = rtb * 0.5 / rt;
    zb += 2.0 * z * Db;
    D0b += Db;
}

// Intermediates of lam_p<K>.
struct LamP {
    double Pkk, qo, qperp, lP, ea, a_, e1, eb, b_, ssb, C, E, sR10, sB, Y, poly, base, pre;
    double zp, zm, D0p, D0m, hp, hm, lp, lm;
};

// lam_p<K> keeping its intermediates (same formulas, same order).
template <int K>
__device__ __forceinline__ void lam_p_fwd(const DimlessP<double>& g, double sb, LamP& L) {
    L.Pkk = K == 0 ? g.a : g.d;
    const double qd = K == 0 ? g.qx : g.qy;
    L.qo = K == 0 ? g.qy : g.qx;
    L.qperp = fabs(L.qo);
    L.lP = ::log(L.Pkk);
    L.ea = ::exp(1.1 * L.lP - L.Pkk * L.Pkk);
    L.a_ = 1.4 * L.ea;
    L.e1 = ::exp(1.4 * L.lP);
    L.eb = ::exp(-0.5 * L.e1);
    L.b_ = 0.9 * L.Pkk * L.eb;
    L.ssb = ::sqrt(sb);
    L.C = ::sqrt((3.0 - 3.0 * sb) * L.Pkk);
    L.E = 0.8 * L.C;
    L.sR10 = ::sqrt(10.0 - 16.0 * L.ssb + 6.0 * sb);
    const double B = 5.0 - 4.0 * L.ssb + L.sR10;
    L.sB = ::sqrt(B);
    L.Y = B + L.E * L.E - 2.0 * L.E * L.sB;
    L.poly = 0.6 * L.Pkk * L.Pkk - 0.38 * L.Pkk + 0.35;
    const double al = L.qperp * L.poly;
    L.base = 4.0 * sb * sb * L.Y + L.qperp * L.qperp / 10.0;
    L.pre = (L.a_ * sb + L.b_) / (2.0 * sb);
    L.zp = qd + al;
    L.zm = -qd + al;
    L.D0p = -0.8 * L.zp * sb * L.C + L.base;
    L.D0m = -0.8 * L.zm * sb * L.C + L.base;
    L.hp = hyp_bracket(L.zp, L.D0p);
    L.hm = hyp_bracket(L.zm, L.D0m);
    L.lp = L.pre * L.hp + L.E;
    L.lm = -(L.pre * L.hm + L.E);
}

// Reverse of lam_p<K> from its intermediates: adjoints lpb, lmb of (lp, lm)
// -> gb (a or d, qx, qy), sbb.
template <int K>
__device__ __forceinline__ void lam_p_rev(const LamP& L, double sb, double lpb, double lmb,
                                          DimlessBar& gb, double& sbb) {
    const double Pkk = L.Pkk;
    const double preb = lpb * L.hp - lmb * L.hm;
    const double hpb = lpb * L.pre, hmb = -lmb * L.pre;
    double Eb = lpb - lmb;
    double zpb = 0.0, zmb = 0.0, D0pb = 0.0, D0mb = 0.0;
    hyp_bracket_bwd(L.zp, L.D0p, hpb, zpb, D0pb);
    hyp_bracket_bwd(L.zm, L.D0m, hmb, zmb, D0mb);
    double Cb = 0.0;
    const double baseb = D0pb + D0mb;
    zpb += -0.8 * sb * L.C * D0pb;
    zmb += -0.8 * sb * L.C * D0mb;
    sbb += -0.8 * L.C * (L.zp * D0pb + L.zm * D0mb);
    Cb += -0.8 * sb * (L.zp * D0pb + L.zm * D0mb);
    const double qdb = zpb - zmb;
    const double alb = zpb + zmb;
    // pre = a_/2 + b_/(2 sb)
    const double a_b = 0.5 * preb;
    const double b_b = preb / (2.0 * sb);
    sbb -= preb * L.b_ / (2.0 * sb * sb);
    // base = 4 sb^2 Y + qperp^2/10
    sbb += 8.0 * sb * L.Y * baseb;
    const double Yb = 4.0 * sb * sb * baseb;
    double qperpb = L.qperp / 5.0 * baseb;
    // al = qperp poly(Pkk)
    qperpb += alb * L.poly;
    double Pkkb = alb * L.qperp * (1.2 * Pkk - 0.38);
    // Y = B + E^2 - 2 E sqrt(B)
    const double Bb = Yb * (1.0 - L.E / L.sB);
    Eb += Yb * (2.0 * L.E - 2.0 * L.sB);
    // B = 5 - 4 ssb + sqrt(R10), R10 = 10 - 16 ssb + 6 sb
    double ssbb = -4.0 * Bb;
    if (L.sR10 > 0.0) {
        const double R10b = Bb * 0.5 / L.sR10;
        ssbb -= 16.0 * R10b;
        sbb += 6.0 * R10b;
    }
    // E = 0.8 C, C = sqrt((3 - 3 sb) Pkk)
    Cb += 0.8 * Eb;
    if (L.C > 0.0) {
        const double vb = Cb * 0.5 / L.C;
        sbb -= 3.0 * Pkk * vb;
        Pkkb += (3.0 - 3.0 * sb) * vb;
    }
    sbb += ssbb * 0.5 / L.ssb;
    // b_ = 0.9 Pkk exp(-0.5 exp(1.4 lP)), a_ = 1.4 exp(1.1 lP - Pkk^2)
    Pkkb += 0.9 * L.eb * b_b;
    const double ebb = 0.9 * Pkk * b_b;
    const double e1b = -0.5 * ebb * L.eb;
    double lPb = 1.4 * e1b * L.e1;
    const double eab = 1.4 * a_b;
    lPb += 1.1 * eab * L.ea;
    Pkkb -= 2.0 * Pkk * eab * L.ea;
    Pkkb += lPb / Pkk;
    const double sgn = L.qo > 0.0 ? 1.0 : (L.qo < 0.0 ? -1.0 : 0.0);
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
template <int K>
__device__ __forceinline__ void lam_p_bwd(const DimlessP<double>& g, double sb, double lpb,
                                          double lmb, DimlessBar& gb, double& sbb) {
    LamP L;
    lam_p_fwd<K>(g, sb, L);
    lam_p_rev<K>(L, sb, lpb, lmb, gb, sbb);
}

// Intermediates of closure_p<K> (recomputed for the reverse sweep).
struct CloP {
    double P2xx, P2xy, P2yy, P2zz, P3xx, P3xy, P3yy, trP3;
    double Bxx, Bxy, Byy, iB, vx, vy, wx, wy;
    double QKKK, QKKO, QKOO, QKzz, isb, RKK, ROK, yQy;
    double c1, c2, c3, P4KK, P4KO, mKK, mKO, Wq, ssb, Ss, sc3, sc4, sc5;
};

// Forward closure_p<K> keeping its intermediates; outputs QK, RK, SK as in
// closure_p.
template <int K>
__device__ __forceinline__ void closure_p_fwd(const double* Q, const DimlessP<double>& g,
                                              double sb, CloP& c, double* QK, double* RK,
                                              double& SK) {
    const double a = g.a, b = g.b, d = g.d, f = g.f;
    c.P2xx = a * a + b * b; c.P2xy = b * (a + d); c.P2yy = b * b + d * d; c.P2zz = f * f;
    c.P3xx = c.P2xx * a + c.P2xy * b; c.P3xy = c.P2xx * b + c.P2xy * d;
    c.P3yy = c.P2xy * b + c.P2yy * d;
    const double P3zz = c.P2zz * f;
    c.trP3 = c.P3xx + c.P3yy + P3zz;
    c.Bxx = 2.0 * a * g.T2 + 4.0 * c.P3xx;
    c.Bxy = 2.0 * b * g.T2 + 4.0 * c.P3xy;
    c.Byy = 2.0 * d * g.T2 + 4.0 * c.P3yy;
    c.iB = 1.0 / (c.Bxx * c.Byy - c.Bxy * c.Bxy);
    c.vx = (c.Byy * g.qx - c.Bxy * g.qy) * c.iB;
    c.vy = (c.Bxx * g.qy - c.Bxy * g.qx) * c.iB;
    c.wx = a * c.vx + b * c.vy; c.wy = b * c.vx + d * c.vy;
    const double wK = K == 0 ? c.wx : c.wy, wO = K == 0 ? c.wy : c.wx;
    const double vK = K == 0 ? c.vx : c.vy, vO = K == 0 ? c.vy : c.vx;
    const double yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    const double P2KK = K == 0 ? c.P2xx : c.P2yy, P2OO = K == 0 ? c.P2yy : c.P2xx;
    const double P3KK = K == 0 ? c.P3xx : c.P3yy;
    const double PKK = K == 0 ? a : d;
    const double qK = K == 0 ? g.qx : g.qy;
    c.QKKK = 6.0 * wK * P2KK;
    c.QKKO = 4.0 * wK * c.P2xy + 2.0 * wO * P2KK;
    c.QKOO = 2.0 * wK * P2OO + 4.0 * wO * c.P2xy;
    c.QKzz = 2.0 * wK * c.P2zz;
    c.isb = 1.0 / sb;
    c.RKK = (c.QKKK * yK + c.QKKO * yO) * c.isb + 2.0 * (1.0 - sb) * P2KK + PKK * g.trPs;
    c.ROK = (c.QKKO * yK + c.QKOO * yO) * c.isb + 2.0 * (1.0 - sb) * c.P2xy + b * g.trPs;
    c.yQy = c.QKKK * yK * yK + 2.0 * c.QKKO * yK * yO + c.QKOO * yO * yO;
    const double t = g.trPs, t2 = t * t;
    c.c1 = 2.0 * t2 * t + 12.0 * c.trP3 - 2.0 * g.T2 * t;
    c.c2 = 14.0 * g.T2 - 6.0 * t2;
    c.c3 = 20.0 * t;
    c.P4KK = P2KK * P2KK + c.P2xy * c.P2xy;
    c.P4KO = c.P2xy * (c.P2xx + c.P2yy);
    c.mKK = c.c1 * PKK + c.c2 * P2KK + c.c3 * P3KK + 20.0 * c.P4KK;
    c.mKO = c.c1 * b + c.c2 * c.P2xy + c.c3 * c.P3xy + 20.0 * c.P4KO;
    c.Wq = c.mKK * vK + c.mKO * vO;
    c.ssb = ::sqrt(sb);
    c.Ss = c.yQy * c.isb * c.isb + 2.0 * c.ssb * t * qK + (1.0 - c.ssb) * c.Wq;
    const double rho = Q[0];
    c.sc3 = rho * g.th * g.sq; c.sc4 = rho * g.th * g.th; c.sc5 = c.sc4 * g.sq;
    QK[0] = c.QKKK * c.sc3; QK[1] = c.QKKO * c.sc3; QK[2] = c.QKOO * c.sc3; QK[3] = c.QKzz * c.sc3;
    RK[0] = c.RKK * c.sc4; RK[1] = c.ROK * c.sc4;
    SK = c.Ss * c.sc5;
}

// Reverse of closure_p<K>: adjoints (QKb, RKb, SKb) -> gb, sbb, Qb[0].
template <int K>
__device__ __forceinline__ void closure_p_bwd(const double* Q, const DimlessP<double>& g,
                                              double sb, const CloP& c, const double* QKb,
                                              const double* RKb, double SKb, DimlessBar& gb,
                                              double& sbb, double* Qb) {
    const double a = g.a, b = g.b, d = g.d, f = g.f;
    const double wK = K == 0 ? c.wx : c.wy, wO = K == 0 ? c.wy : c.wx;
    const double vK = K == 0 ? c.vx : c.vy, vO = K == 0 ? c.vy : c.vx;
    const double yK = K == 0 ? g.yx : g.yy, yO = K == 0 ? g.yy : g.yx;
    const double P2KK = K == 0 ? c.P2xx : c.P2yy, P2OO = K == 0 ? c.P2yy : c.P2xx;
    const double P3KK = K == 0 ? c.P3xx : c.P3yy;
    const double PKK = K == 0 ? a : d;
    const double qK = K == 0 ? g.qx : g.qy;
    const double t = g.trPs, t2 = t * t;
    const double rho = Q[0];
    // re-dimensionalisation
    const double Ssb = SKb * c.sc5;
    double sc5b = SKb * c.Ss;
    const double RKKb = RKb[0] * c.sc4, ROKb = RKb[1] * c.sc4;
    double sc4b = RKb[0] * c.RKK + RKb[1] * c.ROK;
    double QKKKb = QKb[0] * c.sc3, QKKOb = QKb[1] * c.sc3, QKOOb = QKb[2] * c.sc3;
    const double QKzzb = QKb[3] * c.sc3;
    const double sc3b = QKb[0] * c.QKKK + QKb[1] * c.QKKO + QKb[2] * c.QKOO + QKb[3] * c.QKzz;
    sc4b += sc5b * g.sq;
    gb.sq += sc5b * c.sc4;
    Qb[0] += sc4b * g.th * g.th + sc3b * g.th * g.sq;
    gb.th += sc4b * 2.0 * rho * g.th + sc3b * rho * g.sq;
    gb.sq += sc3b * rho * g.th;
    // Ss = yQy isb^2 + 2 ssb t qK + (1 - ssb) Wq
    double yQyb = Ssb * c.isb * c.isb;
    double isbb = Ssb * c.yQy * 2.0 * c.isb;
    const double ssbb = Ssb * (2.0 * t * qK - c.Wq);
    double tb = Ssb * 2.0 * c.ssb * qK;
    double qKb = Ssb * 2.0 * c.ssb * t;
    const double Wqb = Ssb * (1.0 - c.ssb);
    sbb += ssbb * 0.5 / c.ssb;
    // Wq = mKK vK + mKO vO
    const double mKKb = Wqb * vK, mKOb = Wqb * vO;
    double vKb = Wqb * c.mKK, vOb = Wqb * c.mKO;
    // mKO = c1 b + c2 P2xy + c3 P3xy + 20 P4KO; mKK = c1 PKK + c2 P2KK + c3 P3KK + 20 P4KK
    double c1b = mKOb * b + mKKb * PKK;
    double c2b = mKOb * c.P2xy + mKKb * P2KK;
    double c3b = mKOb * c.P3xy + mKKb * P3KK;
    double bb = mKOb * c.c1;
    double P2xyb = mKOb * c.c2;
    double P3xyb = mKOb * c.c3;
    const double P4KOb = 20.0 * mKOb;
    double PKKb = mKKb * c.c1;
    double P2KKb = mKKb * c.c2;
    double P3KKb = mKKb * c.c3;
    const double P4KKb = 20.0 * mKKb;
    // P4KO = P2xy (P2xx + P2yy); P4KK = P2KK^2 + P2xy^2
    P2xyb += P4KOb * (c.P2xx + c.P2yy) + 2.0 * c.P2xy * P4KKb;
    double P2xxb = P4KOb * c.P2xy, P2yyb = P4KOb * c.P2xy;
    P2KKb += 2.0 * P2KK * P4KKb;
    // c3 = 20 t; c2 = 14 T2 - 6 t^2; c1 = 2 t^3 + 12 trP3 - 2 T2 t
    tb += 20.0 * c3b;
    double T2b = 14.0 * c2b - 2.0 * t * c1b;
    tb += -12.0 * t * c2b + (6.0 * t2 - 2.0 * g.T2) * c1b;
    double trP3b = 12.0 * c1b;
    // yQy = QKKK yK^2 + 2 QKKO yK yO + QKOO yO^2
    QKKKb += yQyb * yK * yK;
    QKKOb += yQyb * 2.0 * yK * yO;
    QKOOb += yQyb * yO * yO;
    double yKb = yQyb * (2.0 * c.QKKK * yK + 2.0 * c.QKKO * yO);
    double yOb = yQyb * (2.0 * c.QKKO * yK + 2.0 * c.QKOO * yO);
    // ROK = (QKKO yK + QKOO yO) isb + 2 (1 - sb) P2xy + b trPs
    QKKOb += ROKb * yK * c.isb;
    QKOOb += ROKb * yO * c.isb;
    yKb += ROKb * c.QKKO * c.isb;
    yOb += ROKb * c.QKOO * c.isb;
    isbb += ROKb * (c.QKKO * yK + c.QKOO * yO);
    sbb -= 2.0 * c.P2xy * ROKb;
    P2xyb += 2.0 * (1.0 - sb) * ROKb;
    bb += t * ROKb;
    tb += b * ROKb;
    // RKK = (QKKK yK + QKKO yO) isb + 2 (1 - sb) P2KK + PKK trPs
    QKKKb += RKKb * yK * c.isb;
    QKKOb += RKKb * yO * c.isb;
    yKb += RKKb * c.QKKK * c.isb;
    yOb += RKKb * c.QKKO * c.isb;
    isbb += RKKb * (c.QKKK * yK + c.QKKO * yO);
    sbb -= 2.0 * P2KK * RKKb;
    P2KKb += 2.0 * (1.0 - sb) * RKKb;
    PKKb += t * RKKb;
    tb += PKK * RKKb;
    sbb -= isbb * c.isb * c.isb;
    // Q_K.. = w P^2 combinations
    double wKb = 2.0 * c.P2zz * QKzzb + 2.0 * P2OO * QKOOb + 4.0 * c.P2xy * QKKOb +
                 6.0 * P2KK * QKKKb;
    double wOb = 4.0 * c.P2xy * QKOOb + 2.0 * P2KK * QKKOb;
    double P2zzb = 2.0 * wK * QKzzb;
    double P2OOb = 2.0 * wK * QKOOb;
    P2xyb += 4.0 * wO * QKOOb + 4.0 * wK * QKKOb;
    P2KKb += 2.0 * wO * QKKOb + 6.0 * wK * QKKKb;
    // map K/O selections back to x/y
    double wxb, wyb, vxb, vyb;
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
    double P3xxb = K == 0 ? P3KKb : 0.0, P3yyb = K == 0 ? 0.0 : P3KKb;
    gb.trPs += tb;
    gb.b += bb;
    // w = P* v (2x2 block)
    gb.a += wxb * c.vx;
    gb.b += wxb * c.vy + wyb * c.vx;
    gb.d += wyb * c.vy;
    vxb += wxb * a + wyb * b;
    vyb += wxb * b + wyb * d;
    // v = B^-1 q* (2x2): vx = (Byy qx - Bxy qy) iB, vy = (Bxx qy - Bxy qx) iB
    const double nxb = vxb * c.iB, nyb = vyb * c.iB;
    const double iBb = vxb * (c.Byy * g.qx - c.Bxy * g.qy) + vyb * (c.Bxx * g.qy - c.Bxy * g.qx);
    double Byyb = nxb * g.qx, Bxxb = nyb * g.qy;
    double Bxyb = -(nxb * g.qy + nyb * g.qx);
    gb.qx += nxb * c.Byy - nyb * c.Bxy;
    gb.qy += -nxb * c.Bxy + nyb * c.Bxx;
    const double detBb = -iBb * c.iB * c.iB;
    Bxxb += detBb * c.Byy;
    Byyb += detBb * c.Bxx;
    Bxyb -= 2.0 * c.Bxy * detBb;
    // B = 2 P* T2 + 4 P*^3 (2x2 block)
    gb.a += 2.0 * g.T2 * Bxxb;
    gb.b += 2.0 * g.T2 * Bxyb;
    gb.d += 2.0 * g.T2 * Byyb;
    T2b += 2.0 * (a * Bxxb + b * Bxyb + d * Byyb);
    P3xxb += 4.0 * Bxxb + trP3b;
    P3xyb += 4.0 * Bxyb;
    P3yyb += 4.0 * Byyb + trP3b;
    const double P3zzb = trP3b;
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
    gb.f += 2.0 * f * P2zzb;
    gb.b += 2.0 * b * P2yyb + (a + d) * P2xyb + 2.0 * b * P2xxb;
    gb.d += 2.0 * d * P2yyb + b * P2xyb;
    gb.a += b * P2xyb + 2.0 * a * P2xxb;
}

// Reverse of flux_p<K>: Fb -> Qb (primitives used directly), Ub (adjoint of
// the conserved vector the flux carries), QKb, RKb, SKb.
template <int K>
__device__ __forceinline__ void flux_p_bwd(const double* Q, const double* U, const double* QK,
                                           const double* RK, const double* Fb, double* Qb,
                                           double* Ub, double* QKb, double* RKb, double& SKb) {
    const double ux = Q[1], uy = Q[2];
    const double uK = K == 0 ? ux : uy, uO = K == 0 ? uy : ux;
    const double Pxx = Q[3], Pxy = Q[4], Pyy = Q[5];
    const double PKK = K == 0 ? Pxx : Pyy;
    const double qK = Q[7 + K];
    const double u2 = ux * ux + uy * uy;
    const double PuK = PKK * uK + Pxy * uO;
    const double QuK = QK[0] * uK + QK[1] * uO;
    const double QuO = QK[1] * uK + QK[2] * uO;
    const double PxK = K == 0 ? Pxx : Pxy, PyK = K == 0 ? Pxy : Pyy;
    const double gK = 2.0 * PuK + qK;
    double uKb = 0.0, uOb = 0.0, uxb = 0.0, uyb = 0.0, u2b = 0.0;
#pragma unroll
    for (int n = 0; n < NP; ++n) {
        Ub[n] += uK * Fb[n];
        uKb += Fb[n] * U[n];
    }
    // energy-like moment
    u2b += Fb[9] * (4.0 * PuK + 2.0 * qK);
    double PuKb = 4.0 * u2 * Fb[9];
    double qKb = 2.0 * u2 * Fb[9];
    const double uQub = 4.0 * Fb[9], uRb = 4.0 * Fb[9];
    SKb += Fb[9];
    uKb += uRb * RK[0] + uQub * QuK;
    uOb += uRb * RK[1] + uQub * QuO;
    double RK0b = uRb * uK, RK1b = uRb * uO;
    double QuKb = uQub * uK, QuOb = uQub * uO;
    // third moments
    uyb += Fb[8] * gK;
    uxb += Fb[7] * gK;
    const double gKb = uy * Fb[8] + ux * Fb[7];
    u2b += Fb[8] * PyK + Fb[7] * PxK;
    double PyKb = u2 * Fb[8], PxKb = u2 * Fb[7];
    const double QuYb = 2.0 * Fb[8], QuXb = 2.0 * Fb[7];
    if (K == 0) {
        QuKb += QuXb; QuOb += QuYb;
        RK0b += Fb[7]; RK1b += Fb[8];
    } else {
        QuOb += QuXb; QuKb += QuYb;
        RK1b += Fb[7]; RK0b += Fb[8];
    }
    PuKb += 2.0 * gKb;
    qKb += gKb;
    // second moments
    double QK0b = 0.0, QK1b = 0.0, QK2b = 0.0;
    const double QK3b = Fb[6];
    uyb += 2.0 * PyK * Fb[5];
    PyKb += 2.0 * uy * Fb[5];
    const double QyyKb = Fb[5];
    uxb += PyK * Fb[4];
    PyKb += ux * Fb[4];
    uyb += PxK * Fb[4];
    PxKb += uy * Fb[4];
    QK1b += Fb[4];
    uxb += 2.0 * PxK * Fb[3];
    PxKb += 2.0 * ux * Fb[3];
    const double QxxKb = Fb[3];
    if (K == 0) { QK0b += QxxKb; QK2b += QyyKb; } else { QK2b += QxxKb; QK0b += QyyKb; }
    // momentum and the P_iK of the second moments
    double Pxxb = 0.0, Pxyb = 0.0, Pyyb = 0.0;
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
    const double PKKb = PuKb * uK;
    Pxyb += PuKb * uO;
    if (K == 0) Pxxb += PKKb; else Pyyb += PKKb;
    uxb += 2.0 * ux * u2b + (K == 0 ? uKb : uOb);
    uyb += 2.0 * uy * u2b + (K == 0 ? uOb : uKb);
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
__device__ __forceinline__ void prim2cons_p_bwd(const double* Q, const double* Ub, double* Qb) {
    const double rho = Q[0], ux = Q[1], uy = Q[2];
    const double Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const double qx = Q[7], qy = Q[8];
    const double u2 = ux * ux + uy * uy;
    const double trP = Pxx + Pyy + Pzz;
    const double Pux = Pxx * ux + Pxy * uy, Puy = Pxy * ux + Pyy * uy;
    const double e = rho * u2 + trP;
    double rhob = Ub[0], uxb = 0.0, uyb = 0.0, u2b = 0.0, trPb = 0.0;
    double Pxxb = Ub[3], Pxyb = Ub[4], Pyyb = Ub[5], Pzzb = Ub[6];
    double qxb = Ub[7], qyb = Ub[8];
    // U9 = rho u2^2 + 2 u2 trP + 4 uPu + 4 uq + R
    rhob += Ub[9] * u2 * u2;
    u2b += Ub[9] * (2.0 * rho * u2 + 2.0 * trP);
    trPb += 2.0 * u2 * Ub[9];
    const double uPub = 4.0 * Ub[9], uqb = 4.0 * Ub[9];
    // U7, U8 = u_i e + 2 (P u)_i + q_i
    uyb += Ub[8] * e;
    uxb += Ub[7] * e;
    const double eb = Ub[8] * uy + Ub[7] * ux;
    double Puyb = 2.0 * Ub[8], Puxb = 2.0 * Ub[7];
    // second moments rho u_i u_j + P_ij
    rhob += Ub[5] * uy * uy + Ub[4] * ux * uy + Ub[3] * ux * ux + Ub[2] * uy + Ub[1] * ux;
    uyb += 2.0 * rho * uy * Ub[5] + rho * ux * Ub[4] + rho * Ub[2];
    uxb += rho * uy * Ub[4] + 2.0 * rho * ux * Ub[3] + rho * Ub[1];
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
    uxb += 2.0 * ux * u2b;
    uyb += 2.0 * uy * u2b;
    Qb[0] += rhob; Qb[1] += uxb; Qb[2] += uyb;
    Qb[3] += Pxxb; Qb[4] += Pxyb; Qb[5] += Pyyb; Qb[6] += Pzzb;
    Qb[7] += qxb; Qb[8] += qyb; Qb[9] += Ub[9];
}

// Reverse of face_eval_p<K>: adjoints of (U, F, lmin, lmax) of one face
// state -> Qb (added).
template <int K>
__device__ __forceinline__ void face_eval_p_bwd(const double* Q, double sl, double kw,
                                                const double* Ubar_in, const double* Fb,
                                                double lminb, double lmaxb, double* Qb) {
    DimlessP<double> g;
    dimless_p(Q, g);
    const double sb = clamp_sigma(g.sig, sl);
    CloP c;
    double QK[4], RK[2], SK;
    closure_p_fwd<K>(Q, g, sb, c, QK, RK, SK);
    double U[NP];
    prim2cons_p(Q, U);
    double lp, lm;
    lam_p<double, K>(g, sb, lp, lm);
    DimlessBar gb;
    gb.zero();
    double sbb = 0.0;
    // lmax = u_K + k lp sq, lmin = u_K + k lm sq
    Qb[1 + K] += lmaxb + lminb;
    gb.sq += kw * (lmaxb * lp + lminb * lm);
    const double lpb = lmaxb * kw * g.sq, lmb = lminb * kw * g.sq;
    // flux
    double Ub[NP];
#pragma unroll
    for (int n = 0; n < NP; ++n) Ub[n] = Ubar_in[n];
    double QKb[4] = {0.0, 0.0, 0.0, 0.0}, RKb[2] = {0.0, 0.0}, SKb = 0.0;
    flux_p_bwd<K>(Q, U, QK, RK, Fb, Qb, Ub, QKb, RKb, SKb);
    prim2cons_p_bwd(Q, Ub, Qb);
    closure_p_bwd<K>(Q, g, sb, c, QKb, RKb, SKb, gb, sbb, Qb);
    lam_p_bwd<K>(g, sb, lpb, lmb, gb, sbb);
    if (!(g.sig < sl) && !(g.sig > 1.0)) gb.sig += sbb;
    dimless_p_bwd(Q, g, gb, Qb);
}

// One face state evaluated once and reversed: the primal outputs (U, F,
// lmin, lmax) are handed to `outadj`, which returns their adjoints (the
// numerical-flux reverse needs both states of the face); the reverse then
// reuses the primal intermediates.  Adds to Qb.
template <int K, class OutAdj>
__device__ __forceinline__ void face_side_adj(const double* Q, double sl, double kw,
                                              OutAdj&& outadj, double* Qb) {
    DimlessP<double> g;
    dimless_p(Q, g);
    const double sb = clamp_sigma(g.sig, sl);
    CloP c;
    double QK[4], RK[2], SK;
    closure_p_fwd<K>(Q, g, sb, c, QK, RK, SK);
    double U[NP], F[NP];
    prim2cons_p(Q, U);
    flux_p<double, K>(Q, U, QK, RK, SK, F);
    LamP L;
    lam_p_fwd<K>(g, sb, L);
    const double lmax = Q[1 + K] + kw * L.lp * g.sq;
    const double lmin = Q[1 + K] + kw * L.lm * g.sq;
    double Ub[NP], Fb[NP], lminb, lmaxb;
    outadj(U, F, lmin, lmax, Ub, Fb, lminb, lmaxb);
    DimlessBar gb;
    gb.zero();
    double sbb = 0.0;
    Qb[1 + K] += lmaxb + lminb;
    gb.sq += kw * (lmaxb * L.lp + lminb * L.lm);
    const double lpb = lmaxb * kw * g.sq, lmb = lminb * kw * g.sq;
    double QKb[4] = {0.0, 0.0, 0.0, 0.0}, RKb[2] = {0.0, 0.0}, SKb = 0.0;
    flux_p_bwd<K>(Q, U, QK, RK, Fb, Qb, Ub, QKb, RKb, SKb);
    prim2cons_p_bwd(Q, Ub, Qb);
    closure_p_bwd<K>(Q, g, sb, c, QKb, RKb, SKb, gb, sbb, Qb);
    lam_p_rev<K>(L, sb, lpb, lmb, gb, sbb);
    if (!(g.sig < sl) && !(g.sig > 1.0)) gb.sig += sbb;
    dimless_p_bwd(Q, g, gb, Qb);
}

// Reverse of source_p with the local relaxation time tau_p: W = adjoint of
// the source vector C -> Qb; returns the adjoint of tau_ref.
__device__ __forceinline__ double source_p_bwd(int model, double tau_ref, double rho_ref,
                                               double T_ref, const double* Q, const double* W,
                                               double* Qb) {
    const double rho = Q[0], ux = Q[1], uy = Q[2];
    const double Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const double qx = Q[7], qy = Q[8], R = Q[9];
    const double tau = tau_p(model, tau_ref, rho_ref, T_ref, Q);
    const double p = (Pxx + Pyy + Pzz) / 3.0;
    const double Pux = Pxx * ux + Pxy * uy, Puy = Pxy * ux + Pyy * uy;
    const double uPu = ux * Pux + uy * Puy, uq = ux * qx + uy * qy, u2 = ux * ux + uy * uy;
    // C_k = -N_k / tau
    const double N[10] = {0.0, 0.0, 0.0, Pxx - p, Pxy, Pyy - p, Pzz - p,
                          2.0 * Pux + qx - 2.0 * ux * p, 2.0 * Puy + qy - 2.0 * uy * p,
                          (4.0 * uPu + 4.0 * uq + R) - (4.0 * u2 * p + 15.0 * p * p / rho)};
    double WN = 0.0;
#pragma unroll
    for (int k = 3; k < NP; ++k) WN += W[k] * N[k];
    const double itau = 1.0 / tau;
    const double taub = WN * itau * itau;
    double n[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) n[k] = -W[k] * itau;
    double rhob = 0.0, uxb = 0.0, uyb = 0.0, pb = 0.0, u2b = 0.0;
    double Pxxb = n[3], Pxyb = n[4], Pyyb = n[5], Pzzb = n[6];
    pb -= n[3] + n[5] + n[6];
    double qxb = n[7], qyb = n[8], Rb = n[9];
    const double uPub = 4.0 * n[9], uqb = 4.0 * n[9];
    u2b -= 4.0 * p * n[9];
    pb -= (4.0 * u2 + 30.0 * p / rho) * n[9];
    rhob += 15.0 * p * p / (rho * rho) * n[9];
    double Puxb = 2.0 * n[7], Puyb = 2.0 * n[8];
    uxb -= 2.0 * p * n[7];
    uyb -= 2.0 * p * n[8];
    pb -= 2.0 * ux * n[7] + 2.0 * uy * n[8];
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
    uxb += 2.0 * ux * u2b;
    uyb += 2.0 * uy * u2b;
    double tau_refb;
    if (model == 1) {
        tau_refb = taub;
    } else {
        // tau = tau_ref (rho_ref / rho) sqrt(T_ref / T), T = tr P / (3 rho)
        const double T = (Pxx + Pyy + Pzz) / (3.0 * rho);
        const double Tb = -taub * tau / (2.0 * T);
        rhob += -taub * tau / rho - Tb * T / rho;
        const double trb = Tb / (3.0 * rho);
        Pxxb += trb; Pyyb += trb; Pzzb += trb;
        tau_refb = taub * tau / tau_ref;
    }
    Pxxb += pb / 3.0; Pyyb += pb / 3.0; Pzzb += pb / 3.0;
    Qb[0] += rhob; Qb[1] += uxb; Qb[2] += uyb;
    Qb[3] += Pxxb; Qb[4] += Pxyb; Qb[5] += Pyyb; Qb[6] += Pzzb;
    Qb[7] += qxb; Qb[8] += qyb; Qb[9] += Rb;
    return tau_refb;
}

// Reverse of the planar primitive recovery Q = prim(U): Qb -> Ub (added).
__device__ __forceinline__ void cons2prim_p_bwd(const double* Q, const double* Qbar, double* Ub) {
    const double rho = Q[0], ux = Q[1], uy = Q[2];
    const double Pxx = Q[3], Pxy = Q[4], Pyy = Q[5], Pzz = Q[6];
    const double qx = Q[7], qy = Q[8];
    const double u2 = ux * ux + uy * uy, trP = Pxx + Pyy + Pzz;
    double rhob = Qbar[0], uxb = Qbar[1], uyb = Qbar[2];
    double Pxxb = Qbar[3], Pxyb = Qbar[4], Pyyb = Qbar[5], Pzzb = Qbar[6];
    double qxb = Qbar[7], qyb = Qbar[8];
    const double Rb = Qbar[9];
    // R = U9 - rho u2^2 - 2 u2 trP - 4 uPu - 4 uq
    Ub[9] += Rb;
    rhob -= Rb * u2 * u2;
    double u2b = -Rb * (2.0 * rho * u2 + 2.0 * trP);
    double trPb = -2.0 * u2 * Rb;
    const double uPub = -4.0 * Rb, uqb = -4.0 * Rb;
    uxb += uqb * qx;
    qxb += uqb * ux;
    uyb += uqb * qy;
    qyb += uqb * uy;
    uxb += uPub * (2.0 * ux * Pxx + 2.0 * uy * Pxy);
    uyb += uPub * (2.0 * ux * Pxy + 2.0 * uy * Pyy);
    Pxxb += uPub * ux * ux;
    Pxyb += 2.0 * uPub * ux * uy;
    Pyyb += uPub * uy * uy;
    // q_i = U_i - rho u_i u2 - u_i trP - 2 (P u)_i
    Ub[7] += qxb;
    Ub[8] += qyb;
    rhob -= qxb * ux * u2 + qyb * uy * u2;
    uxb -= qxb * (rho * u2 + trP + 2.0 * Pxx) + 2.0 * qyb * Pxy;
    uyb -= qyb * (rho * u2 + trP + 2.0 * Pyy) + 2.0 * qxb * Pxy;
    u2b -= qxb * rho * ux + qyb * rho * uy;
    trPb -= qxb * ux + qyb * uy;
    Pxxb -= 2.0 * qxb * ux;
    Pxyb -= 2.0 * qxb * uy + 2.0 * qyb * ux;
    Pyyb -= 2.0 * qyb * uy;
    Pxxb += trPb; Pyyb += trPb; Pzzb += trPb;
    uxb += 2.0 * ux * u2b;
    uyb += 2.0 * uy * u2b;
    // P_ij = U_ij - rho u_i u_j
    Ub[6] += Pzzb;
    Ub[5] += Pyyb;
    Ub[4] += Pxyb;
    Ub[3] += Pxxb;
    rhob -= Pyyb * uy * uy + Pxyb * ux * uy + Pxxb * ux * ux;
    uyb -= 2.0 * rho * uy * Pyyb + rho * ux * Pxyb;
    uxb -= rho * uy * Pxyb + 2.0 * rho * ux * Pxxb;
    // u_i = U_i / rho
    Ub[2] += uyb / rho;
    Ub[1] += uxb / rho;
    rhob -= (uyb * uy + uxb * ux) / rho;
    Ub[0] += rhob;
}

// Shared limiter with its selected field and the partial derivatives of
// phi_{k*} with respect to dm and dp (zero when no field sets phi).
struct PhiAdj {
    double phi, ddm, ddp;
    int ks;
};

template <int NF>
__device__ __forceinline__ PhiAdj phi_adj(const double* qm, const double* q0, const double* qp,
                                          int lim) {
    PhiAdj r{1.0, 0.0, 0.0, -1};
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const double dm = q0[k] - qm[k], dp = qp[k] - q0[k];
        const double pk = phi_field(dm, dp, lim);
        if (pk < r.phi) {
            r.phi = pk;
            r.ks = k;
            if (mul_rn(dm, dp) > 0.0) {
                if (lim == 1) {
                    const double s = dm * dm + dp * dp;
                    r.ddm = 2.0 * dp * (dp * dp - dm * dm) / (s * s);
                    r.ddp = 2.0 * dm * (dm * dm - dp * dp) / (s * s);
                } else {
                    const double am = fabs(dm), ap = fabs(dp), s = am + ap;
                    const double sm = dm > 0.0 ? 1.0 : -1.0, sp = dp > 0.0 ? 1.0 : -1.0;
                    if (am < ap) {
                        r.ddm = sm * 2.0 * ap / (s * s);
                        r.ddp = -sp * 2.0 * am / (s * s);
                    } else {
                        r.ddp = sp * 2.0 * am / (s * s);
                        r.ddm = -sm * 2.0 * ap / (s * s);
                    }
                }
            } else {
                r.ddm = r.ddp = 0.0;      // constant branch
            }
        }
    }
    return r;
}

// Reverse of the MUSCL face value qf = q0 + hs (phi cen), cen = (qp - qm)/2
// (computed as ((q0 - qm) + (qp - q0))/2), with phi = phi_{k*}(q0 - qm,
// qp - q0): adjoint qfb -> contributions to the three stencil cells.  A
// field that is flat across the stencil (both differences exactly zero)
// has the zero slope, whose derivative is zero (the same choice as the
// oracle's tangent): a perturbation of a flat stencil is limited, not
// passed on with phi = 1.
template <int NF>
__device__ __forceinline__ void muscl_bwd(const double* qm, const double* q0, const double* qp,
                                          const PhiAdj& ph, double hs, const double* qfb,
                                          double* bm, double* b0, double* bp) {
    double phib = 0.0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const double dm = q0[k] - qm[k], dp = qp[k] - q0[k];
        b0[k] += qfb[k];
        if (dm == 0.0 && dp == 0.0) continue;
        const double cen = 0.5 * (dm + dp);
        const double cb = hs * ph.phi * qfb[k];
        bm[k] -= 0.5 * cb;
        bp[k] += 0.5 * cb;
        phib += hs * cen * qfb[k];
    }
    if (ph.ks >= 0) {
        const double dmb = phib * ph.ddm, dpb = phib * ph.ddp;
#pragma unroll
        for (int k = 0; k < NF; ++k)
            if (k == ph.ks) {
                b0[k] += dmb - dpb;
                bm[k] -= dmb;
                bp[k] += dpb;
            }
    }
}

}  // namespace adj
}  // namespace mxe
