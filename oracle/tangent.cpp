/*
 * tangent.cpp -- forward-mode tangent of the oracle (TEST INFRASTRUCTURE ONLY).
 *
 * The oracle's own source (maxent_oracle.c) is compiled a second time with
 * its arithmetic type replaced by a dual number v + d*eps (eps^2 = 0): every
 * elementary operation carries its first derivative along by the chain rule,
 * so one run gives the primal trajectory (bitwise the plain oracle's: the
 * value parts follow exactly the same operations in the same order) and its
 * directional derivative J.v, exact up to rounding.  Branches (limiter cases,
 * sigma clamp, HLL upwinding, min/max) are taken on the value parts, so the
 * tangent is that of the discrete map on the branch the primal follows:
 * minmod and min/max differentiate the selected argument, an active clamp
 * has derivative zero.  Used to check the CUDA adjoint (reverse mode) by
 * the identity <ybar, J v> = <J^T ybar, v>.
 *
 * Only the tests may load this library.  It shares no code with the CUDA
 * library.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

namespace ortan {

struct dual {
    double v, d;
    dual() : v(0.0), d(0.0) {}
    dual(double x) : v(x), d(0.0) {}
    dual(double x, double dx) : v(x), d(dx) {}
    dual& operator+=(const dual& b) { d += b.d; v += b.v; return *this; }
    dual& operator-=(const dual& b) { d -= b.d; v -= b.v; return *this; }
    dual& operator*=(const dual& b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
    dual& operator/=(const dual& b) { *this = dual(v / b.v, (d * b.v - v * b.d) / (b.v * b.v)); return *this; }
};

inline dual operator+(const dual& a, const dual& b) { return dual(a.v + b.v, a.d + b.d); }
inline dual operator-(const dual& a, const dual& b) { return dual(a.v - b.v, a.d - b.d); }
inline dual operator-(const dual& a) { return dual(-a.v, -a.d); }
inline dual operator*(const dual& a, const dual& b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline dual operator/(const dual& a, const dual& b) {
    return dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline bool operator<(const dual& a, const dual& b) { return a.v < b.v; }
inline bool operator>(const dual& a, const dual& b) { return a.v > b.v; }
inline bool operator<=(const dual& a, const dual& b) { return a.v <= b.v; }
inline bool operator>=(const dual& a, const dual& b) { return a.v >= b.v; }
inline bool operator==(const dual& a, const dual& b) { return a.v == b.v; }
inline bool operator!=(const dual& a, const dual& b) { return a.v != b.v; }

// d sqrt(x) = dx / (2 sqrt x); at x = 0 with dx = 0 the derivative is 0
inline dual sqrt(const dual& a) {
    double s = ::sqrt(a.v);
    return dual(s, a.d == 0.0 ? 0.0 : a.d / (2.0 * s));
}
inline dual exp(const dual& a) {
    double e = ::exp(a.v);
    return dual(e, a.d * e);
}
inline dual log(const dual& a) { return dual(::log(a.v), a.d / a.v); }
// x^p for a constant exponent p
inline dual pow(const dual& a, double p) {
    return dual(::pow(a.v, p), a.d == 0.0 ? 0.0 : p * ::pow(a.v, p - 1.0) * a.d);
}
inline dual fabs(const dual& a) { return a.v < 0.0 ? -a : a; }
inline bool isnan(const dual& a) { return a.v != a.v; }
// the value alone (its derivative dropped)
inline dual value_of(const dual& a) { return dual(a.v, 0.0); }

}  // namespace ortan

namespace ortan {
#define OR_REAL ortan::dual
#define OR_VALUE(x) value_of(x)
#define OR_TANGENT_BUILD
#include "maxent_oracle.c"
#undef OR_TANGENT_BUILD
#undef OR_VALUE
#undef OR_REAL
}  // namespace ortan

extern "C" {

/* Size in bytes of the dual-number configuration the caller passes (the
 * double layout of or_cfg with each physical quantity widened to (v, d)). */
size_t or_tangent_cfg_size(void) { return sizeof(ortan::or_cfg); }

/* n steps of the prescribed sizes dts from U (interior nx*ny*nf, AoS) in
 * the direction dU of the state and the directions carried by the dual
 * configuration (imposed boundary states, tau_ref, rho_ref, T_ref).
 * Uout receives the primal state, dUout its tangent.  The step sizes are
 * constants (not differentiated).  Returns 0. */
int or_tangent_run(const ortan::or_cfg *c, const double *U, const double *dU, int nsteps,
                   const double *dts, double *Uout, double *dUout) {
    const int nf = c->system == 5 ? 5 : 14;
    const size_t n = (size_t)c->nx * c->ny * nf;
    ortan::dual *X = (ortan::dual *)malloc(n * sizeof(ortan::dual));
    for (size_t k = 0; k < n; ++k) X[k] = ortan::dual(U[k], dU[k]);
    for (int s = 0; s < nsteps; ++s) ortan::or_step(c, X, ortan::dual(dts[s]));
    for (size_t k = 0; k < n; ++k) {
        Uout[k] = X[k].v;
        dUout[k] = X[k].d;
    }
    free(X);
    return 0;
}

/* Tangent of the residual L(U) = -div F + C (one evaluation, boundary
 * conditions applied as in a step): Lout and dLout are nx*ny*nf. */
int or_tangent_residual(const ortan::or_cfg *c, const double *U, const double *dU,
                        double *Lout, double *dLout) {
    const int nf = c->system == 5 ? 5 : 14;
    ortan::blk b;
    ortan::blk_init(c, &b, 0, 0, c->nx, c->ny);
    const size_t nb = (size_t)b.W * b.H * nf;
    ortan::dual *A = (ortan::dual *)calloc(nb, sizeof(ortan::dual));
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
            for (int k = 0; k < nf; ++k) {
                size_t o = ((size_t)j * c->nx + i) * nf + k;
                ortan::cell(&b, A, i, j)[k] = ortan::dual(U[o], dU[o]);
            }
    const size_t n = (size_t)c->nx * c->ny * nf;
    ortan::dual *L = (ortan::dual *)malloc(n * sizeof(ortan::dual));
    ortan::fill_bc(c, &b, A);
    ortan::residual_region(c, &b, A, 0, c->nx, 0, c->ny, L);
    for (size_t k = 0; k < n; ++k) {
        Lout[k] = L[k].v;
        dLout[k] = L[k].d;
    }
    free(L);
    free(A);
    free(b.gp);
    return 0;
}

}  // extern "C"
