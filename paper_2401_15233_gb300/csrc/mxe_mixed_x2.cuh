// mxe_mixed_x2.cuh -- pieces of the mixed-precision path shared by the 2D
// packed stage kernel and the batched tube kernel: the shared limiter by
// ratios, the face flux of a face evaluated as one packed FP32 pair of face
// states (planar state), its FP64 re-evaluation, and the exact FP32 -> FP64
// conversion of the accumulator's increments.
#pragma once
#include "mxe_mixed.cuh"
#include "mxe_planar_x2.cuh"

namespace mxe {

// One field's contribution to the shared limiter of one direction, tracked
// as the ratio r = min(|dm|, |dp|) / max(|dm|, |dp|) of the most stringent
// field so far (n / x).  Both limiters are increasing in r on [0, 1]
// (minmod 2r/(1+r), van Albada 2r/(1+r^2)), so the field with the smallest
// r sets phi, and ratios are compared cross-multiplied: one division per
// cell and direction instead of one per field.  Opposite signs give r = 0;
// a field with dm = dp = 0, or flat by the tolerance test, never lowers phi.
template <int NF>
__device__ __forceinline__ void phi_ratio_step(float dm, float dp, float w0,
                                               const FlatRef<float>& fr, int k, float& n,
                                               float& x) {
    const float am = fabsf(dm), ap = fabsf(dp);
    const float mx = fmaxf(am, ap);
    const float mn = dm * dp > 0.0f ? fminf(am, ap) : 0.0f;
    if (mx > 0.0f && mn * x < n * mx) {
        if (!(mx <= FLAT_REL_F32 * fabsf(w0) || field_flat<NF>(fr, k, mx))) {
            n = mn;
            x = mx;
        }
    }
}
__device__ __forceinline__ float phi_of_ratio(float n, float x, int lim) {
    return lim == 1 ? __fdividef(2.0f * n * x, n * n + x * x) : __fdividef(2.0f * n, n + x);
}

// The same for one direction (stride 1: x, stride BX: y).
template <int NF, int NBOX>
__device__ __forceinline__ float phi_one_m(const float* W, int c, int stride, int lim) {
    const FlatRef<float> fr = flat_ref<NF>(W + c, NBOX);
    float n = 1.0f, x = 1.0f;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * NBOX + c;
        const float w0 = w[0];
        phi_ratio_step<NF>(w0 - w[-stride], w[stride] - w0, w0, fr, k, n, x);
    }
    return phi_of_ratio(n, x, lim);
}

// FP64 face flux of a face whose packed FP32 evaluation found an
// ill-conditioned closure in either face state: both states are evaluated
// again in FP64 (kept out of line and called with the two input states by
// value, so that nothing else is live across the call).
template <int NF>
struct FacePairIn {
    float q[2 * NF];
};
template <int NF>
struct FaceFluxOut {
    float f[NF];
};
template <int K>
__device__ __noinline__ FaceFluxOut<NP> face_flux_fp64(FacePairIn<NP> in, double sl, double kw,
                                                       int flux) {
    constexpr int NF = NP;
    double QL[NF], QR[NF], UL[NF], UR[NF], FL[NF], FR[NF], lminL, lmaxL, lminR, lmaxR;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        QL[k] = (double)in.q[k];
        QR[k] = (double)in.q[NF + k];
    }
    PhysPlanar::face<double, K>(QL, sl, kw, UL, FL, lminL, lmaxL);
    PhysPlanar::face<double, K>(QR, sl, kw, UR, FR, lminR, lmaxR);
    FaceFluxOut<NF> r;
    if (flux == 1) {
        double sp = fmax(fmax(fabs(lminL), fabs(lmaxL)), fmax(fabs(lminR), fabs(lmaxR)));
#pragma unroll
        for (int k = 0; k < NF; ++k) r.f[k] = (float)(0.5 * (FL[k] + FR[k]) - 0.5 * sp * (UR[k] - UL[k]));
        return r;
    }
    double SL = fmin(lminL, lminR), SR = fmax(lmaxL, lmaxR);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        double f;
        if (SL >= 0.0) f = FL[k];
        else if (SR <= 0.0) f = FR[k];
        else f = (SR * FL[k] - SL * FR[k] + SL * SR * (UR[k] - UL[k])) / (SR - SL);
        r.f[k] = (float)f;
    }
    return r;
}

// Both face states of the face between box cells cl and cl + stride along K
// (planar state), evaluated as one packed FP32 pair (left state in lane x,
// right in lane y): the reconstruction shares the four stencil cells, and
// no face state is staged in shared memory.  A face with an ill-conditioned
// closure in either state (the policy of face_state_m) takes its flux from
// face_flux_fp64 instead.
template <int K, int NBOX>
__device__ __forceinline__ void face_flux_x2(const float* W, int cl, int stride, float phl,
                                             float phr, const ParamsT<float>& p,
                                             const MixedPolicy& mp, double sl64, double kw64,
                                             float* F, unsigned& nflag) {
    using namespace x2;
    constexpr int NF = NP;
    v2 Q[NF];
    const v2 hp = make_float2(0.25f * phl, -0.25f * phr);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * NBOX + cl;
        const float wm = w[-stride], w0 = w[0], w1 = w[stride], w2 = w[2 * stride];
        Q[k] = fma(hp, sub(make_float2(w1, w2), make_float2(wm, w0)), make_float2(w0, w1));
    }
    v2 U[NF], Fv[NF], lmin, lmax, sig, det;
    face_eval_x2<K>(Q, p.sigma_lim, p.k_ws, U, Fv, lmin, lmax, sig, det);
    if (p.flux == 1) {
        float s = fmaxf(fmaxf(fabsf(lmin.x), fabsf(lmax.x)), fmaxf(fabsf(lmin.y), fabsf(lmax.y)));
#pragma unroll
        for (int k = 0; k < NF; ++k)
            F[k] = 0.5f * (Fv[k].x + Fv[k].y) - 0.5f * s * (U[k].y - U[k].x);
    } else {
        float SL = fminf(lmin.x, lmin.y), SR = fmaxf(lmax.x, lmax.y);
        if (SL >= 0.0f) {
#pragma unroll
            for (int k = 0; k < NF; ++k) F[k] = Fv[k].x;
        } else if (SR <= 0.0f) {
#pragma unroll
            for (int k = 0; k < NF; ++k) F[k] = Fv[k].y;
        } else {
            float inv = 1.0f / (SR - SL);
            float cl_ = SR * inv, cr_ = -SL * inv, cu = SL * SR * inv;
#pragma unroll
            for (int k = 0; k < NF; ++k)
                F[k] = cl_ * Fv[k].x + cr_ * Fv[k].y + cu * (U[k].y - U[k].x);
        }
    }
    if (mp.sig_lo > 0.0f || mp.sig_hi < 1.0f || mp.det_min > 0.0f) {
        const bool fx = (sig.x >= p.sigma_lim && sig.x < mp.sig_lo) || sig.x > mp.sig_hi ||
                        det.x < mp.det_min || !(sig.x == sig.x);
        const bool fy = (sig.y >= p.sigma_lim && sig.y < mp.sig_lo) || sig.y > mp.sig_hi ||
                        det.y < mp.det_min || !(sig.y == sig.y);
        nflag += (fx ? 1u : 0u) + (fy ? 1u : 0u);
        if (__any_sync(__activemask(), fx || fy) && (fx || fy)) {
            FacePairIn<NF> in;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                in.q[k] = Q[k].x;
                in.q[NF + k] = Q[k].y;
            }
            FaceFluxOut<NF> r = face_flux_fp64<K>(in, sl64, kw64, p.flux);
#pragma unroll
            for (int k = 0; k < NF; ++k) F[k] = r.f[k];
        }
    }
}

// Exact FP32 -> FP64 conversion by integer operations (GB300's FP64 pipe
// retires 2 operations per clock per SM; a conversion there costs as much as
// the accumulator add itself).  The exponent is re-biased by 1023 - 127 and
// the mantissa shifted into place; zero and the values the FP32 stage flushes
// to zero map to a signed zero, infinities and NaNs keep their class.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u, em = b & 0x7fffffffu;
    unsigned hi = sign | ((em >> 3) + (896u << 20));
    unsigned lo = em << 29;
    if (em < 0x00800000u) hi = sign, lo = 0u;                            // zero (FTZ)
    if (em >= 0x7f800000u) hi = sign | 0x7ff00000u | ((em >> 3) & 0xfffffu);   // inf, NaN
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace mxe
