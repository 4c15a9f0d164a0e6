// mxe_policy.cuh -- physics policies of the 2D stage kernels: the general
// 14-moment state and the planar state (z-odd moments identically zero,
// ten active fields).  A policy supplies the number of active fields, their
// positions in the 14-field conserved layout, and the point functions.
#pragma once
#include "mxe_planar.cuh"

namespace mxe {

template <class T>
struct ParamsT {
    T sigma_lim, k_ws;
    int flux, limiter, order;
    int tau_model;
    T tau_ref, rho_ref, T_ref;
    int src_implicit;           // point-implicit source (relax after each stage)
};

template <class T>
__host__ __device__ inline ParamsT<T> make_params(const SchemeParams& sp, const RelaxParams& rp) {
    ParamsT<T> p;
    p.sigma_lim = T(sp.sigma_lim);
    p.k_ws = T(sp.k_ws);
    p.flux = sp.flux;
    p.limiter = sp.limiter;
    p.order = sp.order;
    p.tau_model = rp.model;
    p.tau_ref = T(rp.tau_ref);
    p.rho_ref = T(rp.rho_ref);
    p.T_ref = T(rp.T_ref);
    p.src_implicit = rp.implicit;
    return p;
}

struct PhysGeneral {
    static constexpr int NF = 14;
    static __host__ __device__ constexpr int ufield(int k) { return k; }
    static __device__ __forceinline__ void cons2prim_rn(const double* U, double* Q) {
        cons2prim14_rn(U, Q);
    }
    // fused, one reciprocal (the mixed path's FP64 re-sync)
    static __device__ __forceinline__ void cons2prim_fast(const double* U, double* Q) {
        cons2prim14(U, Q);
    }
    template <class T, int K>
    static __device__ __forceinline__ void face(const T* Q, T sl, T kw, T* U, T* F, T& lo, T& hi) {
        face_eval14<T, K>(Q, sl, kw, U, F, lo, hi);
    }
    // with the conditioning of the closure (raw sigma, det P*)
    template <class T, int K>
    static __device__ __forceinline__ void face_c(const T* Q, T sl, T kw, T* U, T* F, T& lo,
                                                  T& hi, T& sig, T& det) {
        face_eval14<T, K>(Q, sl, kw, U, F, lo, hi, sig, det);
    }
    template <class T>
    static __device__ __forceinline__ void source(const T* Q, T tau, T* C) { source14(Q, tau, C); }
    template <class T>
    static __device__ __forceinline__ T tau(const ParamsT<T>& p, const T* Q) {
        if (p.tau_model == 1) return p.tau_ref;
        T Tt = (Q[4] + Q[7] + Q[9]) / (T(3) * Q[0]);
        return p.tau_ref * (p.rho_ref / Q[0]) * M<T>::sqrt_(p.T_ref / Tt);
    }
    template <class T>
    static __device__ __forceinline__ void rates(const T* Q, T sl, T kw, T& ax, T& ay) {
        Dimless14<T> d;
        dimless14(Q, d);
        ax = amax14<T, 0>(Q, d, sl, kw);
        ay = amax14<T, 1>(Q, d, sl, kw);
    }
    // x rate alone (1D problems)
    template <class T>
    static __device__ __forceinline__ T rate_x(const T* Q, T sl, T kw) {
        Dimless14<T> d;
        dimless14(Q, d);
        return amax14<T, 0>(Q, d, sl, kw);
    }
    static __device__ __forceinline__ void increment(const float* W, const float* dU, float* Wn) {
        prim_increment14(W, dU, Wn);
    }
    static __device__ __forceinline__ void relax_cons(double* U, const double* Q, double tau,
                                                      double h) {
        relax14_cons(U, Q, tau, h);
    }
    template <class T>
    static __device__ __forceinline__ void relax_prim(T* W, T g, T* N) {
        relax14_prim(W, g, N);
    }
    template <class T>
    static __device__ __forceinline__ bool nonpositive(const T* Q) {
        return Q[0] <= T(0) || Q[4] <= T(0) || Q[7] <= T(0) || Q[9] <= T(0);
    }
};

struct PhysPlanar {
    static constexpr int NF = NP;
    static __host__ __device__ constexpr int ufield(int k) { return planar_field(k); }
    static __device__ __forceinline__ void cons2prim_rn(const double* U, double* Q) {
        cons2prim_p_rn(U, Q);
    }
    static __device__ __forceinline__ void cons2prim_fast(const double* U, double* Q) {
        cons2prim_p(U, Q);
    }
    template <class T, int K>
    static __device__ __forceinline__ void face(const T* Q, T sl, T kw, T* U, T* F, T& lo, T& hi) {
        face_eval_p<T, K>(Q, sl, kw, U, F, lo, hi);
    }
    template <class T, int K>
    static __device__ __forceinline__ void face_c(const T* Q, T sl, T kw, T* U, T* F, T& lo,
                                                  T& hi, T& sig, T& det) {
        face_eval_p<T, K>(Q, sl, kw, U, F, lo, hi, sig, det);
    }
    template <class T>
    static __device__ __forceinline__ void source(const T* Q, T tau, T* C) { source_p(Q, tau, C); }
    template <class T>
    static __device__ __forceinline__ T tau(const ParamsT<T>& p, const T* Q) {
        return tau_p(p.tau_model, p.tau_ref, p.rho_ref, p.T_ref, Q);
    }
    template <class T>
    static __device__ __forceinline__ void rates(const T* Q, T sl, T kw, T& ax, T& ay) {
        DimlessP<T> g;
        dimless_p(Q, g);
        ax = amax_p<T, 0>(Q, g, sl, kw);
        ay = amax_p<T, 1>(Q, g, sl, kw);
    }
    template <class T>
    static __device__ __forceinline__ T rate_x(const T* Q, T sl, T kw) {
        DimlessP<T> g;
        dimless_p(Q, g);
        return amax_p<T, 0>(Q, g, sl, kw);
    }
    static __device__ __forceinline__ void increment(const float* W, const float* dU, float* Wn) {
        prim_increment_p(W, dU, Wn);
    }
    static __device__ __forceinline__ void relax_cons(double* U, const double* Q, double tau,
                                                      double h) {
        relax_p_cons(U, Q, tau, h);
    }
    template <class T>
    static __device__ __forceinline__ void relax_prim(T* W, T g, T* N) {
        relax_p_prim(W, g, N);
    }
    template <class T>
    static __device__ __forceinline__ bool nonpositive(const T* Q) {
        return Q[0] <= T(0) || Q[3] <= T(0) || Q[5] <= T(0) || Q[6] <= T(0);
    }
};

}  // namespace mxe
