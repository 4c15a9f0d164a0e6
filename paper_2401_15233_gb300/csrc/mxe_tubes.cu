// mxe_tubes.cu -- persistent batched solver for 1D problems (the 5-moment
// system of Sec. 2.3 and the 14-moment system of Sec. 2.4 in one space
// dimension), FP64 path.
//
// One thread block owns one tube for the whole launch and loops over time
// steps on its own clock (dt from an in-block CFL reduction), so tubes of
// different lengths and Knudsen numbers never wait for one another and no
// grid-wide synchronisation exists.  Within a stage the block sweeps its
// tube in chunks of NT-1 cells: stage the primitives of the chunk plus a
// 2-cell halo in shared memory, one shared limiter per cell, one thread per
// face (two face states, closure, flux, wave speeds, HLL/Rusanov), then
// flux differences, BGK source and the RK update.
#include "mxe_internal.h"

namespace mxe {

constexpr int NT1 = 128;
constexpr int C1 = NT1 - 1;           // cells per chunk
constexpr int BOX1 = C1 + 4;          // staged cells per chunk

template <int NF> struct Sys;
template <> struct Sys<5> {
    static __device__ __forceinline__ void cons2prim(const double* U, double* Q) { cons2prim5_rn(U, Q); }
    static __device__ __forceinline__ void prim2cons(const double* Q, double* U) { prim2cons5(Q, U); }
    static __device__ __forceinline__ void relax(double* U, const double* Q, double tau, double h) {
        relax5_cons(U, Q, tau, h);
    }
    static __device__ __forceinline__ void eval(const double* Q, const SchemeParams& sp, double* U,
                                                double* F, double& lo, double& hi) {
        face_eval5(Q, sp, U, F, lo, hi);
    }
    static __device__ __forceinline__ double amax(const double* Q, const SchemeParams& sp) {
        double a, s;
        rate5(Q, sp, a, s);
        return a;
    }
    static __device__ __forceinline__ void source(const double* Q, double tau, double* C) {
        source5(Q, tau, C);
    }
};
template <> struct Sys<14> {
    static __device__ __forceinline__ void cons2prim(const double* U, double* Q) { cons2prim14_rn(U, Q); }
    static __device__ __forceinline__ void prim2cons(const double* Q, double* U) { prim2cons14(Q, U); }
    static __device__ __forceinline__ void relax(double* U, const double* Q, double tau, double h) {
        relax14_cons(U, Q, tau, h);
    }
    static __device__ __forceinline__ void eval(const double* Q, const SchemeParams& sp, double* U,
                                                double* F, double& lo, double& hi) {
        face_eval14<double, 0>(Q, sp, U, F, lo, hi);
    }
    static __device__ __forceinline__ double amax(const double* Q, const SchemeParams& sp) {
        Dimless14<double> d;
        dimless14(Q, d);
        return amax14<double, 0>(Q, d, sp);
    }
    static __device__ __forceinline__ void source(const double* Q, double tau, double* C) {
        source14(Q, tau, C);
    }
};

template <int NF>
__device__ __forceinline__ void load_prim_1d(const TubeArgs& a, const double* U,
                                             const TubeDesc& td, int gi, double* Q) {
    if (gi < 0 || gi >= td.n) {
        int s = gi < 0 ? 0 : 1;
        int ty = a.bc_type[s];
        if (ty == 2) {
#pragma unroll
            for (int k = 0; k < NF; ++k) Q[k] = a.ghost[s * 14 + k];
            return;
        }
        if (ty == 1) gi = ((gi % td.n) + td.n) % td.n;
        else gi = gi < 0 ? 0 : td.n - 1;
    }
    double Uc[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) Uc[k] = U[(long long)k * td.n + gi];
    Sys<NF>::cons2prim(Uc, Q);
}

template <int NF>
__device__ __forceinline__ void riemann_1d(const double* QL, const double* QR,
                                           const SchemeParams& sp, double* Fo) {
    double UL[NF], FL[NF], lminL, lmaxL;
    Sys<NF>::eval(QL, sp, UL, FL, lminL, lmaxL);
    double UR[NF], FR[NF], lminR, lmaxR;
    Sys<NF>::eval(QR, sp, UR, FR, lminR, lmaxR);
    if (sp.flux == 1) {
        double s = fabs(lminL);
        s = fabs(lmaxL) > s ? fabs(lmaxL) : s;
        s = fabs(lminR) > s ? fabs(lminR) : s;
        s = fabs(lmaxR) > s ? fabs(lmaxR) : s;
#pragma unroll
        for (int k = 0; k < NF; ++k) Fo[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * s * (UR[k] - UL[k]);
        return;
    }
    double SL = lminL < lminR ? lminL : lminR;
    double SR = lmaxL > lmaxR ? lmaxL : lmaxR;
    if (SL >= 0.0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) Fo[k] = FL[k];
    } else if (SR <= 0.0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) Fo[k] = FR[k];
    } else {
#pragma unroll
        for (int k = 0; k < NF; ++k)
            Fo[k] = (SR * FL[k] - SL * FR[k] + SL * SR * (UR[k] - UL[k])) / (SR - SL);
    }
}

__device__ __forceinline__ double block_max_1d(double r, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, r, o);
        r = v > r ? v : r;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = r;
    __syncthreads();
    double m = red[0];
#pragma unroll
    for (int w = 1; w < NT1 / 32; ++w) m = red[w] > m ? red[w] : m;
    return m;
}

// One stage over the whole tube: out = base + coef dt L(in).  Returns the
// thread's max CFL rate of `out` if `final`.
template <int NF>
__device__ double tube_stage(const TubeArgs& a, const TubeDesc& td, const double* in,
                             const double* base, double* out, double coef, double dt,
                             bool final, double* W, double* Fb, double* ph,
                             unsigned& status) {
    const int tid = threadIdx.x;
    const int n = td.n;
    double rmax = 0.0;
    for (int c0 = 0; c0 < n; c0 += C1) {
        for (int idx = tid; idx < BOX1; idx += NT1) {
            double Q[NF];
            load_prim_1d<NF>(a, in, td, c0 - 2 + idx, Q);
#pragma unroll
            for (int k = 0; k < NF; ++k) W[k * BOX1 + idx] = Q[k];
        }
        __syncthreads();
        for (int idx = tid; idx < C1 + 2; idx += NT1) {       // box cells 1..C1+2
            int c = idx + 1;
            double phi = 0.0;
            if (a.sp.order == 2) {
                phi = 1.0;
                const FlatRef<double> fr = flat_ref<NF>(W + c, BOX1);
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    const double* w = W + k * BOX1 + c;
                    phi_accumulate<NF>(phi, w[0] - w[-1], w[1] - w[0], a.sp.limiter, fr, k);
                }
            }
            ph[idx] = phi;
        }
        __syncthreads();
        {   // face tid between box cells tid+1 | tid+2
            double QL[NF], QR[NF], F[NF];
            int cl = tid + 1, cr = tid + 2;
            double pl = ph[cl - 1], pr = ph[cr - 1];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                const double* w = W + k * BOX1;
                QL[k] = muscl_face(w[cl - 1], w[cl], w[cl + 1], pl, 0.5);
                QR[k] = muscl_face(w[cr - 1], w[cr], w[cr + 1], pr, -0.5);
            }
            riemann_1d<NF>(QL, QR, a.sp, F);
#pragma unroll
            for (int k = 0; k < NF; ++k) Fb[k * NT1 + tid] = F[k];
        }
        __syncthreads();
        int i = c0 + tid;
        if (tid < C1 && i < n) {
            double Qc[NF], L[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) Qc[k] = W[k * BOX1 + tid + 2];
            if (td.rp.model != 0 && !td.rp.implicit) {
                double tau = tau_of<double>(td.rp, Qc, NF);
                Sys<NF>::source(Qc, tau, L);
            } else {
#pragma unroll
                for (int k = 0; k < NF; ++k) L[k] = 0.0;
            }
            double Un[NF];
            bool bad = false;
            double cdt = mul_rn(coef, dt);
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                L[k] -= (Fb[k * NT1 + tid + 1] - Fb[k * NT1 + tid]) / td.dx;
                Un[k] = add_rn(base[(long long)k * n + i], mul_rn(cdt, L[k]));
            }
            if (td.rp.model != 0 && td.rp.implicit) {   // point-implicit source over cdt
                double Qv[NF];
                Sys<NF>::cons2prim(Un, Qv);
                Sys<NF>::relax(Un, Qv, tau_of<double>(td.rp, Qv, NF), cdt);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                out[(long long)k * n + i] = Un[k];
                bad |= !isfinite(Un[k]);
            }
            if (final) {
                double Qn[NF];
                Sys<NF>::cons2prim(Un, Qn);
                if (bad) status |= ST_NONFINITE;
                if (Qn[0] <= 0.0 || Qn[NF == 5 ? 2 : 4] <= 0.0) status |= ST_NONPOSITIVE;
                double r = Sys<NF>::amax(Qn, a.sp) / td.dx;
                if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);
                rmax = r > rmax ? r : rmax;
            }
        }
        __syncthreads();
    }
    return rmax;
}

template <int NF>
__device__ void tubes_body(const TubeArgs& a) {
    __shared__ double W[NF * BOX1];
    __shared__ double Fb[NF * NT1];
    __shared__ double ph[C1 + 2];
    __shared__ double red[NT1 / 32];
    __shared__ unsigned sstat;
    const int b = blockIdx.x;
    if (b >= a.ntubes) return;
    const TubeDesc td = a.tubes[b];
    TubeClock* ck = a.clk + b;
    double* U = a.U + td.off;
    double* Us = a.Us + td.off;
    const int tid = threadIdx.x;
    unsigned status = 0;

    // CFL rate of the current state
    double r = 0.0;
    for (int i = tid; i < td.n; i += NT1) {
        double Uc[NF], Q[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Uc[k] = U[(long long)k * td.n + i];
        Sys<NF>::cons2prim(Uc, Q);
        double ri = Sys<NF>::amax(Q, a.sp) / td.dx;
        if (!(ri >= 0.0)) ri = __longlong_as_double(0x7ff0000000000000ll);
        r = ri > r ? ri : r;
    }
    double m = block_max_1d(r, red);
    double t = ck->t;
    long long steps = ck->steps;
    double last_dt = ck->last_dt;
    for (int s = 0; s < a.max_steps; ++s) {
        double dt;
        if (a.dt_fixed) {
            if (s >= a.n_fixed) break;
            dt = a.dt_fixed[s];
        } else {
            if (!(t < a.t_end)) break;
            dt = a.cfl / m;
            if (t + dt > a.t_end) dt = a.t_end - t;
        }
        if (!(dt > 0.0)) break;
        double rr;
        if (a.integrator == 1) {
            tube_stage<NF>(a, td, U, U, Us, 0.5, dt, false, W, Fb, ph, status);
            rr = tube_stage<NF>(a, td, Us, U, U, 1.0, dt, true, W, Fb, ph, status);
        } else {
            rr = tube_stage<NF>(a, td, U, U, Us, 1.0, dt, true, W, Fb, ph, status);
            for (int i = tid; i < NF * td.n; i += NT1) U[i] = Us[i];
            __syncthreads();
        }
        if (tid == 0) sstat = 0u;
        m = block_max_1d(rr, red);           // contains __syncthreads
        if (status) atomicOr(&sstat, status);
        __syncthreads();
        unsigned bst = sstat;
        t += dt;
        last_dt = dt;
        ++steps;
        if (bst) break;                      // block-uniform
        __syncthreads();
    }
    if (status) atomicOr(&ck->status, status);
    __syncthreads();
    if (tid == 0) {
        ck->t = t;
        ck->steps = steps;
        ck->last_dt = last_dt;
        ck->rate = m;
    }
}

extern "C" __global__ void __launch_bounds__(NT1) mxe_tubes5_f64(const TubeArgs a) {
    tubes_body<5>(a);
}
extern "C" __global__ void __launch_bounds__(NT1) mxe_tubes14_f64(const TubeArgs a) {
    tubes_body<14>(a);
}

int tubes_threads() { return NT1; }

}  // namespace mxe
