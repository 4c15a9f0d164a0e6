// mxe_adjoint.cu -- discrete adjoint (reverse mode) of one RK stage of the
// 2D 14-moment scheme for planar states, FP64.
//
// A stage is U_out = U_base + c dt L(U_in) with L(U) = -sum_d (F_{d,f+1/2}
// - F_{d,f-1/2}) / dx_d + C(U) (Sec. 3).  Given V (the adjoint of U_out)
// and coef = c dt, the kernels form
//   out = b1 + b2 + coef (dL/dU(U_in))^T V
// plus the adjoints of the imposed boundary states and of tau_ref:
//   mxe_adj_prims   primitives of U_in (FP64, oracle-order rounding)
//   mxe_adj_faces   two lanes per face, one per face state: recompute the
//                   reconstruction and the face state once (intermediates
//                   kept), exchange the primal outputs with the partner lane,
//                   reverse HLL / Rusanov, the face evaluation and the MUSCL
//                   + shared limiter; write the primitive adjoint
//                   contributions to the four stencil cells f-2 .. f+1
//   mxe_adj_cells   one thread per cell: gather the contributions of the
//                   eight faces that touch it (and of ghost cells that copy
//                   it), reverse the BGK source and the primitive recovery
//   mxe_adj_ghosts  contributions to Dirichlet ghost cells -> adjoint of the
//                   imposed primitive states
// Branches follow the primal (see mxe_adjoint.cuh).
#include "mxe_adjoint.cuh"
#include "mxe_internal.h"
#include "mxe_policy.cuh"

namespace mxe {

struct AdjArgs {
    const double* U;            // U_in, pitched 14-field layout
    const double* V;            // adjoint of U_out times c dt (same layout)
    const double* b1;           // optional base terms (same layout) or NULL
    const double* b2;
    double* out;                // adjoint of U_in (may alias b1)
    double* P;                  // primitives of U_in, NP compact fields, pitched
    double* Cx;                 // [4][NP][ny][nx+1] x-face contributions
    double* Cy;                 // [4][NP][ny+1][nx] y-face contributions
    double* gbar;               // [4][GHOST_SLOTS][14] adjoint of imposed states (accumulated)
    double* taubar;             // adjoint of tau_ref (accumulated)
    double coef;                // c dt of the stage: V is scaled by it
    // FP32 face-state reverse: per-cell data formed once in FP64
    float* Pf;                  // [NP][ny][pitch] primitives
    float* Vf;                  // [NP][ny][pitch] coef * V
    float* DX;                  // [NP][ny][nx+3] Q(i+1) - Q(i), i = -2 .. nx (ghosts included)
    float* DY;                  // [NP][ny+3][nx] Q(j+1) - Q(j), j = -2 .. ny
    float* LX;                  // [4][ny][nx+2] x limiter of cell i = -1 .. nx (phi, dphi/ddm,
                                //   dphi/ddp, selected field), formed in FP64
    float* LY;                  // [4][ny+2][nx] y limiter of cell j = -1 .. ny
    int f32;                    // contributions Cx, Cy stored as float
    int frozen_phi;             // the shared limiter held constant in the derivative
    Grid2D g;
    ParamsT<double> p;
};

__device__ __forceinline__ long long cx_index(const Grid2D& g, int s, int k, int j, int f) {
    return (((long long)s * NP + k) * g.ny + j) * (g.nx + 1) + f;
}
__device__ __forceinline__ long long cy_index(const Grid2D& g, int s, int k, int f, int i) {
    return (((long long)s * NP + k) * (g.ny + 1) + f) * g.nx + i;
}

// Ghost-cell classification along a side: Dirichlet slot (returns the
// state's row in the ghost table, sets slot), or the interior cell it
// copies (transmissive clamp / periodic wrap; returns nullptr).
__device__ __forceinline__ const double* ghost_of(const Grid2D& g, int side, int t, int& slot) {
    const SideDesc& sd = g.side[side];
    slot = -1;
    if (sd.type == 1) return nullptr;
    for (int n = 0; n < sd.nspans; ++n)
        if (t >= sd.lo[n] && t <= sd.hi[n]) {
            slot = 1 + n;
            return g.ghost + (side * GHOST_SLOTS + 1 + n) * 14;
        }
    if (sd.type == 2) {
        slot = 0;
        return g.ghost + (side * GHOST_SLOTS) * 14;
    }
    return nullptr;
}

// primitive state at stencil position (i, j) (one of them may be outside)
__device__ __forceinline__ void stencil_prim(const AdjArgs& a, int i, int j, double* Q) {
    const Grid2D& g = a.g;
    int slot;
    if (i < 0 || i >= g.nx) {
        const double* gs = ghost_of(g, i < 0 ? 0 : 1, j, slot);
        if (gs) {
#pragma unroll
            for (int k = 0; k < NP; ++k) Q[k] = gs[planar_field(k)];
            return;
        }
        i = g.side[0].type == 1 ? ((i % g.nx) + g.nx) % g.nx : (i < 0 ? 0 : g.nx - 1);
    } else if (j < 0 || j >= g.ny) {
        const double* gs = ghost_of(g, j < 0 ? 2 : 3, i, slot);
        if (gs) {
#pragma unroll
            for (int k = 0; k < NP; ++k) Q[k] = gs[planar_field(k)];
            return;
        }
        j = g.side[2].type == 1 ? ((j % g.ny) + g.ny) % g.ny : (j < 0 ? 0 : g.ny - 1);
    }
    const double* p = a.P + (long long)j * g.pitch + i;
#pragma unroll
    for (int k = 0; k < NP; ++k) Q[k] = p[k * g.fstride];
}

extern "C" __global__ void mxe_adj_prims(const AdjArgs a) {
    const Grid2D& g = a.g;
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= g.nx) return;
    long long o = (long long)j * g.pitch + i;
    double Uc[NP], Q[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Uc[k] = a.U[o + planar_field(k) * g.fstride];
    cons2prim_p_rn(Uc, Q);
#pragma unroll
    for (int k = 0; k < NP; ++k) a.P[o + k * g.fstride] = Q[k];
    if (a.f32) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            a.Pf[o + k * g.fstride] = (float)Q[k];
            a.Vf[o + k * g.fstride] = (float)(a.coef * a.V[o + planar_field(k) * g.fstride]);
        }
    }
}

// FP32 path: stencil differences in FP64, stored in FP32 (their own
// relative precision, not that of the states), ghost cells included.
__device__ __forceinline__ long long dx_index(const Grid2D& g, int k, int j, int i) {
    return ((long long)k * g.ny + j) * (g.nx + 3) + (i + 2);
}
__device__ __forceinline__ long long dy_index(const Grid2D& g, int k, int j, int i) {
    return ((long long)k * (g.ny + 3) + (j + 2)) * g.nx + i;
}
__device__ __forceinline__ long long lx_index(const Grid2D& g, int m, int j, int i) {
    return ((long long)m * g.ny + j) * (g.nx + 2) + (i + 1);
}
__device__ __forceinline__ long long ly_index(const Grid2D& g, int m, int j, int i) {
    return ((long long)m * (g.ny + 2) + (j + 1)) * g.nx + i;
}

// The shared limiter of every cell and direction (ghost cells next to the
// boundary included) in FP64, so that the FP32 reverse takes the FP64
// branches: phi, its derivatives and the field that sets it.
extern "C" __global__ void mxe_adj_limiters(const AdjArgs a) {
    const Grid2D& g = a.g;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int nxc = (g.nx + 2) * g.ny, nyc = g.nx * (g.ny + 2);
    int i, j, K;
    if (id < nxc) {
        j = id / (g.nx + 2);
        i = id % (g.nx + 2) - 1;
        K = 0;
    } else if (id < nxc + nyc) {
        const int r = id - nxc;
        i = r % g.nx;
        j = r / g.nx - 1;
        K = 1;
    } else {
        return;
    }
    double qm[NP], q0[NP], qp[NP];
    stencil_prim(a, K == 0 ? i - 1 : i, K == 0 ? j : j - 1, qm);
    stencil_prim(a, i, j, q0);
    stencil_prim(a, K == 0 ? i + 1 : i, K == 0 ? j : j + 1, qp);
    adj::PhiAdj<double> ph{1.0, 0.0, 0.0, -1};
    if (a.p.order == 2) ph = adj::phi_adj<double, NP>(qm, q0, qp, a.p.limiter);
    else ph.phi = 0.0;
    if (a.frozen_phi) ph.ks = -1;
    float* L = K == 0 ? a.LX : a.LY;
    const float v[4] = {(float)ph.phi, (float)ph.ddm, (float)ph.ddp, (float)ph.ks};
#pragma unroll
    for (int m = 0; m < 4; ++m) L[K == 0 ? lx_index(g, m, j, i) : ly_index(g, m, j, i)] = v[m];
}

extern "C" __global__ void mxe_adj_diffs(const AdjArgs a) {
    const Grid2D& g = a.g;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int nxp = (g.nx + 3) * g.ny, nyp = g.nx * (g.ny + 3);
    if (id < nxp) {                                  // x pairs (i, i+1) of row j
        const int j = id / (g.nx + 3), i = id % (g.nx + 3) - 2;
        double q0[NP], q1[NP];
        stencil_prim(a, i, j, q0);
        stencil_prim(a, i + 1, j, q1);
#pragma unroll
        for (int k = 0; k < NP; ++k) a.DX[dx_index(g, k, j, i)] = (float)(q1[k] - q0[k]);
    } else if (id < nxp + nyp) {                     // y pairs (j, j+1) of column i
        const int r = id - nxp;
        const int i = r % g.nx, j = r / g.nx - 2;
        double q0[NP], q1[NP];
        stencil_prim(a, i, j, q0);
        stencil_prim(a, i, j + 1, q1);
#pragma unroll
        for (int k = 0; k < NP; ++k) a.DY[dy_index(g, k, j, i)] = (float)(q1[k] - q0[k]);
    }
}

// Adjoint of the numerical flux for one of its two states (own = left if
// isL): given both states' primal outputs and Fb, the adjoints of the own
// state's (U, F, lmin, lmax).
template <int K, class T>
__device__ __forceinline__ void riemann_bwd_side(const ParamsT<double>& p, bool isL,
                                                 const T* UL, const T* FL, T lminL,
                                                 T lmaxL, const T* UR, const T* FR,
                                                 T lminR, T lmaxR, const T* Fb,
                                                 T* Ub, T* Fob, T& lminb,
                                                 T& lmaxb) {
#pragma unroll
    for (int k = 0; k < NP; ++k) Ub[k] = Fob[k] = T(0.0);
    lminb = lmaxb = T(0.0);
    if (p.flux == 1) {
        T s = fabs(lminL);
        int sel = 0;
        if (fabs(lmaxL) > s) { s = fabs(lmaxL); sel = 1; }
        if (fabs(lminR) > s) { s = fabs(lminR); sel = 2; }
        if (fabs(lmaxR) > s) { s = fabs(lmaxR); sel = 3; }
        T sb = T(0.0);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            Fob[k] = T(0.5) * Fb[k];
            Ub[k] = (isL ? T(0.5) : -T(0.5)) * s * Fb[k];
            sb -= T(0.5) * Fb[k] * (UR[k] - UL[k]);
        }
        const T lam = sel == 0 ? lminL : sel == 1 ? lmaxL : sel == 2 ? lminR : lmaxR;
        const T g = lam > T(0.0) ? sb : (lam < T(0.0) ? -sb : T(0.0));
        if (isL) {
            if (sel == 0) lminb = g;
            if (sel == 1) lmaxb = g;
        } else {
            if (sel == 2) lminb = g;
            if (sel == 3) lmaxb = g;
        }
        return;
    }
    const T SL = lminL < lminR ? lminL : lminR;
    const T SR = lmaxL > lmaxR ? lmaxL : lmaxR;
    if (SL >= T(0.0)) {
        if (isL)
#pragma unroll
            for (int k = 0; k < NP; ++k) Fob[k] = Fb[k];
        return;
    }
    if (SR <= T(0.0)) {
        if (!isL)
#pragma unroll
            for (int k = 0; k < NP; ++k) Fob[k] = Fb[k];
        return;
    }
    const T inv = T(1.0) / (SR - SL);
    const T SLR = SL * SR;
    T SRb = T(0.0), SLb = T(0.0);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const T dU = UR[k] - UL[k];
        const T F = (SR * FL[k] - SL * FR[k] + SLR * dU) * inv;
        Fob[k] = isL ? Fb[k] * SR * inv : -Fb[k] * SL * inv;
        Ub[k] = isL ? -Fb[k] * SLR * inv : Fb[k] * SLR * inv;
        SRb += Fb[k] * (FL[k] + SL * dU - F) * inv;
        SLb += Fb[k] * (-FR[k] + SR * dU + F) * inv;
    }
    const bool selL_min = lminL < lminR, selL_max = lmaxL > lmaxR;
    if (isL == selL_min) lminb = SLb;
    if (isL == selL_max) lmaxb = SRb;
}

__device__ __forceinline__ double shfl1(double v, unsigned m = 0xffffffffu) {
    return __shfl_xor_sync(m, v, 1);
}
__device__ __forceinline__ float shfl1(float v, unsigned m = 0xffffffffu) {
    return __shfl_xor_sync(m, v, 1);
}

// One face state per thread, two threads (adjacent lanes) per face: lane
// parity 0 = left state (cell f-1, stencil f-2..f), 1 = right state (cell f,
// stencil f-1..f+1).  f in [0, n_K] on line t (row j for x-faces, column i
// for y-faces).  Threads past the last face compute the last face (the
// shuffles need the whole warp) and write nothing.
template <int K, class T>
__device__ __forceinline__ void adj_face_side(const AdjArgs& a, int f, int t, bool valid) {
    const Grid2D& g = a.g;
    const ParamsT<double>& p = a.p;
    const int nK = K == 0 ? g.nx : g.ny;
    const bool isL = (threadIdx.x & 1) == 0;
    const int c0 = isL ? f - 1 : f;                      // own cell
    // reconstruction and limiter in FP64 (differences of nearby states); the
    // face state itself in T.  The stencil is loaded again for the
    // reconstruction reverse rather than kept live through the face state.
    auto load_stencil = [&](double (*Qs)[NP]) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (K == 0) stencil_prim(a, c0 - 1 + m, t, Qs[m]);
            else stencil_prim(a, t, c0 - 1 + m, Qs[m]);
        }
    };
    adj::PhiAdj<double> ph{0.0, 0.0, 0.0, -1};
    const double hs = isL ? 0.5 : -0.5;
    T Qf[NP];
    {
        double Qs[3][NP];
        load_stencil(Qs);
        if (p.order == 2) ph = adj::phi_adj<double, NP>(Qs[0], Qs[1], Qs[2], p.limiter);
        if (a.frozen_phi) ph.ks = -1;
#pragma unroll
        for (int k = 0; k < NP; ++k)
            Qf[k] = (T)muscl_face(Qs[0][k], Qs[1][k], Qs[2][k], ph.phi, hs);
    }
    // adjoint of the face flux: L_l -= F idx, L_r += F idx
    const double idx = K == 0 ? g.idx : g.idy;
    // The reverse is linear in the flux adjoint: it runs on Fb scaled by a
    // power of two (so that FP32 cannot overflow) and the result is scaled
    // back.  A face whose flux adjoint is zero contributes nothing.
    double Fbd[NP];
    {
        const int l = f - 1, r = f;
        const long long ol = K == 0 ? (long long)t * g.pitch + l : (long long)l * g.pitch + t;
        const long long orr = K == 0 ? (long long)t * g.pitch + r : (long long)r * g.pitch + t;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const long long fo = planar_field(k) * g.fstride;
            const double vl = l >= 0 ? a.V[ol + fo] : 0.0;
            const double vr = r < nK ? a.V[orr + fo] : 0.0;
            Fbd[k] = ((vr - vl) * a.coef) * idx;
        }
    }
    double fmax = 0.0;
#pragma unroll
    for (int k = 0; k < NP; ++k) fmax = fmax > fabs(Fbd[k]) ? fmax : fabs(Fbd[k]);
    const bool live = fmax > 0.0;                       // same in both lanes of the face
    const unsigned mask = __ballot_sync(0xffffffffu, live);
    int ex = 0;
    if (live) frexp(fmax, &ex);
    const double scale = ldexp(1.0, ex);
    T Fb[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Fb[k] = (T)(Fbd[k] / scale);
    T Qb[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Qb[k] = T(0);
    auto outadj = [&](const T* U, const T* F, T lmin, T lmax, T* Ub, T* Fob, T& lminb,
                      T& lmaxb) {
        T Up[NP], Fp[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            Up[k] = shfl1(U[k], mask);
            Fp[k] = shfl1(F[k], mask);
        }
        const T lminp = shfl1(lmin, mask), lmaxp = shfl1(lmax, mask);
        if (isL)
            riemann_bwd_side<K, T>(p, true, U, F, lmin, lmax, Up, Fp, lminp, lmaxp, Fb, Ub, Fob,
                                lminb, lmaxb);
        else
            riemann_bwd_side<K, T>(p, false, Up, Fp, lminp, lmaxp, U, F, lmin, lmax, Fb, Ub, Fob,
                                lminb, lmaxb);
    };
    if (live) adj::face_side_adj<T, K>(Qf, (T)p.sigma_lim, (T)p.k_ws, outadj, Qb);
    // reconstruction reverse -> own stencil (bm, b0, bp)
    double Qbd[NP], bm[NP], b0[NP], bp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        Qbd[k] = (double)Qb[k] * scale;
        bm[k] = b0[k] = bp[k] = 0.0;
    }
    if (p.order == 2) {
        double Qs[3][NP];
        load_stencil(Qs);
        adj::muscl_bwd<double, NP>(Qs[0], Qs[1], Qs[2], ph, hs, Qbd, bm, b0, bp);
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) b0[k] = Qbd[k];
    }
    // slots of the face: 0 = f-2, 1 = f-1, 2 = f, 3 = f+1.  Left state: bm,
    // b0, bp -> slots 0, 1, 2; right state: slots 1, 2, 3.  Exchange the
    // overlap so that each lane writes two slots.
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const double send = isL ? bp[k] : bm[k];
        const double recv = shfl1(send);
        if (!valid) continue;
        const double lo = isL ? bm[k] : b0[k] + recv;   // slot 0 (L) or 2 (R)
        const double hi = isL ? b0[k] + recv : bp[k];   // slot 1 (L) or 3 (R)
        const int s0 = isL ? 0 : 2;
        if (K == 0) {
            a.Cx[cx_index(g, s0, k, t, f)] = lo;
            a.Cx[cx_index(g, s0 + 1, k, t, f)] = hi;
        } else {
            a.Cy[cy_index(g, s0, k, f, t)] = lo;
            a.Cy[cy_index(g, s0 + 1, k, f, t)] = hi;
        }
    }
}

// FP32 variant: everything from the per-cell FP32 data (primitives, the
// FP64-formed stencil differences, coef * V), no FP64 arithmetic except for
// the own cell of a boundary face that is a ghost cell.  Contributions are
// stored as float.
template <int K>
__device__ __forceinline__ void adj_face_side_f32(const AdjArgs& a, int f, int t, bool valid) {
    const Grid2D& g = a.g;
    const ParamsT<double>& p = a.p;
    const int nK = K == 0 ? g.nx : g.ny;
    const bool isL = (threadIdx.x & 1) == 0;
    const int c0 = isL ? f - 1 : f;                      // own cell
    float dm[NP], dp[NP], Qf[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        dm[k] = K == 0 ? a.DX[dx_index(g, k, t, c0 - 1)] : a.DY[dy_index(g, k, c0 - 1, t)];
        dp[k] = K == 0 ? a.DX[dx_index(g, k, t, c0)] : a.DY[dy_index(g, k, c0, t)];
    }
    if (c0 >= 0 && c0 < nK) {
        const long long o = K == 0 ? (long long)t * g.pitch + c0 : (long long)c0 * g.pitch + t;
#pragma unroll
        for (int k = 0; k < NP; ++k) Qf[k] = a.Pf[o + k * g.fstride];
    } else {
        double Qd[NP];
        if (K == 0) stencil_prim(a, c0, t, Qd);
        else stencil_prim(a, t, c0, Qd);
#pragma unroll
        for (int k = 0; k < NP; ++k) Qf[k] = (float)Qd[k];
    }
    adj::PhiAdj<float> ph;
    {
        const float* L = K == 0 ? a.LX : a.LY;
        auto at = [&](int m) {
            return L[K == 0 ? lx_index(g, m, t, c0) : ly_index(g, m, c0, t)];
        };
        ph.phi = at(0);
        ph.ddm = at(1);
        ph.ddp = at(2);
        ph.ks = (int)at(3);
    }
    const float hs = isL ? 0.5f : -0.5f;
#pragma unroll
    for (int k = 0; k < NP; ++k) Qf[k] = Qf[k] + hs * (ph.phi * (0.5f * (dm[k] + dp[k])));
    // flux adjoint from coef * V (0 at ghost cells), scaled by a power of two
    const float idx = (float)(K == 0 ? g.idx : g.idy);
    float Fb[NP];
    {
        const int l = f - 1, r = f;
        const long long ol = K == 0 ? (long long)t * g.pitch + l : (long long)l * g.pitch + t;
        const long long orr = K == 0 ? (long long)t * g.pitch + r : (long long)r * g.pitch + t;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float vl = l >= 0 ? a.Vf[ol + k * g.fstride] : 0.0f;
            const float vr = r < nK ? a.Vf[orr + k * g.fstride] : 0.0f;
            Fb[k] = (vr - vl) * idx;
        }
    }
    float fmax = 0.0f;
#pragma unroll
    for (int k = 0; k < NP; ++k) fmax = fmaxf(fmax, fabsf(Fb[k]));
    const bool live = fmax > 0.0f;
    const unsigned mask = __ballot_sync(0xffffffffu, live);
    int ex = 0;
    if (live) frexpf(fmax, &ex);
    // exponent shifts (a power-of-two factor 2^-ex itself can overflow FP32
    // when the adjoint is still tiny, i.e. subnormal, at the edge of its support)
#pragma unroll
    for (int k = 0; k < NP; ++k) Fb[k] = ldexpf(Fb[k], -ex);
    float Qb[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Qb[k] = 0.0f;
    auto outadj = [&](const float* U, const float* F, float lmin, float lmax, float* Ub,
                      float* Fob, float& lminb, float& lmaxb) {
        float Up[NP], Fp[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            Up[k] = shfl1(U[k], mask);
            Fp[k] = shfl1(F[k], mask);
        }
        const float lminp = shfl1(lmin, mask), lmaxp = shfl1(lmax, mask);
        if (isL)
            riemann_bwd_side<K, float>(p, true, U, F, lmin, lmax, Up, Fp, lminp, lmaxp, Fb, Ub,
                                       Fob, lminb, lmaxb);
        else
            riemann_bwd_side<K, float>(p, false, Up, Fp, lminp, lmaxp, U, F, lmin, lmax, Fb, Ub,
                                       Fob, lminb, lmaxb);
    };
    if (live)
        adj::face_side_adj<float, K>(Qf, (float)p.sigma_lim, (float)p.k_ws, outadj, Qb);
    float bm[NP], b0[NP], bp[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        Qb[k] = ldexpf(Qb[k], ex);
        bm[k] = b0[k] = bp[k] = 0.0f;
    }
    if (p.order == 2) {
        adj::muscl_bwd_d<float, NP>(dm, dp, ph, hs, Qb, bm, b0, bp);
    } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) b0[k] = Qb[k];
    }
    float* Cf = reinterpret_cast<float*>(K == 0 ? a.Cx : a.Cy);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float send = isL ? bp[k] : bm[k];
        const float recv = shfl1(send);
        if (!valid) continue;
        const float lo = isL ? bm[k] : b0[k] + recv;
        const float hi = isL ? b0[k] + recv : bp[k];
        const int s0 = isL ? 0 : 2;
        if (K == 0) {
            Cf[cx_index(g, s0, k, t, f)] = lo;
            Cf[cx_index(g, s0 + 1, k, t, f)] = hi;
        } else {
            Cf[cy_index(g, s0, k, f, t)] = lo;
            Cf[cy_index(g, s0 + 1, k, f, t)] = hi;
        }
    }
}

// 128 threads = 64 faces of one line (x) or 64 columns of one face row (y)
template <class T>
__device__ __forceinline__ void faces_x(const AdjArgs& a) {
    const int f = blockIdx.x * 64 + (threadIdx.x >> 1), j = blockIdx.y;
    const bool valid = f <= a.g.nx;
    if (sizeof(T) == 4) adj_face_side_f32<0>(a, valid ? f : a.g.nx, j, valid);
    else adj_face_side<0, T>(a, valid ? f : a.g.nx, j, valid);
}
template <class T>
__device__ __forceinline__ void faces_y(const AdjArgs& a) {
    const int i = blockIdx.x * 64 + (threadIdx.x >> 1), f = blockIdx.y;
    const bool valid = i < a.g.nx;
    if (sizeof(T) == 4) adj_face_side_f32<1>(a, f, valid ? i : a.g.nx - 1, valid);
    else adj_face_side<1, T>(a, f, valid ? i : a.g.nx - 1, valid);
}
// FP64 reverse (exact linearisation) and FP32 reverse (the face states
// recomputed and reversed in FP32 from per-cell FP32 data)
extern "C" __global__ void __launch_bounds__(128) mxe_adj_faces_x(const AdjArgs a) { faces_x<double>(a); }
extern "C" __global__ void __launch_bounds__(128) mxe_adj_faces_y(const AdjArgs a) { faces_y<double>(a); }
extern "C" __global__ void __launch_bounds__(128) mxe_adj_faces_x_f32(const AdjArgs a) { faces_x<float>(a); }
extern "C" __global__ void __launch_bounds__(128) mxe_adj_faces_y_f32(const AdjArgs a) { faces_y<float>(a); }

// Sum of the x-face contributions to stencil position (v, j): slot s of face
// f targets cell f - 2 + s.
__device__ __forceinline__ void gather_x(const AdjArgs& a, int v, int j, double* Qb) {
    const Grid2D& g = a.g;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int f = v + 2 - s;
        if (f < 0 || f > g.nx) continue;
        const float* cf = reinterpret_cast<const float*>(a.Cx);
#pragma unroll
        for (int k = 0; k < NP; ++k)
            Qb[k] += a.f32 ? (double)cf[cx_index(g, s, k, j, f)] : a.Cx[cx_index(g, s, k, j, f)];
    }
}
__device__ __forceinline__ void gather_y(const AdjArgs& a, int i, int w, double* Qb) {
    const Grid2D& g = a.g;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int f = w + 2 - s;
        if (f < 0 || f > g.ny) continue;
        const float* cf = reinterpret_cast<const float*>(a.Cy);
#pragma unroll
        for (int k = 0; k < NP; ++k)
            Qb[k] += a.f32 ? (double)cf[cy_index(g, s, k, f, i)] : a.Cy[cy_index(g, s, k, f, i)];
    }
}

// Interior cell copied by ghost position v of the line t along direction K
// (transmissive: nearest cell; periodic: wrapped), or -1 (Dirichlet ghost).
template <int K>
__device__ __forceinline__ int ghost_image(const Grid2D& g, int v, int t) {
    const int n = K == 0 ? g.nx : g.ny;
    const int side = (K == 0 ? 0 : 2) + (v < 0 ? 0 : 1);
    int slot;
    if (ghost_of(g, side, t, slot)) return -1;
    if (g.side[side].type == 1) return ((v % n) + n) % n;
    return v < 0 ? 0 : n - 1;
}

__device__ __forceinline__ double block_sum_128(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

extern "C" __global__ void __launch_bounds__(128) mxe_adj_cells(const AdjArgs a) {
    __shared__ double red[4];
    const Grid2D& g = a.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    double taub = 0.0;
    if (i < g.nx) {
        double Qb[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) Qb[k] = 0.0;
        gather_x(a, i, j, Qb);
        gather_y(a, i, j, Qb);
        // ghost cells that copy this cell
        if (i < 2 || i >= g.nx - 2) {
            const int vs[4] = {-2, -1, g.nx, g.nx + 1};
#pragma unroll
            for (int n = 0; n < 4; ++n)
                if (ghost_image<0>(g, vs[n], j) == i) gather_x(a, vs[n], j, Qb);
        }
        if (j < 2 || j >= g.ny - 2) {
            const int ws[4] = {-2, -1, g.ny, g.ny + 1};
#pragma unroll
            for (int n = 0; n < 4; ++n)
                if (ghost_image<1>(g, ws[n], i) == j) gather_y(a, i, ws[n], Qb);
        }
        const long long o = (long long)j * g.pitch + i;
        double Q[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) Q[k] = a.P[o + k * g.fstride];
        if (a.p.tau_model != 0) {
            double W[NP];
#pragma unroll
            for (int k = 0; k < NP; ++k) W[k] = a.coef * a.V[o + planar_field(k) * g.fstride];
            taub = adj::source_p_bwd(a.p.tau_model, a.p.tau_ref, a.p.rho_ref, a.p.T_ref, Q, W, Qb);
        }
        double Ub[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) Ub[k] = 0.0;
        adj::cons2prim_p_bwd(Q, Qb, Ub);
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const long long ok = o + k * g.fstride;
            double v = 0.0;
            if (a.b1) v += a.b1[ok];
            if (a.b2) v += a.b2[ok];
            a.out[ok] = v;
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) a.out[o + planar_field(k) * g.fstride] += Ub[k];
    }
    const double s = block_sum_128(taub, red);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(a.taubar, s);
}

// Dirichlet ghost positions: adjoint of the imposed primitive states.
extern "C" __global__ void mxe_adj_ghosts(const AdjArgs a) {
    const Grid2D& g = a.g;
    const int per = 2 * (2 * g.ny + 2 * g.nx);
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= per) return;
    // positions: side 0, 1 (2 layers x ny), then side 2, 3 (2 layers x nx)
    int side, layer, t;
    if (id < 4 * g.ny) {
        side = id / (2 * g.ny);
        layer = (id / g.ny) % 2;
        t = id % g.ny;
    } else {
        const int r = id - 4 * g.ny;
        side = 2 + r / (2 * g.nx);
        layer = (r / g.nx) % 2;
        t = r % g.nx;
    }
    int slot;
    if (!ghost_of(g, side, t, slot)) return;
    double Qb[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) Qb[k] = 0.0;
    if (side < 2) {
        const int v = side == 0 ? -1 - layer : g.nx + layer;
        gather_x(a, v, t, Qb);
    } else {
        const int w = side == 2 ? -1 - layer : g.ny + layer;
        gather_y(a, t, w, Qb);
    }
    double* dst = a.gbar + (side * GHOST_SLOTS + slot) * 14;
#pragma unroll
    for (int k = 0; k < NP; ++k)
        if (Qb[k] != 0.0) atomicAdd(dst + planar_field(k), Qb[k]);
}

// dense (14, ny, nx) <-> pitched 14-field layout
// Dense (14, ny, nx) <-> pitched layout of an adjoint state.  Unpacking
// (to_pitched = 0) also sets *nonfinite when a value is not finite (the
// FP32 face-state reverse can leave its range), if nonfinite is given.
extern "C" __global__ void mxe_adj_pack(const double* dense, double* pitched, Grid2D g, int to_pitched,
                                        unsigned long long* nonfinite) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= g.nx) return;
    bool bad = false;
    for (int k = 0; k < 14; ++k) {
        const long long d = ((long long)k * g.ny + j) * g.nx + i;
        const long long p = (long long)k * g.fstride + (long long)j * g.pitch + i;
        if (to_pitched) {
            pitched[p] = dense[d];
        } else {
            const double v = pitched[p];
            const_cast<double*>(dense)[d] = v;
            bad |= !isfinite(v);
        }
    }
    if (bad && nonfinite) atomicOr(nonfinite, 1ull);
}

size_t adj_args_size() { return sizeof(AdjArgs); }

// floats of the FP32 per-cell data of a grid (Pf, Vf, DX, DY, LX, LY)
long long adj_f32_floats(const Grid2D& g) {
    return 2LL * NP * g.fstride + (long long)NP * g.ny * (g.nx + 3) +
           (long long)NP * (g.ny + 3) * g.nx + 4LL * g.ny * (g.nx + 2) + 4LL * (g.ny + 2) * g.nx;
}

// Host launcher of one stage reverse (declared in mxe_capi.cu).
cudaError_t adj_stage(const double* U, const double* V, double coef, const double* b1,
                      const double* b2, double* out, double* P, double* Cx, double* Cy,
                      double* gbar, double* taubar, const Grid2D& g, const ParamsT<double>& p,
                      bool f32, float* f32buf, bool frozen_phi, cudaStream_t st) {
    AdjArgs a;
    a.U = U; a.V = V; a.coef = coef; a.b1 = b1; a.b2 = b2; a.out = out;
    a.f32 = f32 ? 1 : 0;
    a.frozen_phi = frozen_phi ? 1 : 0;
    a.Pf = f32buf;
    a.Vf = f32buf + (long long)NP * g.fstride;
    a.DX = a.Vf + (long long)NP * g.fstride;
    a.DY = a.DX + (long long)NP * g.ny * (g.nx + 3);
    a.LX = a.DY + (long long)NP * (g.ny + 3) * g.nx;
    a.LY = a.LX + 4LL * g.ny * (g.nx + 2);
    a.P = P; a.Cx = Cx; a.Cy = Cy; a.gbar = gbar; a.taubar = taubar;
    a.g = g; a.p = p;
    dim3 cg((g.nx + 127) / 128, g.ny);
    mxe_adj_prims<<<cg, 128, 0, st>>>(a);
    if (f32) {
        const int npairs = (g.nx + 3) * g.ny + g.nx * (g.ny + 3);
        mxe_adj_diffs<<<(npairs + 127) / 128, 128, 0, st>>>(a);
        const int ncl = (g.nx + 2) * g.ny + g.nx * (g.ny + 2);
        mxe_adj_limiters<<<(ncl + 127) / 128, 128, 0, st>>>(a);
        mxe_adj_faces_x_f32<<<dim3((g.nx + 1 + 63) / 64, g.ny), 128, 0, st>>>(a);
        mxe_adj_faces_y_f32<<<dim3((g.nx + 63) / 64, g.ny + 1), 128, 0, st>>>(a);
    } else {
        mxe_adj_faces_x<<<dim3((g.nx + 1 + 63) / 64, g.ny), 128, 0, st>>>(a);
        mxe_adj_faces_y<<<dim3((g.nx + 63) / 64, g.ny + 1), 128, 0, st>>>(a);
    }
    mxe_adj_ghosts<<<(4 * (g.nx + g.ny) + 127) / 128, 128, 0, st>>>(a);
    mxe_adj_cells<<<cg, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mxe
