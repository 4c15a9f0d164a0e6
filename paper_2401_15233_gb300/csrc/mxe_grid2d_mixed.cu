// mxe_grid2d_mixed.cu -- mixed-precision fused stage for the 14-moment
// system on a 2D grid (GB300: FP64 issues at 1/64 of the FP32 rate).
//
// State: the conserved moments U^n stay in FP64 (the conservation
// accumulator).  Every stage runs in FP32 on primitive moments:
//   W   FP32 primitives of U^n        (stencil input of stage 1)
//   Ws  FP32 primitives of U*         (stage-1 output, stencil of stage 2)
// Stage 1:  L = L(W);    W*      = prim(U^n + dt/2 L)
// Stage 2:  L = L(W*);   U^{n+1} = U^n + dt L (FP64 add of the FP32
//           increment);  W^{n+1} = prim(U^{n+1})
// The primitives of U + dU are formed from the FP32 increment dU with
// formulas whose terms all scale with dU (prim_increment14), so the
// bulk-motion cancellation of a conserved-to-primitive conversion never
// happens in FP32.  W is re-derived from U in FP64 every few steps
// (mxe_resync14_2d) so that its FP32 rounding does not accumulate.
// Face states whose closure is ill-conditioned (sigma in [sigma_lim,
// sig_lo) near the Junk subspace, sigma > sig_hi near the realizability
// boundary, or det P* < det_min) are re-evaluated in FP64.
//
// Same tiling as the FP64 kernel: 15 x 16 cells per block, 2-cell halo in
// shared memory, one thread per face.
#include "mxe_internal.h"

namespace mxe {

constexpr int TXm = 15, TYm = 16, NTm = 256;
constexpr int BXm = TXm + 4, BYm = TYm + 4;
constexpr int NPHXm = (TXm + 2) * TYm;
constexpr int NPHYm = TXm * (TYm + 2);
constexpr int FS = 30;                               // U(14) F(14) lmin lmax

struct MixedPolicy {
    float sig_lo, sig_hi, det_min;
};

__device__ __forceinline__ void load_prim_f32(const Stage2DArgs& a, int gi, int gj, float* Q) {
    const Grid2D& g = a.g;
    bool xin = (gi >= 0 && gi < g.nx), yin = (gj >= 0 && gj < g.ny);
    const double* gs = nullptr;
    if (!xin && yin) {
        int s = gi < 0 ? 0 : 1;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gi = ((gi % g.nx) + g.nx) % g.nx;
        } else {
            for (int n = 0; n < sd.nspans; ++n)
                if (gj >= sd.lo[n] && gj <= sd.hi[n]) gs = g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
            if (!gs && sd.type == 2) gs = g.ghost + (s * GHOST_SLOTS) * 14;
            if (!gs) gi = gi < 0 ? 0 : g.nx - 1;
        }
    } else if (xin && !yin) {
        int s = gj < 0 ? 2 : 3;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gj = ((gj % g.ny) + g.ny) % g.ny;
        } else {
            for (int n = 0; n < sd.nspans; ++n)
                if (gi >= sd.lo[n] && gi <= sd.hi[n]) gs = g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
            if (!gs && sd.type == 2) gs = g.ghost + (s * GHOST_SLOTS) * 14;
            if (!gs) gj = gj < 0 ? 0 : g.ny - 1;
        }
    } else if (!xin && !yin) {
        gi = gi < 0 ? 0 : g.nx - 1;
        gj = gj < 0 ? 0 : g.ny - 1;
    }
    if (gs) {
#pragma unroll
        for (int k = 0; k < 14; ++k) Q[k] = (float)gs[k];
        return;
    }
    const float* p = a.Win + (long long)gj * g.pitch + gi;
#pragma unroll
    for (int k = 0; k < 14; ++k) Q[k] = __ldg(p + k * g.fstride);
}

// FP64 re-evaluation of one face state (kept out of line: rare path)
template <int K>
__device__ __noinline__ void face_eval14_fp64(const float* Qf, const SchemeParams& sp, float* out) {
    double Q[14], U[14], F[14], lo, hi;
#pragma unroll
    for (int k = 0; k < 14; ++k) Q[k] = (double)Qf[k];
    face_eval14<double, K>(Q, sp, U, F, lo, hi);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        out[k] = (float)U[k];
        out[14 + k] = (float)F[k];
    }
    out[28] = (float)lo;
    out[29] = (float)hi;
}

// One face state: conserved U, flux F, wave speeds into out[30]; FP64
// re-evaluation where the closure is ill-conditioned.  Returns the flag.
template <int K>
__device__ __forceinline__ bool face_state_eval(const float* Qf, const SchemeParams& sp,
                                                const MixedPolicy& mp, float* out) {
    Dimless14<float> d;
    dimless14(Qf, d);
    float sb = clamp_sigma(d.sig, (float)sp.sigma_lim);
    bool flag = (d.sig >= (float)sp.sigma_lim && d.sig < mp.sig_lo) || d.sig > mp.sig_hi ||
                d.det < mp.det_min || !(d.sig == d.sig);
    float Qk[6], Rk[3], Sk;
    closure14_slice<float, K>(Qf, d, sb, Qk, Rk, Sk);
    prim2cons14(Qf, out);
    flux14<float, K>(Qf, out, Qk, Rk, Sk, out + 14);
    float lp, lm;
    lam14_star<float, K>(d, sb, lp, lm);
    float k = (float)sp.k_ws;
    out[29] = Qf[1 + K] + k * lp * d.sq;
    out[28] = Qf[1 + K] + k * lm * d.sq;
    if (__any_sync(__activemask(), flag)) {
        if (flag) face_eval14_fp64<K>(Qf, sp, out);
    }
    return flag;
}

template <class T>
__device__ __forceinline__ T phi_box_m(const T* W, int c, int stride, int lim) {
    T phi = T(1);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const T* w = W + k * BXm * BYm + c;
        T pk = phi_field(w[0] - w[-stride], w[stride] - w[0], lim);
        phi = pk < phi ? pk : phi;
    }
    return phi;
}

// Face flux of face `tid` in direction K; L face state staged in Ls (per
// thread slot) to keep register pressure low.
template <int K>
__device__ __forceinline__ void face_flux_m(const float* W, int cl, int cr, int stride, float phl,
                                            float phr, const SchemeParams& sp,
                                            const MixedPolicy& mp, float* Ls, float* F,
                                            unsigned& nflag) {
    float Qf[14], R[FS];
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const float* w = W + k * BXm * BYm;
        Qf[k] = muscl_face(w[cl - stride], w[cl], w[cl + stride], phl, 0.5f);
    }
    float Lv[FS];
    nflag += face_state_eval<K>(Qf, sp, mp, Lv) ? 1u : 0u;
#pragma unroll
    for (int n = 0; n < FS; ++n) Ls[n * NTm] = Lv[n];
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const float* w = W + k * BXm * BYm;
        Qf[k] = muscl_face(w[cr - stride], w[cr], w[cr + stride], phr, -0.5f);
    }
    nflag += face_state_eval<K>(Qf, sp, mp, R) ? 1u : 0u;
    float lminL = Ls[28 * NTm], lmaxL = Ls[29 * NTm];
    float lminR = R[28], lmaxR = R[29];
    if (sp.flux == 1) {
        float s = fmaxf(fmaxf(fabsf(lminL), fabsf(lmaxL)), fmaxf(fabsf(lminR), fabsf(lmaxR)));
#pragma unroll
        for (int k = 0; k < 14; ++k)
            F[k] = 0.5f * (Ls[(14 + k) * NTm] + R[14 + k]) - 0.5f * s * (R[k] - Ls[k * NTm]);
        return;
    }
    float SL = fminf(lminL, lminR), SR = fmaxf(lmaxL, lmaxR);
    if (SL >= 0.0f) {
#pragma unroll
        for (int k = 0; k < 14; ++k) F[k] = Ls[(14 + k) * NTm];
    } else if (SR <= 0.0f) {
#pragma unroll
        for (int k = 0; k < 14; ++k) F[k] = R[14 + k];
    } else {
        float inv = 1.0f / (SR - SL);
#pragma unroll
        for (int k = 0; k < 14; ++k)
            F[k] = (SR * Ls[(14 + k) * NTm] - SL * R[14 + k] + SL * SR * (R[k] - Ls[k * NTm])) * inv;
    }
}

__device__ __forceinline__ void block_max_atomic_m(double r, unsigned long long* dst, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, r, o);
        r = v > r ? v : r;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = r;
    __syncthreads();
    if (wid == 0) {
        r = lane < (NTm / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            double v = __shfl_xor_sync(0xffffffffu, r, o);
            r = v > r ? v : r;
        }
        if (lane == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(r));
    }
}

__device__ __forceinline__ double step_dt_m(const DevClock* clk, int slot, double cfl,
                                            double t_end, double dt_fixed, double& t) {
    t = clk->t[slot];
    if (dt_fixed > 0.0) return dt_fixed;
    double m = __longlong_as_double((long long)clk->rate[slot]);
    double dt = cfl / m;
    if (t + dt > t_end) dt = t_end - t;
    return dt;
}

extern "C" __global__ void __launch_bounds__(NTm, 2)
mxe_stage14_2d_mixed(const Stage2DArgs a, const MixedPolicy mp) {
    extern __shared__ __align__(16) float smf[];
    float* W = smf;                                  // [14][BY][BX]
    float* Fb = W + 14 * BXm * BYm;                  // [14][256]
    float* Ls = Fb + 14 * NTm;                       // [30][256] left face states
    float* phx = Ls + FS * NTm;                      // [TY][TX+2]
    float* phy = phx + NPHXm;                        // [TY+2][TX]
    double* red = (double*)(phy + NPHYm + (NPHYm & 1));   // [8]
    unsigned* cnt = (unsigned*)(red + 8);            // [1]

    const int tid = threadIdx.x;
    __shared__ double sdt[2];
    if (tid == 0) {
        double tt;
        sdt[0] = step_dt_m(a.clk, a.slot, a.cfl, a.t_end, a.dt_fixed, tt);
        sdt[1] = tt;
    }
    __syncthreads();
    const double dt = sdt[0], t = sdt[1];
    if (a.final_stage && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        int s1 = (a.slot + 1) % 3, s2 = (a.slot + 2) % 3;
        a.clk->rate[s2] = 0ull;
        if (!(dt > 0.0)) {
            a.clk->t[s1] = t;
            a.clk->rate[s1] = a.clk->rate[a.slot];
        } else {
            a.clk->t[s1] = t + dt;
            a.clk->last_dt = dt;
            a.clk->steps += 1;
        }
    }
    if (!(dt > 0.0)) return;
    if (tid == 0) *cnt = 0u;

    const Grid2D& g = a.g;
    const int i0 = blockIdx.x * TXm, j0 = blockIdx.y * TYm;
    for (int c = tid; c < BXm * BYm; c += NTm) {
        int bx = c % BXm, by = c / BXm;
        float Q[14];
        load_prim_f32(a, i0 + bx - 2, j0 + by - 2, Q);
#pragma unroll
        for (int k = 0; k < 14; ++k) W[k * BXm * BYm + c] = Q[k];
    }
    __syncthreads();
    const int order = a.sp.order, lim = a.sp.limiter;
    for (int n = tid; n < NPHXm; n += NTm) {
        int bx = 1 + n % (TXm + 2), by = 2 + n / (TXm + 2);
        phx[n] = order == 2 ? phi_box_m(W, by * BXm + bx, 1, lim) : 0.0f;
    }
    for (int n = tid; n < NPHYm; n += NTm) {
        int bx = 2 + n % TXm, by = 1 + n / TXm;
        phy[n] = order == 2 ? phi_box_m(W, by * BXm + bx, BXm, lim) : 0.0f;
    }
    __syncthreads();

    unsigned nflag = 0;
    {
        int fx = tid & 15, cy = tid >> 4, by = cy + 2;
        float F[14];
        face_flux_m<0>(W, by * BXm + fx + 1, by * BXm + fx + 2, 1, phx[cy * (TXm + 2) + fx],
                       phx[cy * (TXm + 2) + fx + 1], a.sp, mp, Ls + tid, F, nflag);
#pragma unroll
        for (int k = 0; k < 14; ++k) Fb[k * NTm + tid] = F[k];
    }
    __syncthreads();
    const int cx = tid % TXm, cy = tid / TXm;
    const bool owner = tid < TXm * TYm;
    float L[14];
    if (owner) {
        float Qc[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) Qc[k] = W[k * BXm * BYm + (cy + 2) * BXm + cx + 2];
        if (a.rp.model != 0) {
            float tau = tau_of<float>(a.rp, Qc, 14);
            source14(Qc, tau, L);
        } else {
#pragma unroll
            for (int k = 0; k < 14; ++k) L[k] = 0.0f;
        }
        const float idx = (float)g.idx;
#pragma unroll
        for (int k = 0; k < 14; ++k)
            L[k] -= (Fb[k * NTm + cy * 16 + cx + 1] - Fb[k * NTm + cy * 16 + cx]) * idx;
    }
    __syncthreads();
    if (tid < TXm * (TYm + 1)) {
        int fcx = tid % TXm, fy = tid / TXm, bx = fcx + 2;
        float F[14];
        face_flux_m<1>(W, (fy + 1) * BXm + bx, (fy + 2) * BXm + bx, BXm, phy[fy * TXm + fcx],
                       phy[(fy + 1) * TXm + fcx], a.sp, mp, Ls + tid, F, nflag);
#pragma unroll
        for (int k = 0; k < 14; ++k) Fb[k * NTm + tid] = F[k];
    }
    __syncthreads();

    double r = 0.0;
    if (owner) {
        const float idy = (float)g.idy;
#pragma unroll
        for (int k = 0; k < 14; ++k)
            L[k] -= (Fb[k * NTm + (cy + 1) * TXm + cx] - Fb[k * NTm + cy * TXm + cx]) * idy;
        int gi = i0 + cx, gj = j0 + cy;
        if (gi < g.nx && gj < g.ny) {
            long long o = (long long)gj * g.pitch + gi;
            float cdt = (float)(a.coef * dt);
            float dU[14], Wc[14], Wn[14];
#pragma unroll
            for (int k = 0; k < 14; ++k) dU[k] = cdt * L[k];
            if (!a.final_stage) {
                // W* = prim(U^n + dt/2 L): base primitives are this cell's W^n (= stencil)
#pragma unroll
                for (int k = 0; k < 14; ++k) Wc[k] = W[k * BXm * BYm + (cy + 2) * BXm + cx + 2];
                prim_increment14(Wc, dU, Wn);
#pragma unroll
                for (int k = 0; k < 14; ++k) a.Wout[o + k * g.fstride] = Wn[k];
            } else {
                bool bad = false;
#pragma unroll
                for (int k = 0; k < 14; ++k) {
                    double un = a.Ubase[o + k * g.fstride] + (double)dU[k];
                    a.Uout[o + k * g.fstride] = un;
                    bad |= !isfinite(un);
                    Wc[k] = a.Wbase[o + k * g.fstride];
                }
                prim_increment14(Wc, dU, Wn);
#pragma unroll
                for (int k = 0; k < 14; ++k) a.Wout[o + k * g.fstride] = Wn[k];
                if (Wn[0] <= 0.0f || Wn[4] <= 0.0f || Wn[7] <= 0.0f || Wn[9] <= 0.0f)
                    atomicOr(&a.clk->status, ST_NONPOSITIVE);
                if (bad) atomicOr(&a.clk->status, ST_NONFINITE);
                Dimless14<float> d;
                dimless14(Wn, d);
                float ax = amax14<float, 0>(Wn, d, a.sp);
                float ay = amax14<float, 1>(Wn, d, a.sp);
                r = (double)(ax * (float)g.idx + ay * (float)g.idy);
                if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);
            }
        }
    }
    // counters: face states evaluated / re-evaluated in FP64
    unsigned wf = __reduce_add_sync(0xffffffffu, nflag);
    if ((tid & 31) == 0 && wf) atomicAdd(cnt, wf);
    if (a.final_stage) block_max_atomic_m(r, &a.clk->rate[(a.slot + 1) % 3], red);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.clk->n_face, (unsigned long long)(2 * (16 * 16 + TXm * (TYm + 1))));
        if (*cnt) atomicAdd(&a.clk->n_face64, (unsigned long long)*cnt);
    }
}

size_t stage14_2d_mixed_smem() {
    return sizeof(float) * (14 * BXm * BYm + 14 * NTm + FS * NTm + NPHXm + NPHYm + 1) +
           sizeof(double) * 8 + 16;
}

// W = FP32 primitives of U, converted in FP64 (set-up and periodic re-sync).
extern "C" __global__ void mxe_resync14_2d(const double* U, float* W, Grid2D g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    long long o = (long long)j * g.pitch + i;
    double Uc[14], Q[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) Uc[k] = U[o + k * g.fstride];
    cons2prim14_rn(Uc, Q);
#pragma unroll
    for (int k = 0; k < 14; ++k) W[o + k * g.fstride] = (float)Q[k];
}

// Initial CFL rate from the FP32 primitives.
extern "C" __global__ void mxe_rate14_2d_mixed(const float* W, Grid2D g, SchemeParams sp,
                                               DevClock* clk, int slot) {
    __shared__ double red[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    double r = 0.0;
    if (i < g.nx) {
        long long o = (long long)j * g.pitch + i;
        float Q[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) Q[k] = W[o + k * g.fstride];
        Dimless14<float> d;
        dimless14(Q, d);
        float ax = amax14<float, 0>(Q, d, sp);
        float ay = amax14<float, 1>(Q, d, sp);
        r = (double)(ax * (float)g.idx + ay * (float)g.idy);
        if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);
    }
    block_max_atomic_m(r, &clk->rate[slot], red);
}

}  // namespace mxe
