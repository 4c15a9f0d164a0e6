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
// formulas whose terms all scale with dU (prim_increment14 / _p), so the
// bulk-motion cancellation of a conserved-to-primitive conversion never
// happens in FP32.  W is re-derived from U in FP64 every few steps (inside
// the final stage of that step, or by mxe_resync14_2d when the state is set)
// so that its FP32 rounding does not accumulate.
// Face states whose closure is ill-conditioned (sigma in [sigma_lim,
// sig_lo) near the Junk subspace, sigma > sig_hi near the realizability
// boundary, or det P* < det_min) are re-evaluated in FP64.
//
// Same tiling as the FP64 kernel: 15 x 16 cells per block, 2-cell halo in
// shared memory, one thread per face; instantiated for the general and the
// planar (ten-moment) state.
#include "mxe_internal.h"
#include "mxe_mixed_x2.cuh"

namespace mxe {

constexpr int TXm = 15, TYm = 16, NTm = 256;
constexpr int BXm = TXm + 4, BYm = TYm + 4;
constexpr int NBOXm = BXm * BYm;
constexpr int NPHXm = (TXm + 2) * TYm;
constexpr int NPHYm = TXm * (TYm + 2);



__device__ __forceinline__ const double* map_cell_m(const Grid2D& g, int& gi, int& gj) {
    bool xin = (gi >= 0 && gi < g.nx), yin = (gj >= 0 && gj < g.ny);
    if (!xin && yin) {
        int s = gi < 0 ? 0 : 1;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gi = ((gi % g.nx) + g.nx) % g.nx;
            return nullptr;
        }
        for (int n = 0; n < sd.nspans; ++n)
            if (gj >= sd.lo[n] && gj <= sd.hi[n]) return g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
        if (sd.type == 2) return g.ghost + (s * GHOST_SLOTS) * 14;
        gi = gi < 0 ? 0 : g.nx - 1;
    } else if (xin && !yin) {
        int s = gj < 0 ? 2 : 3;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gj = ((gj % g.ny) + g.ny) % g.ny;
            return nullptr;
        }
        for (int n = 0; n < sd.nspans; ++n)
            if (gi >= sd.lo[n] && gi <= sd.hi[n]) return g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
        if (sd.type == 2) return g.ghost + (s * GHOST_SLOTS) * 14;
        gj = gj < 0 ? 0 : g.ny - 1;
    } else if (!xin && !yin) {
        gi = gi < 0 ? 0 : g.nx - 1;
        gj = gj < 0 ? 0 : g.ny - 1;
    }
    return nullptr;
}

template <class PH>
__device__ __forceinline__ void load_prim_f32(const Stage2DArgs& a, int gi, int gj, float* Q) {
    const Grid2D& g = a.g;
    const double* gs = map_cell_m(g, gi, gj);
    if (gs) {
#pragma unroll
        for (int k = 0; k < PH::NF; ++k) Q[k] = (float)gs[PH::ufield(k)];
        return;
    }
    const float* p = a.Win + (long long)gj * g.pitch + gi;
#pragma unroll
    for (int k = 0; k < PH::NF; ++k) Q[k] = __ldg(p + k * g.fstride);
}

template <int NF>
__device__ __forceinline__ float phi_box_m(const float* W, int c, int stride, int lim) {
    float phi = 1.0f;
    const FlatRef<float> fr = flat_ref<NF>(W + c, NBOXm);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * NBOXm + c;
        float dm = w[0] - w[-stride], dp = w[stride] - w[0];
        float pk;
        if (dm * dp > 0.0f) {
            if (lim == 1) {      // approximate quotient (2 ulp): the limiter is a ratio
                pk = __fdividef(2.0f * dm * dp, dm * dm + dp * dp);
            } else {
                float am = fabsf(dm), ap = fabsf(dp);
                pk = __fdividef(2.0f * fminf(am, ap), am + ap);
            }
        } else {
            pk = (dm == 0.0f && dp == 0.0f) ? 1.0f : 0.0f;
        }
        if (pk < phi) {          // a flat field (phi_k = 1) never lowers phi
            const float m = abs_max(dm, dp);
            if (!(m <= FLAT_REL_F32 * fabsf(w[0]) || field_flat<NF>(fr, k, m))) phi = pk;
        }
    }
    return phi;
}

// Shared limiter of box cell c in x (result .x) and y (.y): the stencil
// centre and the flat-test reference are loaded once for both directions.
template <int NF, int NBOX, int BX>
__device__ __forceinline__ float2 phi_pair_m(const float* W, int c, int lim) {
    using namespace x2;
    const FlatRef<float> fr = flat_ref<NF>(W + c, NBOX);
    float nx = 1.0f, xx = 1.0f, ny = 1.0f, xy = 1.0f;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * NBOX + c;
        const float w0 = w[0];
        // the x and y differences as the lanes of packed subtractions
        const v2 dm = sub(S(w0), make_float2(w[-1], w[-BX]));
        const v2 dp = sub(make_float2(w[1], w[BX]), S(w0));
        phi_ratio_step<NF>(dm.x, dp.x, w0, fr, k, nx, xx);
        phi_ratio_step<NF>(dm.y, dp.y, w0, fr, k, ny, xy);
    }
    return make_float2(phi_of_ratio(nx, xx, lim), phi_of_ratio(ny, xy, lim));
}

template <int NF>
__device__ __forceinline__ void face_prims_m(const float* W, int c, int stride, float phi,
                                             float hs, float* Qf) {
    float hp = hs * phi;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * NBOXm + c;
        float cen = 0.5f * (w[stride] - w[-stride]);
        Qf[k] = w[0] + hp * cen;
    }
}

// Face flux of face `tid` in direction K; the left face state is staged in
// this thread's column of Ls to keep register pressure low.
template <class PH, int K>
__device__ __forceinline__ void face_flux_m(const float* W, int cl, int cr, int stride, float phl,
                                            float phr, const ParamsT<float>& p,
                                            const MixedPolicy& mp, double sl64, double kw64,
                                            float* Ls, float* F, unsigned& nflag) {
    constexpr int NF = PH::NF;
    constexpr int FS = 2 * NF + 2;
    float Qf[NF], R[FS], Lv[FS];
    face_prims_m<NF>(W, cl, stride, phl, 0.5f, Qf);
    nflag += face_state_m<PH, K>(Qf, p, mp, sl64, kw64, Lv) ? 1u : 0u;
#pragma unroll
    for (int n = 0; n < FS; ++n) Ls[n * NTm] = Lv[n];
    face_prims_m<NF>(W, cr, stride, phr, -0.5f, Qf);
    nflag += face_state_m<PH, K>(Qf, p, mp, sl64, kw64, R) ? 1u : 0u;
    float lminL = Ls[(2 * NF) * NTm], lmaxL = Ls[(2 * NF + 1) * NTm];
    float lminR = R[2 * NF], lmaxR = R[2 * NF + 1];
    if (p.flux == 1) {
        float s = fmaxf(fmaxf(fabsf(lminL), fabsf(lmaxL)), fmaxf(fabsf(lminR), fabsf(lmaxR)));
#pragma unroll
        for (int k = 0; k < NF; ++k)
            F[k] = 0.5f * (Ls[(NF + k) * NTm] + R[NF + k]) - 0.5f * s * (R[k] - Ls[k * NTm]);
        return;
    }
    float SL = fminf(lminL, lminR), SR = fmaxf(lmaxL, lmaxR);
    if (SL >= 0.0f) {
#pragma unroll
        for (int k = 0; k < NF; ++k) F[k] = Ls[(NF + k) * NTm];
    } else if (SR <= 0.0f) {
#pragma unroll
        for (int k = 0; k < NF; ++k) F[k] = R[NF + k];
    } else {
        float inv = 1.0f / (SR - SL);
        float cl_ = SR * inv, cr_ = -SL * inv, cu = SL * SR * inv;
#pragma unroll
        for (int k = 0; k < NF; ++k)
            F[k] = cl_ * Ls[(NF + k) * NTm] + cr_ * R[NF + k] + cu * (R[k] - Ls[k * NTm]);
    }
}

__device__ __forceinline__ void block_max_atomic_m(float r, unsigned long long* dst, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = r;
    __syncthreads();
    if (wid == 0) {
        r = lane < (NTm / 32) ? red[lane] : 0.0f;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (lane == 0)
            atomicMax(dst, (unsigned long long)__double_as_longlong((double)r));
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

// Own-cell prefetch of the final stage (U^n FP64 and W^n FP32 into shared
// memory at kernel start): an option of the ten-field planar state at two
// blocks per SM (at three blocks per SM its shared memory does not fit, and
// the same cells are prefetched into L2 instead).
template <int NF, bool PFON>
constexpr int prefetch_cells() { return (PFON && NF == NP) ? TXm * TYm : 0; }

// shared memory: own-cell prefetch, stencil box, x face fluxes, staged
// left face states (whose first NF rows then hold the y face fluxes),
// limiters, reduction scratch
template <int NF, bool PFON>
constexpr size_t smem_mixed() {
    return sizeof(double) * (NF * prefetch_cells<NF, PFON>()) +
           sizeof(float) * (NF * prefetch_cells<NF, PFON>() + NF * NBOXm + NF * NTm +
                            (2 * NF + 2) * NTm + NPHXm + NPHYm + 8);
}

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}


template <class PH, bool PFON>
__device__ __forceinline__ void stage_mixed(const Stage2DArgs& a, const ParamsT<float>& p,
                                            const MixedPolicy& mp) {
    constexpr int NF = PH::NF;
    constexpr int NC = TXm * TYm;
    constexpr int PF = prefetch_cells<NF, PFON>();
    extern __shared__ __align__(16) double smd[];
    double* Upf = smd;                               // [NF][PF] own-cell U^n (final stage)
    float* Wpf = (float*)(Upf + NF * PF);            // [NF][PF] own-cell W^n (final stage)
    float* W = Wpf + NF * PF;                        // [NF][BY][BX]
    float* Fx = W + NF * NBOXm;                      // [NF][256] x-face fluxes
    float* Ls = Fx + NF * NTm;                       // [2NF+2][256] left face states
    // y-face fluxes: column tid of Ls, written by thread tid once its y face
    // is done with the staged left state (no other thread uses that column)
    float* Fy = Ls;
    float* phx = Ls + (2 * NF + 2) * NTm;            // [TY][TX+2]
    float* phy = phx + NPHXm;                        // [TY+2][TX]
    float* red = phy + NPHYm;                        // [8]
    __shared__ double sdt[2];
    __shared__ unsigned cnt;

    const int tid = threadIdx.x;
    if (tid == 0) {
        double tt;
        sdt[0] = step_dt_m(a.clk, a.slot, a.cfl, a.t_end, a.dt_fixed, tt);
        sdt[1] = tt;
        cnt = 0u;
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
            if (a.dt_hist && a.clk->steps < a.dt_hist_cap) a.dt_hist[a.clk->steps] = dt;
            a.clk->steps += 1;
        }
    }
    if (!(dt > 0.0)) return;

    const Grid2D& g = a.g;
    const int i0 = blockIdx.x * TXm, j0 = blockIdx.y * TYm;
    const int cx = tid % TXm, cy = tid / TXm;
    const bool owner = tid < NC;
    const int gi = i0 + cx, gj = j0 + cy;
    const bool inside = owner && gi < g.nx && gj < g.ny;
    const long long o = (long long)gj * g.pitch + gi;
    // final stage: start fetching this cell's U^n and W^n now; they are
    // needed only after all face fluxes are done (into shared memory, or
    // into L2 where there is no room)
    if (PF && a.final_stage && inside) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            cp_async8(Upf + k * PF + tid, a.Ubase + o + PH::ufield(k) * g.fstride);
            cp_async4(Wpf + k * PF + tid, a.Wbase + o + k * g.fstride);
        }
    } else if (a.final_stage && inside) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Ubase + o + PH::ufield(k) * g.fstride));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Wbase + o + k * g.fstride));
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    for (int c = tid; c < NBOXm; c += NTm) {
        int bx = c % BXm, by = c / BXm;
        float Q[NF];
        load_prim_f32<PH>(a, i0 + bx - 2, j0 + by - 2, Q);
#pragma unroll
        for (int k = 0; k < NF; ++k) W[k * NBOXm + c] = Q[k];
    }
    __syncthreads();
    for (int n = tid; n < NPHXm + NPHYm; n += NTm) {
        float v = 0.0f;
        if (n < NPHXm) {
            int bx = 1 + n % (TXm + 2), by = 2 + n / (TXm + 2);
            if (p.order == 2) v = phi_box_m<NF>(W, by * BXm + bx, 1, p.limiter);
            phx[n] = v;
        } else {
            int m = n - NPHXm;
            int bx = 2 + m % TXm, by = 1 + m / TXm;
            if (p.order == 2) v = phi_box_m<NF>(W, by * BXm + bx, BXm, p.limiter);
            phy[m] = v;
        }
    }
    __syncthreads();

    const double sl64 = a.sp.sigma_lim, kw64 = a.sp.k_ws;
    unsigned nflag = 0;
    {   // x face tid, then y face tid (no barrier in between)
        int fx = tid & 15, fcy = tid >> 4, by = fcy + 2;
        float F[NF];
        face_flux_m<PH, 0>(W, by * BXm + fx + 1, by * BXm + fx + 2, 1, phx[fcy * (TXm + 2) + fx],
                           phx[fcy * (TXm + 2) + fx + 1], p, mp, sl64, kw64, Ls + tid, F, nflag);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fx[k * NTm + tid] = F[k];
        if (tid < TXm * (TYm + 1)) {
            int fcx = tid % TXm, fy = tid / TXm, bx = fcx + 2;
            face_flux_m<PH, 1>(W, (fy + 1) * BXm + bx, (fy + 2) * BXm + bx, BXm,
                               phy[fy * TXm + fcx], phy[(fy + 1) * TXm + fcx], p, mp, sl64, kw64,
                               Ls + tid, F, nflag);
#pragma unroll
            for (int k = 0; k < NF; ++k) Fy[k * NTm + tid] = F[k];
        }
    }
    // final stage without the shared-memory prefetch: load this cell's U^n
    // and W^n now, so that their latency overlaps the barrier and the
    // source and flux-difference arithmetic below
    double Ureg[PF ? 1 : NF];
    float Wreg[PF ? 1 : NF];
    if (!PF && a.final_stage && inside) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            Ureg[k] = a.Ubase[o + PH::ufield(k) * g.fstride];
            Wreg[k] = a.Wbase[o + k * g.fstride];
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();

    float r = 0.0f;
    if (owner) {
        float L[NF];
        float Qc[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Qc[k] = W[k * NBOXm + (cy + 2) * BXm + cx + 2];
        if (p.tau_model != 0 && !p.src_implicit) {
            PH::source(Qc, PH::tau(p, Qc), L);
        } else {
#pragma unroll
            for (int k = 0; k < NF; ++k) L[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            L[k] -= (Fx[k * NTm + cy * 16 + cx + 1] - Fx[k * NTm + cy * 16 + cx]) * a.idxf;
            L[k] -= (Fy[k * NTm + (cy + 1) * TXm + cx] - Fy[k * NTm + cy * TXm + cx]) * a.idyf;
        }
        if (inside) {
            float cdt = (float)(a.coef * dt);
            float dU[NF], Wc[NF], Wn[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) dU[k] = cdt * L[k];
            const bool implicit = p.tau_model != 0 && p.src_implicit;
            if (!a.final_stage) {
                // W* = prim(U^n + dt/2 L): base primitives are this cell's W^n (= stencil)
#pragma unroll
                for (int k = 0; k < NF; ++k) Wc[k] = W[k * NBOXm + (cy + 2) * BXm + cx + 2];
                PH::increment(Wc, dU, Wn);
                if (implicit) {      // point-implicit source over cdt
                    float N[NF];
                    PH::relax_prim(Wn, 1.0f / (1.0f + cdt / PH::tau(p, Wn)), N);
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) a.Wout[o + k * g.fstride] = Wn[k];
            } else {
                bool bad = false;
#pragma unroll
                for (int k = 0; k < NF; ++k) Wc[k] = PF ? Wpf[k * PF + tid] : Wreg[k];
                PH::increment(Wc, dU, Wn);
                if (implicit) {      // relax W, and U by (g - 1)(U - U_M)
                    float N[NF];
                    float gm = 1.0f / (1.0f + cdt / PH::tau(p, Wn));
                    PH::relax_prim(Wn, gm, N);
#pragma unroll
                    for (int k = 0; k < NF; ++k) dU[k] += (gm - 1.0f) * N[k];
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    double ub = PF ? Upf[k * PF + tid] : Ureg[k];
                    double un = ub + (double)dU[k];
                    a.Uout[o + PH::ufield(k) * g.fstride] = un;
                    bad |= !isfinite(un);
                }
                if (a.resync) {      // the periodic re-sync: W^{n+1} = prim(U^{n+1}) in FP64
                    double Un[NF], Q64[NF];
#pragma unroll
                    for (int k = 0; k < NF; ++k) Un[k] = a.Uout[o + PH::ufield(k) * g.fstride];
                    PH::cons2prim_fast(Un, Q64);
#pragma unroll
                    for (int k = 0; k < NF; ++k) Wn[k] = (float)Q64[k];
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) a.Wout[o + k * g.fstride] = Wn[k];
                if (PH::nonpositive(Wn)) atomicOr(&a.clk->status, ST_NONPOSITIVE);
                if (bad) atomicOr(&a.clk->status, ST_NONFINITE);
                float ax, ay;
                PH::rates(Wn, p.sigma_lim, p.k_ws, ax, ay);
                r = ax * a.idxf + ay * a.idyf;
                if (!(r >= 0.0f)) r = __int_as_float(0x7f800000);     // NaN -> inf
            }
        }
    }
    unsigned wf = __reduce_add_sync(0xffffffffu, nflag);
    if ((tid & 31) == 0 && wf) atomicAdd(&cnt, wf);
    if (a.final_stage) block_max_atomic_m(r, &a.clk->rate[(a.slot + 1) % 3], red);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.clk->n_face, (unsigned long long)(2 * (16 * 16 + TXm * (TYm + 1))));
        if (cnt) atomicAdd(&a.clk->n_face64, (unsigned long long)cnt);
    }
}

extern "C" __global__ void __launch_bounds__(NTm, 2)
mxe_stage14_2d_mixed(const Stage2DArgs a, const ParamsT<float> p, const MixedPolicy mp) {
    stage_mixed<PhysGeneral, false>(a, p, mp);
}
// general state at three blocks per SM (at most 80 registers)
extern "C" __global__ void __launch_bounds__(NTm, 3)
mxe_stage14_2d_mixed_b3(const Stage2DArgs a, const ParamsT<float> p, const MixedPolicy mp) {
    stage_mixed<PhysGeneral, false>(a, p, mp);
}
extern "C" __global__ void __launch_bounds__(NTm, 2)
mxe_stage14_2d_mixed_planar(const Stage2DArgs a, const ParamsT<float> p, const MixedPolicy mp) {
    stage_mixed<PhysPlanar, true>(a, p, mp);
}
// planar state at three blocks per SM (at most 80 registers, L2 prefetch)
extern "C" __global__ void __launch_bounds__(NTm, 3)
mxe_stage14_2d_mixed_planar_b3(const Stage2DArgs a, const ParamsT<float> p,
                               const MixedPolicy mp) {
    stage_mixed<PhysPlanar, false>(a, p, mp);
}

// ---------------------------------------------------------------------------
// Packed planar stage (the default for planar states).  A block of NTP
// threads owns a TX x TY tile; every thread evaluates up to two x faces and
// two y faces as packed pairs of face states, the limiters of about two
// cells (both directions of an interior cell in one evaluation), and
// updates up to two cells.  The tile is 31 x 15: a row of 32 x faces is one
// warp (no shared-memory bank conflicts in the face phase), the owned cells
// of a warp sit in one or two rows (124-byte segments of each field in
// global memory), and against the 15 x 16 tile of the scalar kernels the
// halo cells loaded, the limiters evaluated and the faces computed twice
// per owned cell, and the per-block fixed work, are about halved.
template <int TX_, int TY_>
struct TileGeo {
    static constexpr int TX = TX_, TY = TY_;
    static constexpr int BX = TX + 4, BY = TY + 4, NBOX = BX * BY;
    static constexpr int NC = TX * TY;             // owned cells
    static constexpr int NFX = (TX + 1) * TY;      // x faces
    static constexpr int NFY = TX * (TY + 1);      // y faces
    static constexpr int NPX = (TX + 2) * TY;      // x limiters
    static constexpr int NPY = TX * (TY + 2);      // y limiters
    // limiter work items: the owned cells (both directions), then the halo
    // columns (x only) and the halo rows (y only)
    static constexpr int NLIM = NC + 2 * TY + 2 * TX;
};
using TileP = TileGeo<31, 15>;
constexpr int NTP = 256;
static_assert(TileP::NFX <= 2 * NTP && TileP::NFY <= 2 * NTP && TileP::NC <= 2 * NTP,
              "two faces per direction and two cells per thread");

// shared memory of the packed stage: stencil box, x and y face fluxes,
// limiters, reduction scratch
template <class G>
constexpr size_t smem_mixed_x2() {
    return sizeof(float) * (NP * G::NBOX + NP * G::NFX + NP * G::NFY + G::NPX + G::NPY + 8);
}

template <class G>
__device__ __forceinline__ void stage_mixed_x2(const Stage2DArgs& a, const ParamsT<float>& p,
                                               const MixedPolicy& mp) {
    using PH = PhysPlanar;
    constexpr int NF = NP;
    extern __shared__ __align__(16) double smd[];
    float* W = (float*)smd;                          // [NF][BY][BX]
    float* Fx = W + NF * G::NBOX;                    // [NF][TY][TX+1]
    float* Fy = Fx + NF * G::NFX;                    // [NF][TY+1][TX]
    float* phx = Fy + NF * G::NFY;                   // [TY][TX+2]
    float* phy = phx + G::NPX;                       // [TY+2][TX]
    float* red = phy + G::NPY;                       // [8]
    __shared__ double sdt[2];
    __shared__ float scdt;
    __shared__ unsigned cnt;

    const int tid = threadIdx.x;
    if (tid == 0) {
        double tt;
        sdt[0] = step_dt_m(a.clk, a.slot, a.cfl, a.t_end, a.dt_fixed, tt);
        sdt[1] = tt;
        scdt = (float)(a.coef * sdt[0]);
        cnt = 0u;
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
            if (a.dt_hist && a.clk->steps < a.dt_hist_cap) a.dt_hist[a.clk->steps] = dt;
            a.clk->steps += 1;
        }
    }
    if (!(dt > 0.0)) return;

    const Grid2D& g = a.g;
    const int i0 = blockIdx.x * G::TX, j0 = blockIdx.y * G::TY;
    // final stage: the owned cells' U^n and W^n are needed only after the
    // face fluxes; start moving them into L2 now
    if (a.final_stage) {
        for (int c = tid; c < G::NC; c += NTP) {
            const int gi = i0 + c % G::TX, gj = j0 + c / G::TX;
            if (gi < g.nx && gj < g.ny) {
                const long long o = (long long)gj * g.pitch + gi;
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Ubase + o + PH::ufield(k) * g.fstride));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Wbase + o + k * g.fstride));
                }
            }
        }
    }
    const bool interior = i0 >= 2 && j0 >= 2 && i0 + G::TX + 2 <= g.nx && j0 + G::TY + 2 <= g.ny;
    if (interior) {      // the whole box inside the grid: asynchronous copies, no ghost cells
        const float* src = a.Win + (long long)(j0 - 2) * g.pitch + (i0 - 2);
        for (int c = tid; c < G::NBOX; c += NTP) {
            const float* s0 = src + (long long)(c / G::BX) * g.pitch + c % G::BX;
#pragma unroll
            for (int k = 0; k < NF; ++k) cp_async4(W + k * G::NBOX + c, s0 + k * g.fstride);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    } else {
        for (int c = tid; c < G::NBOX; c += NTP) {
            const int bx = c % G::BX, by = c / G::BX;
            float Q[NF];
            load_prim_f32<PH>(a, i0 + bx - 2, j0 + by - 2, Q);
#pragma unroll
            for (int k = 0; k < NF; ++k) W[k * G::NBOX + c] = Q[k];
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    for (int n = tid; n < G::NLIM; n += NTP) {
        if (n < G::NC) {                   // owned cell: both directions
            const int bx = 2 + n % G::TX, by = 2 + n / G::TX;
            float2 v = make_float2(0.0f, 0.0f);
            if (p.order == 2) v = phi_pair_m<NF, G::NBOX, G::BX>(W, by * G::BX + bx, p.limiter);
            phx[(by - 2) * (G::TX + 2) + bx - 1] = v.x;
            phy[(by - 1) * G::TX + bx - 2] = v.y;
        } else if (n < G::NC + 2 * G::TY) {     // halo column: x only
            const int m = n - G::NC;
            const int bx = (m < G::TY) ? 1 : G::TX + 2, by = 2 + m % G::TY;
            float v = 0.0f;
            if (p.order == 2) v = phi_one_m<NF, G::NBOX>(W, by * G::BX + bx, 1, p.limiter);
            phx[(by - 2) * (G::TX + 2) + bx - 1] = v;
        } else {                                // halo row: y only
            const int m = n - G::NC - 2 * G::TY;
            const int by = (m < G::TX) ? 1 : G::TY + 2, bx = 2 + m % G::TX;
            float v = 0.0f;
            if (p.order == 2) v = phi_one_m<NF, G::NBOX>(W, by * G::BX + bx, G::BX, p.limiter);
            phy[(by - 1) * G::TX + bx - 2] = v;
        }
    }
    __syncthreads();

    const double sl64 = a.sp.sigma_lim, kw64 = a.sp.k_ws;
    unsigned nflag = 0;
#pragma unroll 1
    for (int f = tid; f < G::NFX; f += NTP) {       // x faces: TY rows of TX + 1
        const int fx = f % (G::TX + 1), fy = f / (G::TX + 1);
        float F[NF];
        face_flux_x2<0, G::NBOX>(W, (fy + 2) * G::BX + fx + 1, 1, phx[fy * (G::TX + 2) + fx],
                                 phx[fy * (G::TX + 2) + fx + 1], p, mp, sl64, kw64, F, nflag);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fx[k * G::NFX + f] = F[k];
    }
#pragma unroll 1
    for (int f = tid; f < G::NFY; f += NTP) {       // y faces: TY + 1 rows of TX
        const int fx = f % G::TX, fy = f / G::TX;
        float F[NF];
        face_flux_x2<1, G::NBOX>(W, (fy + 1) * G::BX + fx + 2, G::BX, phy[fy * G::TX + fx],
                                 phy[(fy + 1) * G::TX + fx], p, mp, sl64, kw64, F, nflag);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fy[k * G::NFY + f] = F[k];
    }
    __syncthreads();

    float r = 0.0f;
    const float cdt = scdt;
    const bool implicit = p.tau_model != 0 && p.src_implicit;
#pragma unroll 1
    for (int c = tid; c < G::NC; c += NTP) {
        const int cx = c % G::TX, cy = c / G::TX;
        const int gi = i0 + cx, gj = j0 + cy;
        if (gi >= g.nx || gj >= g.ny) continue;
        const long long o = (long long)gj * g.pitch + gi;
        const int cb = (cy + 2) * G::BX + cx + 2;
        // final stage: this cell's W^n and U^n, loaded first so that their
        // latency overlaps the source and flux-difference arithmetic
        float Wc[NF];
        double Ub[NF];
        if (a.final_stage) {
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                Wc[k] = a.Wbase[o + k * g.fstride];
                Ub[k] = a.Ubase[o + PH::ufield(k) * g.fstride];
            }
        }
        float L[NF], Qc[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Qc[k] = W[k * G::NBOX + cb];
        if (p.tau_model != 0 && !p.src_implicit) {
            PH::source(Qc, PH::tau(p, Qc), L);
        } else {
#pragma unroll
            for (int k = 0; k < NF; ++k) L[k] = 0.0f;
        }
        const int ex = cy * (G::TX + 1) + cx, ey = cy * G::TX + cx;
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            L[k] -= (Fx[k * G::NFX + ex + 1] - Fx[k * G::NFX + ex]) * a.idxf;
            L[k] -= (Fy[k * G::NFY + ey + G::TX] - Fy[k * G::NFY + ey]) * a.idyf;
        }
        float dU[NF], Wn[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) dU[k] = cdt * L[k];
        if (!a.final_stage) {
            // W* = prim(U^n + dt/2 L): the base primitives are this cell's W^n (= stencil)
            PH::increment(Qc, dU, Wn);
            if (implicit) {      // point-implicit source over cdt
                float N[NF];
                PH::relax_prim(Wn, 1.0f / (1.0f + cdt / PH::tau(p, Wn)), N);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) a.Wout[o + k * g.fstride] = Wn[k];
        } else {
            PH::increment(Wc, dU, Wn);
            if (implicit) {      // relax W, and U by (g - 1)(U - U_M)
                float N[NF];
                float gm = 1.0f / (1.0f + cdt / PH::tau(p, Wn));
                PH::relax_prim(Wn, gm, N);
#pragma unroll
                for (int k = 0; k < NF; ++k) dU[k] += (gm - 1.0f) * N[k];
            }
            // U^{n+1} = U^n + dU in FP64 (the conservation accumulator);
            // a non-finite increment marks the state non-finite
            bool bad = false;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                a.Uout[o + PH::ufield(k) * g.fstride] = Ub[k] + f32_to_f64_bits(dU[k]);
                bad |= !(fabsf(dU[k]) < __int_as_float(0x7f800000));
            }
            if (a.resync) {      // the periodic re-sync: W^{n+1} = prim(U^{n+1}) in FP64
                double Un[NF], Q64[NF];
#pragma unroll
                for (int k = 0; k < NF; ++k) Un[k] = a.Uout[o + PH::ufield(k) * g.fstride];
                PH::cons2prim_fast(Un, Q64);
#pragma unroll
                for (int k = 0; k < NF; ++k) Wn[k] = (float)Q64[k];
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) a.Wout[o + k * g.fstride] = Wn[k];
            if (PH::nonpositive(Wn)) atomicOr(&a.clk->status, ST_NONPOSITIVE);
            if (bad) atomicOr(&a.clk->status, ST_NONFINITE);
            float ax, ay;
            x2::rates_x2(Wn, p.sigma_lim, p.k_ws, ax, ay);
            float rc = ax * a.idxf + ay * a.idyf;
            if (!(rc >= 0.0f)) rc = __int_as_float(0x7f800000);     // NaN -> inf
            r = fmaxf(r, rc);
        }
    }
    unsigned wf = __reduce_add_sync(0xffffffffu, nflag);
    if ((tid & 31) == 0 && wf) atomicAdd(&cnt, wf);
    if (a.final_stage) block_max_atomic_m(r, &a.clk->rate[(a.slot + 1) % 3], red);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&a.clk->n_face, (unsigned long long)(2 * (G::NFX + G::NFY)));
        if (cnt) atomicAdd(&a.clk->n_face64, (unsigned long long)cnt);
    }
}

// planar state, packed face-state pairs, 15 x 32 tile, three blocks per SM
extern "C" __global__ void __launch_bounds__(NTP, 3)
mxe_stage14_2d_mixed_planar_x2(const Stage2DArgs a, const ParamsT<float> p,
                               const MixedPolicy mp) {
    stage_mixed_x2<TileP>(a, p, mp);
}
size_t stage14_2d_mixed_x2_smem() { return smem_mixed_x2<TileP>(); }
int stage14_2d_mixed_x2_tile_x() { return TileP::TX; }
int stage14_2d_mixed_x2_tile_y() { return TileP::TY; }

size_t stage14_2d_mixed_smem(bool planar, int blocks_per_sm) {
    if (!planar) return smem_mixed<14, false>();      // both general variants
    return blocks_per_sm >= 3 ? smem_mixed<NP, false>() : smem_mixed<NP, true>();
}

// W = FP32 primitives of U, converted in FP64 (set-up and periodic re-sync).
template <class PH>
__device__ __forceinline__ void resync(const double* U, float* W, const Grid2D& g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx) return;
    long long o = (long long)j * g.pitch + i;
    double Uc[PH::NF], Q[PH::NF];
#pragma unroll
    for (int k = 0; k < PH::NF; ++k) Uc[k] = U[o + PH::ufield(k) * g.fstride];
    PH::cons2prim_fast(Uc, Q);
#pragma unroll
    for (int k = 0; k < PH::NF; ++k) W[o + k * g.fstride] = (float)Q[k];
}
extern "C" __global__ void mxe_resync14_2d(const double* U, float* W, Grid2D g) {
    resync<PhysGeneral>(U, W, g);
}
extern "C" __global__ void mxe_resync14_2d_planar(const double* U, float* W, Grid2D g) {
    resync<PhysPlanar>(U, W, g);
}

// Initial CFL rate from the FP32 primitives.
template <class PH>
__device__ __forceinline__ void rate_mixed(const float* W, const Grid2D& g, const ParamsT<float>& p,
                                           float idxf, float idyf, DevClock* clk, int slot) {
    __shared__ float red[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    float r = 0.0f;
    if (i < g.nx) {
        long long o = (long long)j * g.pitch + i;
        float Q[PH::NF];
#pragma unroll
        for (int k = 0; k < PH::NF; ++k) Q[k] = W[o + k * g.fstride];
        float ax, ay;
        PH::rates(Q, p.sigma_lim, p.k_ws, ax, ay);
        r = ax * idxf + ay * idyf;
        if (!(r >= 0.0f)) r = __int_as_float(0x7f800000);
    }
    block_max_atomic_m(r, &clk->rate[slot], red);
}
extern "C" __global__ void mxe_rate14_2d_mixed(const float* W, Grid2D g, ParamsT<float> p,
                                               float idxf, float idyf, DevClock* clk, int slot) {
    rate_mixed<PhysGeneral>(W, g, p, idxf, idyf, clk, slot);
}
extern "C" __global__ void mxe_rate14_2d_mixed_planar(const float* W, Grid2D g, ParamsT<float> p,
                                                      float idxf, float idyf, DevClock* clk,
                                                      int slot) {
    rate_mixed<PhysPlanar>(W, g, p, idxf, idyf, clk, slot);
}

}  // namespace mxe
