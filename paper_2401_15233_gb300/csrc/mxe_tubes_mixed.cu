// mxe_tubes_mixed.cu -- persistent batched solver for 14-moment problems in
// one space dimension (Sec. 2.4 system, Sec. 3 scheme), mixed precision.
//
// Precision: as in the 2D mixed kernels.  The conserved moments U stay in
// FP64 (the conservation accumulator); every stage runs in FP32 on
// primitive moments (W = prim(U^n), Ws = prim(U*)), the primitives of
// U + dU are formed from the FP32 increment with formulas whose terms all
// scale with dU, W is re-derived from U in FP64 every `resync_every` steps,
// and ill-conditioned face closures are re-evaluated in FP64.
//
// Scheduling: one persistent launch for the whole batch.  A team of CTAs
// (a thread-block cluster of 1..8 CTAs) takes one tube at a time from a
// device work queue whose order is longest-expected-work first, and marches
// it to t_end on the tube's own clock.  Within a stage the team splits the
// tube into chunks of NT-2 cells (chunk j belongs to CTA j mod team); a CTA
// stages a chunk's primitives plus a 2-cell halo in shared memory, forms one
// shared limiter per cell (NT of them: one per thread), evaluates one face
// per thread (planar states: both face states as one packed FP32 pair) and
// updates its cells.  Cluster barriers separate the stages; the team's CFL maximum and
// status bits are combined in the shared memory of CTA 0 of the cluster
// (distributed shared memory).  Every wait in this file is a hardware
// barrier reached by all threads of the team in the same order: there is no
// spin loop.
#include "mxe_internal.h"
#include "mxe_mixed_x2.cuh"

namespace mxe {

// ---- thread-block cluster primitives -------------------------------------
// A launch without cluster dimensions is a cluster of one CTA; all of these
// then act on the CTA itself.
__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cl_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// all threads of all CTAs of the cluster; release/acquire at cluster scope
__device__ __forceinline__ void cl_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// shared::cluster address of `p` (a shared variable) in CTA `rank`
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
    unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_red_max(unsigned addr, unsigned v) {
    asm volatile("red.shared::cluster.max.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_red_or(unsigned addr, unsigned v) {
    asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned cl_ld(unsigned addr) {
    unsigned v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// ---- shared-memory layout of one CTA -------------------------------------
template <int NF, int NT>
struct TubeLayout {
    static constexpr int C = NT - 2;              // cells per chunk (C + 2 limiters)
    static constexpr int BOX = C + 4;             // staged cells (chunk + 2 + 2)
    static constexpr int FS = 2 * NF + 2;         // staged left face state
    static constexpr int W_OFF = 0;               // [NF][BOX] primitives
    static constexpr int F_OFF = W_OFF + NF * BOX;   // [NF][NT] face fluxes
    static constexpr int L_OFF = F_OFF + NF * NT;    // [FS][NT] left face states
    static constexpr int P_OFF = L_OFF + FS * NT;    // [C+2] limiters
    static constexpr int R_OFF = P_OFF + C + 2;      // [NT/32] reduction scratch (rate)
    static constexpr int S_OFF = R_OFF + NT / 32;    // [NT/32] reduction scratch (status)
    static constexpr int TOTAL = S_OFF + NT / 32;
    static constexpr size_t bytes() { return sizeof(float) * TOTAL; }
};

// FP32 primitive stencil value of tube cell gi (boundary ghosts included)
template <class PH>
__device__ __forceinline__ void load_w(const TubeMixedArgs& a, const float* Wt, int n, int gi,
                                       float* Q) {
    if (gi < 0 || gi >= n) {
        int s = gi < 0 ? 0 : 1;
        int ty = a.bc_type[s];
        if (ty == 2) {
#pragma unroll
            for (int k = 0; k < PH::NF; ++k) Q[k] = (float)a.ghost[s * 14 + PH::ufield(k)];
            return;
        }
        if (ty == 1) gi = ((gi % n) + n) % n;
        else gi = gi < 0 ? 0 : n - 1;
    }
    // written by other CTAs of the team in the previous stage: read from L2
#pragma unroll
    for (int k = 0; k < PH::NF; ++k) Q[k] = __ldcg(Wt + (long long)k * n + gi);
}

// Face flux of the face between box cells cl = tid+1 and cr = tid+2; the
// left face state is staged in this thread's column of Ls.
template <class PH, int NT, int BOX>
__device__ __forceinline__ void face_flux_1d(const float* W, int cl, float phl, float phr,
                                             const ParamsT<float>& p, const MixedPolicy& mp,
                                             double sl64, double kw64, float* Ls, float* F,
                                             unsigned& nflag) {
    constexpr int NF = PH::NF;
    constexpr int FS = 2 * NF + 2;
    float Qf[NF], R[FS], Lv[FS];
    const int cr = cl + 1;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * BOX + cl;
        Qf[k] = w[0] + (0.5f * phl) * (0.5f * (w[1] - w[-1]));
    }
    nflag += face_state_m<PH, 0>(Qf, p, mp, sl64, kw64, Lv) ? 1u : 0u;
#pragma unroll
    for (int n = 0; n < FS; ++n) Ls[n * NT] = Lv[n];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float* w = W + k * BOX + cr;
        Qf[k] = w[0] - (0.5f * phr) * (0.5f * (w[1] - w[-1]));
    }
    nflag += face_state_m<PH, 0>(Qf, p, mp, sl64, kw64, R) ? 1u : 0u;
    float lminL = Ls[(2 * NF) * NT], lmaxL = Ls[(2 * NF + 1) * NT];
    float lminR = R[2 * NF], lmaxR = R[2 * NF + 1];
    if (p.flux == 1) {
        float s = fmaxf(fmaxf(fabsf(lminL), fabsf(lmaxL)), fmaxf(fabsf(lminR), fabsf(lmaxR)));
#pragma unroll
        for (int k = 0; k < NF; ++k)
            F[k] = 0.5f * (Ls[(NF + k) * NT] + R[NF + k]) - 0.5f * s * (R[k] - Ls[k * NT]);
        return;
    }
    float SL = fminf(lminL, lminR), SR = fmaxf(lmaxL, lmaxR);
    if (SL >= 0.0f) {
#pragma unroll
        for (int k = 0; k < NF; ++k) F[k] = Ls[(NF + k) * NT];
    } else if (SR <= 0.0f) {
#pragma unroll
        for (int k = 0; k < NF; ++k) F[k] = R[NF + k];
    } else {
        float inv = 1.0f / (SR - SL);
        float cl_ = SR * inv, cr_ = -SL * inv, cu = SL * SR * inv;
#pragma unroll
        for (int k = 0; k < NF; ++k)
            F[k] = cl_ * Ls[(NF + k) * NT] + cr_ * R[NF + k] + cu * (R[k] - Ls[k * NT]);
    }
}

// Per-tube view of one launch
struct TubeView {
    double* U;                  // FP64 conserved moments, 14 fields of n cells
    float* W;                   // FP32 primitives of U^n, NF fields of n cells
    float* Ws;                  // FP32 primitives of the stage state
    int n;
    float idx;                  // 1/dx
    ParamsT<float> p;           // scheme + this tube's relaxation
};

// One stage over the chunks this CTA owns:
//   L = L(Win);  dU = cdt L
//   !final:  Wout = prim(cons(W_own) + dU)  with W_own the stencil's cell
//   final:   U += dU (FP64);  Wout = prim(U) by increment from Wbase (or in
//            FP64 from the new U when `resync`);  returns the CFL rate max.
template <class PH, int NT>
__device__ float tube_stage_m(const TubeMixedArgs& a, const TubeView& v, const MixedPolicy& mp,
                              const float* Win, const float* Wbase, float* Wout, float cdt,
                              bool final, bool resync, unsigned rank, unsigned team, float* sm,
                              unsigned& status, unsigned& nflag) {
    constexpr int NF = PH::NF;
    using LY = TubeLayout<NF, NT>;
    constexpr int C = LY::C, BOX = LY::BOX;
    float* Wb = sm + LY::W_OFF;
    float* Fb = sm + LY::F_OFF;
    float* Ls = sm + LY::L_OFF;
    float* ph = sm + LY::P_OFF;
    const int tid = threadIdx.x;
    const int n = v.n;
    const ParamsT<float>& p = v.p;
    float rmax = 0.0f;
    for (int c0 = (int)rank * C; c0 < n; c0 += (int)team * C) {
        for (int i = tid; i < BOX; i += NT) {
            float Q[NF];
            load_w<PH>(a, Win, n, c0 - 2 + i, Q);
#pragma unroll
            for (int k = 0; k < NF; ++k) Wb[k * BOX + i] = Q[k];
        }
        __syncthreads();
        for (int i = tid; i < C + 2; i += NT)
            ph[i] = p.order == 2 ? phi_one_m<NF, BOX>(Wb, i + 1, 1, p.limiter) : 0.0f;
        __syncthreads();
        if (tid <= C) {                  // C + 1 faces
            float F[NF];
            if constexpr (NF == NP) {
                face_flux_x2<0, BOX>(Wb, tid + 1, 1, ph[tid], ph[tid + 1], p, mp, a.sl64,
                                     a.kw64, F, nflag);
            } else {
                face_flux_1d<PH, NT, BOX>(Wb, tid + 1, ph[tid], ph[tid + 1], p, mp, a.sl64,
                                          a.kw64, Ls + tid, F, nflag);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) Fb[k * NT + tid] = F[k];
        }
        __syncthreads();
        const int i = c0 + tid;
        if (tid < C && i < n) {
            float Qc[NF], L[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) Qc[k] = Wb[k * BOX + tid + 2];
            const bool implicit = p.tau_model != 0 && p.src_implicit;
            if (p.tau_model != 0 && !implicit) {
                PH::source(Qc, PH::tau(p, Qc), L);
            } else {
#pragma unroll
                for (int k = 0; k < NF; ++k) L[k] = 0.0f;
            }
            float dU[NF], Wn[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                L[k] -= (Fb[k * NT + tid + 1] - Fb[k * NT + tid]) * v.idx;
                dU[k] = cdt * L[k];
            }
            if (!final) {
                PH::increment(Qc, dU, Wn);
                if (implicit) {      // point-implicit source over cdt
                    float N[NF];
                    PH::relax_prim(Wn, 1.0f / (1.0f + cdt / PH::tau(p, Wn)), N);
                }
            } else {
                // U += dU in FP64 (the conservation accumulator); a
                // non-finite increment marks the state non-finite
                bool bad = false;
                double Un[NF];
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    Un[k] = v.U[(long long)PH::ufield(k) * n + i] + f32_to_f64_bits(dU[k]);
                    bad |= !(fabsf(dU[k]) < __int_as_float(0x7f800000));
                }
                if (resync) {
                    double Q64[NF];
                    PH::cons2prim_fast(Un, Q64);
#pragma unroll
                    for (int k = 0; k < NF; ++k) Wn[k] = (float)Q64[k];
                } else {
                    float Wc[NF];
#pragma unroll
                    for (int k = 0; k < NF; ++k)
                        Wc[k] = Wbase ? Wbase[(long long)k * n + i] : Qc[k];
                    PH::increment(Wc, dU, Wn);
                }
                if (implicit) {      // relax W, and U by (g - 1)(U - U_M)
                    float N[NF];
                    float gm = 1.0f / (1.0f + cdt / PH::tau(p, Wn));
                    PH::relax_prim(Wn, gm, N);
#pragma unroll
                    for (int k = 0; k < NF; ++k) Un[k] += (double)((gm - 1.0f) * N[k]);
                }
#pragma unroll
                for (int k = 0; k < NF; ++k) v.U[(long long)PH::ufield(k) * n + i] = Un[k];
                if (bad) status |= ST_NONFINITE;
                if (PH::nonpositive(Wn)) status |= ST_NONPOSITIVE;
                float r = PH::rate_x(Wn, p.sigma_lim, p.k_ws) * v.idx;
                if (!(r >= 0.0f)) r = __int_as_float(0x7f800000);      // NaN -> inf
                rmax = fmaxf(rmax, r);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) Wout[(long long)k * n + i] = Wn[k];
        }
        __syncthreads();
    }
    return rmax;
}

// Team-wide max of the CFL rate and OR of the status bits, combined in one
// of three slots in CTA 0 (slot = epoch mod 3).  After the barrier of epoch
// e, CTA 0 clears slot (e+2) mod 3: every CTA read it (epoch e-1) before
// arriving at barrier e, and none writes it (epoch e+2) before barrier e+1,
// which CTA 0 reaches only after the clear.
template <int NT>
__device__ __forceinline__ void team_reduce(float r, unsigned st, unsigned& epoch,
                                            unsigned r_red, unsigned r_stat, unsigned rank,
                                            unsigned* s_red, unsigned* s_stat, float* wred,
                                            unsigned* wst, float* s_m, unsigned* s_st, float& m,
                                            unsigned& st_out) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    st = __reduce_or_sync(0xffffffffu, st);
    if (lane == 0) {
        wred[wid] = r;
        wst[wid] = st;
    }
    __syncthreads();
    const unsigned par = epoch % 3u;
    if (tid == 0) {
        float rb = wred[0];
        unsigned sb = wst[0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w) {
            rb = fmaxf(rb, wred[w]);
            sb |= wst[w];
        }
        cl_red_max(r_red + 4u * par, __float_as_uint(rb));
        if (sb) cl_red_or(r_stat + 4u * par, sb);
    }
    cl_sync();
    if (tid == 0) {
        *s_m = __uint_as_float(cl_ld(r_red + 4u * par));
        *s_st = cl_ld(r_stat + 4u * par);
        if (rank == 0) {
            s_red[(par + 2u) % 3u] = 0u;
            s_stat[(par + 2u) % 3u] = 0u;
        }
    }
    __syncthreads();
    m = *s_m;
    st_out = *s_st;
    ++epoch;
}

template <class PH, int NT>
__device__ void tubes_mixed_body(const TubeMixedArgs& a, const ParamsT<float>& p0,
                                 const MixedPolicy& mp) {
    constexpr int NF = PH::NF;
    using LY = TubeLayout<NF, NT>;
    constexpr int C = LY::C;
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned s_red[3], s_stat[3], s_st, s_cnt;
    __shared__ int s_tube;
    __shared__ float s_m;
    const unsigned rank = cl_rank(), team = cl_size();
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_red[0] = s_red[1] = s_red[2] = 0u;
        s_stat[0] = s_stat[1] = s_stat[2] = 0u;
    }
    const unsigned r_red = cl_map(s_red, 0), r_stat = cl_map(s_stat, 0);
    const unsigned r_tube = cl_map(&s_tube, 0);
    float* wred = sm + LY::R_OFF;
    unsigned* wst = (unsigned*)(sm + LY::S_OFF);
    unsigned epoch = 0;
    for (;;) {
        if (rank == 0 && tid == 0) s_tube = atomicAdd(a.queue, 1);
        if (tid == 0) s_cnt = 0u;
        cl_sync();
        const int q = (int)cl_ld(r_tube);
        if (q >= a.ntubes) {
            cl_sync();               // CTA 0 stays until every CTA has read s_tube
            return;
        }
        const int b = a.order[q];
        const TubeDesc td = a.tubes[b];
        TubeView v;
        v.n = td.n;
        v.U = a.U + td.off;
        v.W = a.W + (long long)NF * td.coff;
        v.Ws = a.Ws + (long long)NF * td.coff;
        v.idx = (float)(1.0 / td.dx);
        v.p = p0;
        v.p.tau_model = td.rp.model;
        v.p.tau_ref = (float)td.rp.tau_ref;
        v.p.rho_ref = (float)td.rp.rho_ref;
        v.p.T_ref = (float)td.rp.T_ref;
        v.p.src_implicit = td.rp.implicit;
        TubeClock* ck = a.clk + b;
        const int n = v.n;

        // W = prim(U) in FP64, and the CFL rate of the current state
        float r = 0.0f;
        for (int c0 = (int)rank * C; c0 < n; c0 += (int)team * C) {
            const int i = c0 + tid;
            if (tid < C && i < n) {
                double Uc[NF], Q[NF];
#pragma unroll
                for (int k = 0; k < NF; ++k) Uc[k] = v.U[(long long)PH::ufield(k) * n + i];
                PH::cons2prim_fast(Uc, Q);
                float Qf[NF];
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    Qf[k] = (float)Q[k];
                    v.W[(long long)k * n + i] = Qf[k];
                }
                float ri = PH::rate_x(Qf, v.p.sigma_lim, v.p.k_ws) * v.idx;
                if (!(ri >= 0.0f)) ri = __int_as_float(0x7f800000);
                r = fmaxf(r, ri);
            }
        }
        float m;
        unsigned bst;
        team_reduce<NT>(r, 0u, epoch, r_red, r_stat, rank, s_red, s_stat, wred, wst, &s_m, &s_st,
                        m, bst);
        double t = ck->t;
        long long steps = ck->steps;
        double last_dt = ck->last_dt;
        unsigned nflag = 0, nface = 0;
        float* Wc = v.W;
        float* Wn = v.Ws;
        bst = 0u;
        for (int s = 0; s < a.max_steps; ++s) {
            double dt;
            if (a.dt_fixed) {
                if (s >= a.n_fixed) break;
                dt = a.dt_fixed[s];
            } else {
                if (!(t < a.t_end)) break;
                dt = a.cfl / (double)m;
                if (t + dt > a.t_end) dt = a.t_end - t;
            }
            if (!(dt > 0.0)) break;
            const bool rs = ((steps + 1) % a.resync_every) == 0;
            unsigned status = 0;
            float rr;
            if (a.integrator == 1) {
                tube_stage_m<PH, NT>(a, v, mp, Wc, nullptr, Wn, (float)(0.5 * dt), false, false,
                                     rank, team, sm, status, nflag);
                cl_sync();
                rr = tube_stage_m<PH, NT>(a, v, mp, Wn, Wc, Wc, (float)dt, true, rs, rank, team,
                                          sm, status, nflag);
                nface += 2u;
            } else {
                rr = tube_stage_m<PH, NT>(a, v, mp, Wc, nullptr, Wn, (float)dt, true, rs, rank,
                                          team, sm, status, nflag);
                float* tmp = Wc;
                Wc = Wn;
                Wn = tmp;
                nface += 1u;
            }
            team_reduce<NT>(rr, status, epoch, r_red, r_stat, rank, s_red, s_stat, wred, wst,
                            &s_m, &s_st, m, bst);
            t += dt;
            last_dt = dt;
            ++steps;
            if (bst) break;          // team-uniform
        }
        // face-state closures: 2 per face, C + 1 faces per chunk and stage
        unsigned wf = __reduce_add_sync(0xffffffffu, nflag);
        if ((tid & 31) == 0 && wf) atomicAdd(&s_cnt, wf);
        __syncthreads();
        if (tid == 0) {
            unsigned nch = 0;
            for (int c0 = (int)rank * C; c0 < n; c0 += (int)team * C) ++nch;
            atomicAdd(&ck->n_face, (unsigned long long)nface * nch * 2ull * (C + 1));
            if (s_cnt) atomicAdd(&ck->n_face64, (unsigned long long)s_cnt);
            if (rank == 0) {
                ck->t = t;
                ck->steps = steps;
                ck->last_dt = last_dt;
                ck->rate = (double)m;
                if (bst) atomicOr(&ck->status, bst);
            }
        }
    }
}

#define MXE_TUBES_MIXED(NAME, PH, NT, MINB)                                                  \
    extern "C" __global__ void __launch_bounds__(NT, MINB)                                   \
        NAME(const TubeMixedArgs a, const ParamsT<float> p, const MixedPolicy mp) {          \
        tubes_mixed_body<PH, NT>(a, p, mp);                                                  \
    }
MXE_TUBES_MIXED(mxe_tubes14_mixed_128, PhysGeneral, 128, 4)
MXE_TUBES_MIXED(mxe_tubes14_mixed_256, PhysGeneral, 256, 2)
MXE_TUBES_MIXED(mxe_tubes14_mixed_planar_128, PhysPlanar, 128, 4)
MXE_TUBES_MIXED(mxe_tubes14_mixed_planar_256, PhysPlanar, 256, 2)
#undef MXE_TUBES_MIXED

// CFL rate max_cells |lambda|_max / dx of every tube's current state (one
// block per tube; the same FP64 primitive recovery and FP32 wave speeds as
// the march), for the host's estimate of each tube's step count when it
// divides the tubes between the team and fill launches.
template <class PH>
__device__ void tube_rates_body(const double* U, const TubeDesc* tubes, float sl, float kw,
                                float* rates) {
    constexpr int NF = PH::NF;
    const TubeDesc td = tubes[blockIdx.x];
    const double* Ut = U + td.off;
    const float idx = (float)(1.0 / td.dx);
    float r = 0.0f;
    for (int i = threadIdx.x; i < td.n; i += blockDim.x) {
        double Uc[NF], Q[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Uc[k] = Ut[(long long)PH::ufield(k) * td.n + i];
        PH::cons2prim_fast(Uc, Q);
        float Qf[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Qf[k] = (float)Q[k];
        float ri = PH::rate_x(Qf, sl, kw) * idx;
        if (!(ri >= 0.0f)) ri = __int_as_float(0x7f800000);
        r = fmaxf(r, ri);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    __shared__ float wr[32];
    if ((threadIdx.x & 31) == 0) wr[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, wr[w]);
        rates[blockIdx.x] = r;
    }
}
extern "C" __global__ void __launch_bounds__(256) mxe_tube_rates14(const double* U,
                                                                  const TubeDesc* tubes, float sl,
                                                                  float kw, float* rates) {
    tube_rates_body<PhysGeneral>(U, tubes, sl, kw, rates);
}
extern "C" __global__ void __launch_bounds__(256) mxe_tube_rates14_planar(const double* U,
                                                                         const TubeDesc* tubes,
                                                                         float sl, float kw,
                                                                         float* rates) {
    tube_rates_body<PhysPlanar>(U, tubes, sl, kw, rates);
}

void tube_rates(bool planar, const double* U, const TubeDesc* tubes, int ntubes, float sl,
                float kw, float* rates, cudaStream_t st) {
    if (planar) mxe_tube_rates14_planar<<<ntubes, 256, 0, st>>>(U, tubes, sl, kw, rates);
    else mxe_tube_rates14<<<ntubes, 256, 0, st>>>(U, tubes, sl, kw, rates);
}

// Kernel and dynamic shared memory of one block shape (nt = 128 or 256).
const void* tubes_mixed_kernel(bool planar, int nt) {
    if (planar) return nt == 256 ? (const void*)mxe_tubes14_mixed_planar_256
                                 : (const void*)mxe_tubes14_mixed_planar_128;
    return nt == 256 ? (const void*)mxe_tubes14_mixed_256 : (const void*)mxe_tubes14_mixed_128;
}
size_t tubes_mixed_smem(bool planar, int nt) {
    if (planar) return nt == 256 ? TubeLayout<NP, 256>::bytes() : TubeLayout<NP, 128>::bytes();
    return nt == 256 ? TubeLayout<14, 256>::bytes() : TubeLayout<14, 128>::bytes();
}

}  // namespace mxe
