// mxe_grid2d.cu -- fused finite-volume stage for the 14-moment system on a
// 2D Cartesian grid (Sec. 3 of Boccelli et al., JCP 2024), FP64 path.
//
// One thread block owns a tile of TX x TY = 15 x 16 cells.  It stages the
// primitive moments of the tile plus a 2-cell halo in shared memory (BCs are
// applied while loading: transmissive, periodic, Dirichlet slots), computes
// one shared limiter per cell and direction, evaluates every x- and y-face
// once (two face states, closure, flux, wave speeds, HLL/Rusanov) with one
// thread per face, differences the face fluxes, adds the BGK source and
// writes the RK stage.  The final stage of a step also reduces the CFL rate
// of the new state (warp shuffle, block, one atomicMax per block) so that
// the next step's dt is formed on the device.
//
// Tile shape: 16 x 16 x-faces and 15 x 17 y-faces map onto 256 threads with
// at most one idle thread.  The kernel is instantiated for the general
// 14-moment state and for planar states (ten active moments).
#include "mxe_internal.h"
#include "mxe_policy.cuh"

namespace mxe {

constexpr int TX = 15, TY = 16, NT2 = 256;
constexpr int BX = TX + 4, BY = TY + 4;          // 19 x 20 staged box
constexpr int NBOX = BX * BY;
constexpr int NPHX = (TX + 2) * TY;              // 272 x-limiters (box cols 1..17)
constexpr int NPHY = TX * (TY + 2);              // 270 y-limiters (box rows 1..18)

// time step of this step (identical in every thread of every block)
__device__ __forceinline__ double step_dt(const DevClock* clk, int slot, double cfl,
                                          double t_end, double dt_fixed, double& t) {
    t = clk->t[slot];
    if (dt_fixed > 0.0) return dt_fixed;
    double m = __longlong_as_double((long long)clk->rate[slot]);
    double dt = cfl / m;
    if (t + dt > t_end) dt = t_end - t;
    return dt;
}

// Boundary logic: returns the ghost state of a Dirichlet ghost cell
// (nullptr otherwise) and maps (gi, gj) into the grid (periodic wrap,
// transmissive clamp).
__device__ __forceinline__ const double* map_cell(const Grid2D& g, int& gi, int& gj) {
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
    } else if (!xin && !yin) {          // corner: never used by the stencil
        gi = gi < 0 ? 0 : g.nx - 1;
        gj = gj < 0 ? 0 : g.ny - 1;
    }
    return nullptr;
}

template <class PH>
__device__ __forceinline__ void load_prim_f64(const Stage2DArgs& a, int gi, int gj, double* Q) {
    const Grid2D& g = a.g;
    const double* gs = map_cell(g, gi, gj);
    if (gs) {
#pragma unroll
        for (int k = 0; k < PH::NF; ++k) Q[k] = gs[PH::ufield(k)];
        return;
    }
    const double* p = a.Uin + (long long)gj * g.pitch + gi;
    double U[PH::NF];
#pragma unroll
    for (int k = 0; k < PH::NF; ++k) U[k] = __ldg(p + PH::ufield(k) * g.fstride);
    PH::cons2prim_rn(U, Q);
}

// Numerical face flux from two face states (HLL with Davis speeds, or
// Rusanov), Sec. 3.1.
template <class PH, int K>
__device__ __forceinline__ void riemann_f64(const double* QL, const double* QR,
                                            const ParamsT<double>& p, double* Fo) {
    constexpr int NF = PH::NF;
    double UL[NF], FL[NF], lminL, lmaxL;
    PH::template face<double, K>(QL, p.sigma_lim, p.k_ws, UL, FL, lminL, lmaxL);
    double UR[NF], FR[NF], lminR, lmaxR;
    PH::template face<double, K>(QR, p.sigma_lim, p.k_ws, UR, FR, lminR, lmaxR);
    if (p.flux == 1) {
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
        double inv = 1.0 / (SR - SL);
        double SLR = SL * SR;
#pragma unroll
        for (int k = 0; k < NF; ++k) Fo[k] = (SR * FL[k] - SL * FR[k] + SLR * (UR[k] - UL[k])) * inv;
    }
}

template <int NF>
__device__ __forceinline__ double phi_box(const double* W, int c, int stride, int lim) {
    double phi = 1.0;
    const FlatRef<double> fr = flat_ref<NF>(W + c, NBOX);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const double* w = W + k * NBOX + c;
        phi_accumulate<NF>(phi, w[0] - w[-stride], w[stride] - w[0], lim, fr, k);
    }
    return phi;
}

template <int NF>
__device__ __forceinline__ void face_state_box(const double* W, int c, int stride, double phi,
                                               double sgn, double* Qf) {
    double hs = mul_rn(sgn, 0.5);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const double* w = W + k * NBOX + c;
        Qf[k] = muscl_face(w[-stride], w[0], w[stride], phi, hs);
    }
}

__device__ __forceinline__ void block_max_atomic(double r, unsigned long long* dst, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double v = __shfl_xor_sync(0xffffffffu, r, o);
        r = v > r ? v : r;
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = r;
    __syncthreads();
    if (wid == 0) {
        r = lane < (NT2 / 32) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            double v = __shfl_xor_sync(0xffffffffu, r, o);
            r = v > r ? v : r;
        }
        if (lane == 0) atomicMax(dst, (unsigned long long)__double_as_longlong(r));
    }
}

// Clock bookkeeping of the final stage (block (0,0), thread 0).
__device__ __forceinline__ void advance_clock(const Stage2DArgs& a, double dt, double t) {
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

template <int NF>
constexpr size_t smem_f64() {
    return sizeof(double) * (NF * NBOX + NF * NT2 + NPHX + NPHY + 8);
}

// ---------------------------------------------------------------------------
// FP64 stage kernel.  Stage 1 of RK2: Uout = Ubase + dt/2 L(Uin);
// final stage (RK2 stage 2 or FE): Uout = Ubase + dt L(Uin), plus the CFL
// rate of Uout, clock advance and status.
// ---------------------------------------------------------------------------
template <class PH>
__device__ __forceinline__ void stage_f64(const Stage2DArgs& a) {
    constexpr int NF = PH::NF;
    extern __shared__ __align__(16) double smem[];
    double* W = smem;                                // [NF][BY][BX]
    double* Fb = W + NF * NBOX;                      // [NF][256]
    double* phx = Fb + NF * NT2;                     // [TY][TX+2]
    double* phy = phx + NPHX;                        // [TY+2][TX]
    double* red = phy + NPHY;                        // [8]
    __shared__ double sdt[2];

    const int tid = threadIdx.x;
    if (tid == 0) {
        double tt;
        sdt[0] = step_dt(a.clk, a.slot, a.cfl, a.t_end, a.dt_fixed, tt);
        sdt[1] = tt;
    }
    __syncthreads();
    const double dt = sdt[0], t = sdt[1];
    if (a.final_stage && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) advance_clock(a, dt, t);
    if (!(dt > 0.0)) return;

    const ParamsT<double> p = make_params<double>(a.sp, a.rp);
    const Grid2D& g = a.g;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    for (int c = tid; c < NBOX; c += NT2) {
        int bx = c % BX, by = c / BX;
        double Q[NF];
        load_prim_f64<PH>(a, i0 + bx - 2, j0 + by - 2, Q);
#pragma unroll
        for (int k = 0; k < NF; ++k) W[k * NBOX + c] = Q[k];
    }
    __syncthreads();
    for (int n = tid; n < NPHX; n += NT2) {
        int bx = 1 + n % (TX + 2), by = 2 + n / (TX + 2);
        phx[n] = p.order == 2 ? phi_box<NF>(W, by * BX + bx, 1, p.limiter) : 0.0;
    }
    for (int n = tid; n < NPHY; n += NT2) {
        int bx = 2 + n % TX, by = 1 + n / TX;
        phy[n] = p.order == 2 ? phi_box<NF>(W, by * BX + bx, BX, p.limiter) : 0.0;
    }
    __syncthreads();
    {   // x faces: face fx in [0,16) of row cy, between box cells fx+1 | fx+2
        int fx = tid & 15, cy = tid >> 4, by = cy + 2;
        double QL[NF], QR[NF], F[NF];
        face_state_box<NF>(W, by * BX + fx + 1, 1, phx[cy * (TX + 2) + fx], 1.0, QL);
        face_state_box<NF>(W, by * BX + fx + 2, 1, phx[cy * (TX + 2) + fx + 1], -1.0, QR);
        riemann_f64<PH, 0>(QL, QR, p, F);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fb[k * NT2 + tid] = F[k];
    }
    __syncthreads();
    const int cx = tid % TX, cy = tid / TX;          // owned cell (tid < 240)
    const bool owner = tid < TX * TY;
    double L[NF];
    if (owner) {
        double Qc[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) Qc[k] = W[k * NBOX + (cy + 2) * BX + cx + 2];
        if (p.tau_model != 0 && !p.src_implicit) {
            PH::source(Qc, PH::tau(p, Qc), L);
        } else {
#pragma unroll
            for (int k = 0; k < NF; ++k) L[k] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < NF; ++k)
            L[k] -= (Fb[k * NT2 + cy * 16 + cx + 1] - Fb[k * NT2 + cy * 16 + cx]) * g.idx;
    }
    __syncthreads();
    if (tid < TX * (TY + 1)) {   // y faces: face fy in [0,17) of column cx
        int fcx = tid % TX, fy = tid / TX, bx = fcx + 2;
        double QL[NF], QR[NF], F[NF];
        face_state_box<NF>(W, (fy + 1) * BX + bx, BX, phy[fy * TX + fcx], 1.0, QL);
        face_state_box<NF>(W, (fy + 2) * BX + bx, BX, phy[(fy + 1) * TX + fcx], -1.0, QR);
        riemann_f64<PH, 1>(QL, QR, p, F);
#pragma unroll
        for (int k = 0; k < NF; ++k) Fb[k * NT2 + tid] = F[k];
    }
    __syncthreads();

    double r = 0.0;
    if (owner) {
#pragma unroll
        for (int k = 0; k < NF; ++k)
            L[k] -= (Fb[k * NT2 + (cy + 1) * TX + cx] - Fb[k * NT2 + cy * TX + cx]) * g.idy;
        int gi = i0 + cx, gj = j0 + cy;
        if (gi < g.nx && gj < g.ny) {
            long long o = (long long)gj * g.pitch + gi;
            double Un[NF];
            bool bad = false;
            double cdt = mul_rn(a.coef, dt);
#pragma unroll
            for (int k = 0; k < NF; ++k)
                Un[k] = add_rn(a.Ubase[o + PH::ufield(k) * g.fstride], mul_rn(cdt, L[k]));
            if (p.tau_model != 0 && p.src_implicit) {   // point-implicit source over cdt
                double Qv[NF];
                PH::cons2prim_rn(Un, Qv);
                PH::relax_cons(Un, Qv, PH::tau(p, Qv), cdt);
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                a.Uout[o + PH::ufield(k) * g.fstride] = Un[k];
                bad |= !isfinite(Un[k]);
            }
            if (a.final_stage) {
                double Qn[NF];
                PH::cons2prim_rn(Un, Qn);
                if (PH::nonpositive(Qn)) atomicOr(&a.clk->status, ST_NONPOSITIVE);
                if (bad) atomicOr(&a.clk->status, ST_NONFINITE);
                if (!a.skip_rate) {
                    double ax, ay;
                    PH::rates(Qn, p.sigma_lim, p.k_ws, ax, ay);
                    r = ax * g.idx;
                    r = r + ay * g.idy;
                    if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);  // NaN -> inf
                }
            }
        }
    }
    if (a.final_stage) block_max_atomic(r, &a.clk->rate[(a.slot + 1) % 3], red);
}

extern "C" __global__ void __launch_bounds__(NT2, 1) mxe_stage14_2d_f64(const Stage2DArgs a) {
    stage_f64<PhysGeneral>(a);
}
extern "C" __global__ void __launch_bounds__(NT2, 1)
mxe_stage14_2d_f64_planar(const Stage2DArgs a) {
    stage_f64<PhysPlanar>(a);
}

size_t stage14_2d_f64_smem(bool planar) {
    return planar ? smem_f64<NP>() : smem_f64<14>();
}

// Initial CFL rate of the current state into slot `slot` of the clock.
template <class PH>
__device__ __forceinline__ void rate_f64(const double* U, const Grid2D& g, const SchemeParams& sp,
                                         DevClock* clk, int slot) {
    __shared__ double red[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    double r = 0.0;
    if (i < g.nx) {
        long long o = (long long)j * g.pitch + i;
        double Un[PH::NF], Qn[PH::NF];
#pragma unroll
        for (int k = 0; k < PH::NF; ++k) Un[k] = U[o + PH::ufield(k) * g.fstride];
        PH::cons2prim_rn(Un, Qn);
        double ax, ay;
        PH::rates(Qn, sp.sigma_lim, sp.k_ws, ax, ay);
        r = ax * g.idx;
        r = r + ay * g.idy;
        if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);
    }
    block_max_atomic(r, &clk->rate[slot], red);
}
extern "C" __global__ void mxe_rate14_2d(const double* U, Grid2D g, SchemeParams sp,
                                         DevClock* clk, int slot) {
    rate_f64<PhysGeneral>(U, g, sp, clk, slot);
}
extern "C" __global__ void mxe_rate14_2d_planar(const double* U, Grid2D g, SchemeParams sp,
                                                DevClock* clk, int slot) {
    rate_f64<PhysPlanar>(U, g, sp, clk, slot);
}

int tile_x() { return TX; }
int tile_y() { return TY; }

}  // namespace mxe
