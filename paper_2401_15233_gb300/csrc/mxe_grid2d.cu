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
// at most one idle thread.
#include "mxe_internal.h"

namespace mxe {

constexpr int TX = 15, TY = 16, NT2 = 256;
constexpr int BX = TX + 4, BY = TY + 4;          // 19 x 20 staged box
constexpr int NPHX = (TX + 2) * TY;              // 272 x-limiters (box cols 1..17)
constexpr int NPHY = TX * (TY + 2);              // 270 y-limiters (box rows 1..18)

__device__ __forceinline__ double rate_bits_to_double(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// time step of this step (identical in every thread of every block)
__device__ __forceinline__ double step_dt(const DevClock* clk, int slot, double cfl,
                                          double t_end, double dt_fixed, double& t) {
    t = clk->t[slot];
    if (dt_fixed > 0.0) return dt_fixed;
    double m = rate_bits_to_double(clk->rate[slot]);
    double dt = cfl / m;
    if (t + dt > t_end) dt = t_end - t;
    return dt;
}

// Primitive state of (possibly ghost) cell (gi, gj), FP64 conserved input.
__device__ __forceinline__ void load_prim_f64(const Stage2DArgs& a, int gi, int gj,
                                              double* Q) {
    const Grid2D& g = a.g;
    bool xin = (gi >= 0 && gi < g.nx), yin = (gj >= 0 && gj < g.ny);
    if (!xin && yin) {
        int s = gi < 0 ? 0 : 1;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gi = ((gi % g.nx) + g.nx) % g.nx;
        } else {
            for (int n = 0; n < sd.nspans; ++n)
                if (gj >= sd.lo[n] && gj <= sd.hi[n]) {
                    const double* gs = g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
#pragma unroll
                    for (int k = 0; k < 14; ++k) Q[k] = gs[k];
                    return;
                }
            if (sd.type == 2) {
                const double* gs = g.ghost + (s * GHOST_SLOTS) * 14;
#pragma unroll
                for (int k = 0; k < 14; ++k) Q[k] = gs[k];
                return;
            }
            gi = gi < 0 ? 0 : g.nx - 1;
        }
    } else if (xin && !yin) {
        int s = gj < 0 ? 2 : 3;
        const SideDesc& sd = g.side[s];
        if (sd.type == 1) {
            gj = ((gj % g.ny) + g.ny) % g.ny;
        } else {
            for (int n = 0; n < sd.nspans; ++n)
                if (gi >= sd.lo[n] && gi <= sd.hi[n]) {
                    const double* gs = g.ghost + (s * GHOST_SLOTS + 1 + n) * 14;
#pragma unroll
                    for (int k = 0; k < 14; ++k) Q[k] = gs[k];
                    return;
                }
            if (sd.type == 2) {
                const double* gs = g.ghost + (s * GHOST_SLOTS) * 14;
#pragma unroll
                for (int k = 0; k < 14; ++k) Q[k] = gs[k];
                return;
            }
            gj = gj < 0 ? 0 : g.ny - 1;
        }
    } else if (!xin && !yin) {          // corner: never used by the stencil
        gi = gi < 0 ? 0 : g.nx - 1;
        gj = gj < 0 ? 0 : g.ny - 1;
    }
    const double* p = a.Uin + (long long)gj * g.pitch + gi;
    double U[14];
#pragma unroll
    for (int k = 0; k < 14; ++k) U[k] = __ldg(p + k * g.fstride);
    cons2prim14_rn(U, Q);
}

// Numerical face flux from two face states (HLL with Davis speeds, or
// Rusanov), Sec. 3.1.
template <class T, int K>
__device__ __forceinline__ void riemann14(const T* QL, const T* QR, const SchemeParams& sp,
                                          T* Fo) {
    T UL[14], FL[14], lminL, lmaxL;
    face_eval14<T, K>(QL, sp, UL, FL, lminL, lmaxL);
    T UR[14], FR[14], lminR, lmaxR;
    face_eval14<T, K>(QR, sp, UR, FR, lminR, lmaxR);
    if (sp.flux == 1) {
        T s = fabs(lminL);
        s = fabs(lmaxL) > s ? fabs(lmaxL) : s;
        s = fabs(lminR) > s ? fabs(lminR) : s;
        s = fabs(lmaxR) > s ? fabs(lmaxR) : s;
#pragma unroll
        for (int k = 0; k < 14; ++k) Fo[k] = T(0.5) * (FL[k] + FR[k]) - T(0.5) * s * (UR[k] - UL[k]);
        return;
    }
    T SL = lminL < lminR ? lminL : lminR;
    T SR = lmaxL > lmaxR ? lmaxL : lmaxR;
    if (SL >= T(0)) {
#pragma unroll
        for (int k = 0; k < 14; ++k) Fo[k] = FL[k];
    } else if (SR <= T(0)) {
#pragma unroll
        for (int k = 0; k < 14; ++k) Fo[k] = FR[k];
    } else {
        T inv = T(1) / (SR - SL);
        T SLR = SL * SR;
#pragma unroll
        for (int k = 0; k < 14; ++k)
            Fo[k] = (SR * FL[k] - SL * FR[k] + SLR * (UR[k] - UL[k])) * inv;
    }
}

// shared limiter of a box cell along a stride (1: x, BX: y) in smem W[14][BY*BX]
template <class T>
__device__ __forceinline__ T shared_phi_box(const T* W, int c, int stride, int lim) {
    T phi = T(1);
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const T* w = W + k * BX * BY + c;
        T dm = w[0] - w[-stride], dp = w[stride] - w[0];
        T pk = phi_field(dm, dp, lim);
        phi = pk < phi ? pk : phi;
    }
    return phi;
}

template <class T>
__device__ __forceinline__ void face_state_box(const T* W, int c, int stride, T phi, T sgn,
                                               T* Qf) {
    T hs = mul_rn(sgn, T(0.5));
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        const T* w = W + k * BX * BY + c;
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

// ---------------------------------------------------------------------------
// FP64 stage kernel.  Stage 1 of RK2: Uout = Ubase + dt/2 L(Uin);
// final stage (RK2 stage 2 or FE): Uout = Ubase + dt L(Uin), plus the CFL
// rate of Uout, clock advance and status.
// ---------------------------------------------------------------------------
extern "C" __global__ void __launch_bounds__(NT2, 1)
mxe_stage14_2d_f64(const Stage2DArgs a) {
    extern __shared__ __align__(16) double smem[];
    double* W = smem;                                // [14][BY][BX]
    double* Fb = W + 14 * BX * BY;                   // [14][256]
    double* phx = Fb + 14 * NT2;                     // [TY][TX+2]
    double* phy = phx + NPHX;                        // [TY+2][TX]
    double* red = phy + NPHY;                        // [8]

    const int tid = threadIdx.x;
    __shared__ double sdt[2];
    if (tid == 0) {
        double tt;
        sdt[0] = step_dt(a.clk, a.slot, a.cfl, a.t_end, a.dt_fixed, tt);
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

    const Grid2D& g = a.g;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;

    for (int c = tid; c < BX * BY; c += NT2) {
        int bx = c % BX, by = c / BX;
        double Q[14];
        load_prim_f64(a, i0 + bx - 2, j0 + by - 2, Q);
#pragma unroll
        for (int k = 0; k < 14; ++k) W[k * BX * BY + c] = Q[k];
    }
    __syncthreads();

    const int order = a.sp.order, lim = a.sp.limiter;
    for (int n = tid; n < NPHX; n += NT2) {
        int bx = 1 + n % (TX + 2), by = 2 + n / (TX + 2);
        phx[n] = order == 2 ? shared_phi_box(W, by * BX + bx, 1, lim) : 0.0;
    }
    for (int n = tid; n < NPHY; n += NT2) {
        int bx = 2 + n % TX, by = 1 + n / TX;
        phy[n] = order == 2 ? shared_phi_box(W, by * BX + bx, BX, lim) : 0.0;
    }
    __syncthreads();

    // ---- x faces: face fx in [0,16) of row cy, between box cells fx+1 | fx+2
    {
        int fx = tid & 15, cy = tid >> 4;
        int by = cy + 2;
        double QL[14], QR[14], F[14];
        face_state_box(W, by * BX + fx + 1, 1, phx[cy * (TX + 2) + fx], 1.0, QL);
        face_state_box(W, by * BX + fx + 2, 1, phx[cy * (TX + 2) + fx + 1], -1.0, QR);
        riemann14<double, 0>(QL, QR, a.sp, F);
#pragma unroll
        for (int k = 0; k < 14; ++k) Fb[k * NT2 + tid] = F[k];
    }
    __syncthreads();
    const int cx = tid % TX, cy = tid / TX;          // owned cell (tid < 240)
    const bool owner = tid < TX * TY;
    double L[14];
    if (owner) {
        double Qc[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) Qc[k] = W[k * BX * BY + (cy + 2) * BX + cx + 2];
        if (a.rp.model != 0) {
            double tau = tau_of<double>(a.rp, Qc, 14);
            source14(Qc, tau, L);
        } else {
#pragma unroll
            for (int k = 0; k < 14; ++k) L[k] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < 14; ++k)
            L[k] -= (Fb[k * NT2 + cy * 16 + cx + 1] - Fb[k * NT2 + cy * 16 + cx]) * g.idx;
    }
    __syncthreads();
    // ---- y faces: face fy in [0,17) of column cx, between box rows fy+1 | fy+2
    if (tid < TX * (TY + 1)) {
        int fcx = tid % TX, fy = tid / TX;
        int bx = fcx + 2;
        double QL[14], QR[14], F[14];
        face_state_box(W, (fy + 1) * BX + bx, BX, phy[fy * TX + fcx], 1.0, QL);
        face_state_box(W, (fy + 2) * BX + bx, BX, phy[(fy + 1) * TX + fcx], -1.0, QR);
        riemann14<double, 1>(QL, QR, a.sp, F);
#pragma unroll
        for (int k = 0; k < 14; ++k) Fb[k * NT2 + tid] = F[k];
    }
    __syncthreads();

    double r = 0.0;
    if (owner) {
#pragma unroll
        for (int k = 0; k < 14; ++k)
            L[k] -= (Fb[k * NT2 + (cy + 1) * TX + cx] - Fb[k * NT2 + cy * TX + cx]) * g.idy;
        int gi = i0 + cx, gj = j0 + cy;
        if (gi < g.nx && gj < g.ny) {
            long long o = (long long)gj * g.pitch + gi;
            double Un[14];
            bool bad = false;
#pragma unroll
            double cdt = mul_rn(a.coef, dt);
#pragma unroll
            for (int k = 0; k < 14; ++k) {
                Un[k] = add_rn(a.Ubase[o + k * g.fstride], mul_rn(cdt, L[k]));
                a.Uout[o + k * g.fstride] = Un[k];
                bad |= !isfinite(Un[k]);
            }
            if (a.final_stage) {
                double Qn[14];
                cons2prim14_rn(Un, Qn);
                if (Qn[0] <= 0.0 || Qn[4] <= 0.0 || Qn[7] <= 0.0 || Qn[9] <= 0.0)
                    atomicOr(&a.clk->status, ST_NONPOSITIVE);
                if (bad) atomicOr(&a.clk->status, ST_NONFINITE);
                Dimless14<double> d;
                dimless14(Qn, d);
                double ax = amax14<double, 0>(Qn, d, a.sp);
                double ay = amax14<double, 1>(Qn, d, a.sp);
                r = ax * g.idx;
                r = r + ay * g.idy;
                if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);  // NaN -> inf
            }
        }
    }
    if (a.final_stage) block_max_atomic(r, &a.clk->rate[(a.slot + 1) % 3], red);
}

size_t stage14_2d_f64_smem() {
    return sizeof(double) * (14 * BX * BY + 14 * NT2 + NPHX + NPHY + 8);
}

// Initial CFL rate of the current state into slot 0 of the clock (t = 0).
extern "C" __global__ void mxe_rate14_2d(const double* U, Grid2D g, SchemeParams sp,
                                         DevClock* clk, int slot) {
    __shared__ double red[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    double r = 0.0;
    if (i < g.nx) {
        long long o = (long long)j * g.pitch + i;
        double Un[14], Qn[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) Un[k] = U[o + k * g.fstride];
        cons2prim14_rn(Un, Qn);
        Dimless14<double> d;
        dimless14(Qn, d);
        double ax = amax14<double, 0>(Qn, d, sp);
        double ay = g.ny > 1 ? amax14<double, 1>(Qn, d, sp) : 0.0;
        r = ax / g.dx;
        if (g.ny > 1) r = r + ay / g.dy;
        if (!(r >= 0.0)) r = __longlong_as_double(0x7ff0000000000000ll);
    }
    block_max_atomic(r, &clk->rate[slot], red);
}

int tile_x() { return TX; }
int tile_y() { return TY; }

}  // namespace mxe
