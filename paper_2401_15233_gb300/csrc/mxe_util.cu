// mxe_util.cu -- set-up and read-back kernels: primitive <-> conserved
// conversion, state validation, ghost-state round trip, diagnostics.
// Nothing here is on the time-stepping path.
#include "mxe_internal.h"

namespace mxe {

// Returns false if the thread has no cell.  dense: offset of field 0 in the
// API's dense array; dev: offset in the device array; fs/dfs: field strides.
__device__ __forceinline__ bool cell_of(const CellMap& m, long long& dense, long long& dfs,
                                        long long& dev, long long& fs, long long& idx) {
    if (m.mode == 0) {
        int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
        if (i >= m.nx || j >= m.ny) return false;
        idx = (long long)j * m.nx + i;
        dense = idx;
        dfs = (long long)m.nx * m.ny;
        dev = (long long)j * m.pitch + i;
        fs = m.fstride;
        return true;
    }
    int b = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m.ntubes || i >= m.tubes[b].n) return false;
    dense = dev = m.tubes[b].off + i;
    dfs = fs = m.tubes[b].n;
    idx = m.tubes[b].off / m.nf + i;     // cell number in the concatenation
    return true;
}

__device__ __forceinline__ double raw_sigma(const double* Q, int nf) {
    if (nf == 5) {
        double th = Q[2] / Q[0];
        double qs = Q[3] / (Q[0] * th * sqrt(th));
        double rs = Q[4] / (Q[0] * th * th);
        return sigma5(qs, rs);
    }
    Dimless14<double> d;
    dimless14(Q, d);
    return d.sig;
}

// sigma <= 1 (with 1e-9 of slack): decided in FP32 where FP32 clearly can
// (sigma_32 <= 0.99 with every |Q| in [1e-30, 1e30] and det P* >= 1e-3, so
// that the FP32 error of sigma is orders of magnitude below the 1e-2
// margin), in FP64 otherwise.  FP64 here runs at 1/64 of the FP32 rate.
__device__ __forceinline__ bool sigma_within_one(const double* Q, int nf) {
    bool screen = true;
    float Qf[14];
    for (int k = 0; k < nf; ++k) {
        double a = fabs(Q[k]);
        screen &= (a == 0.0) || (a >= 1e-30 && a <= 1e30);
        Qf[k] = (float)Q[k];
    }
    if (screen) {
        float s32;
        bool cond = true;
        if (nf == 5) {
            float th = Qf[2] / Qf[0];
            s32 = sigma5(Qf[3] / (Qf[0] * th * sqrtf(th)), Qf[4] / (Qf[0] * th * th));
        } else {
            Dimless14<float> d;
            dimless14(Qf, d);
            s32 = d.sig;
            cond = d.det >= 1e-3f;
        }
        if (cond && s32 <= 0.99f) return true;     // NaN falls through to FP64
    }
    return raw_sigma(Q, nf) <= 1.0 + 1e-9;
}

// 0 ok; 1 non-finite; 2 rho <= 0 or P not positive definite; 3 sigma > 1
__device__ __forceinline__ int check_prim(const double* Q, int nf) {
    for (int k = 0; k < nf; ++k)
        if (!isfinite(Q[k])) return 1;
    if (!(Q[0] > 0.0)) return 2;
    if (nf == 5) {
        if (!(Q[2] > 0.0)) return 2;
    } else {
        double a = Q[4], b = Q[5], c = Q[6], d = Q[7], e = Q[8], f = Q[9];
        double m2 = a * d - b * b;
        double det = a * (d * f - e * e) - b * (b * f - e * c) + c * (b * e - d * c);
        if (!(a > 0.0) || !(m2 > 0.0) || !(det > 0.0)) return 2;
    }
    if (!sigma_within_one(Q, nf)) return 3;
    return 0;
}

__device__ __forceinline__ void to_prim(const double* U, double* Q, int nf) {
    if (nf == 5) cons2prim5(U, Q); else cons2prim14(U, Q);
}
__device__ __forceinline__ void to_cons(const double* Q, double* U, int nf) {
    if (nf == 5) prim2cons5(Q, U); else prim2cons14(Q, U);
}

// Validate a dense input array; the smallest failing cell number and its
// code go to bad[0], bad[1] (64-bit: code in the top bits).
// (the field count is a template parameter so that the per-cell arrays stay
// in registers)
template <int NF>
__device__ __forceinline__ void validate_body(const CellMap& m, int kind, const double* src,
                                              unsigned long long* bad, unsigned* nonplanar,
                                              double* copy) {
    long long dense, dfs, dev, fs, idx;
    const bool has = cell_of(m, dense, dfs, dev, fs, idx);
    bool np = false;
    if (has) {
        double V[NF], Q[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) V[k] = src[dense + k * dfs];
        if (copy) {
#pragma unroll
            for (int k = 0; k < NF; ++k) copy[dense + k * dfs] = V[k];
        }
        if (kind == 0) {
#pragma unroll
            for (int k = 0; k < NF; ++k) Q[k] = V[k];
        } else {
            to_prim(V, Q, NF);
        }
        int code = check_prim(Q, NF);
        if (code) atomicMin(bad, ((unsigned long long)idx << 2) | (unsigned long long)code);
        // planar iff the z-odd moments (u_z, P_xz, P_yz, q_z) vanish; on the
        // conserved side they are rho u_z, E_xz, E_yz, H_z (same positions)
        if (NF == 14) np = V[3] != 0.0 || V[6] != 0.0 || V[8] != 0.0 || V[12] != 0.0;
    }
    // one atomic per warp that saw a non-planar cell (blocks are whole warps)
    if (__any_sync(0xffffffffu, np) && (threadIdx.x & 31) == 0) atomicOr(nonplanar, 1u);
}

// copy (may be null): receives src, same layout (a host-resident src is then
// read once, over the host link, by this kernel)
extern "C" __global__ void mxe_k_validate(CellMap m, int nf, int kind, const double* src,
                                          unsigned long long* bad, unsigned* nonplanar,
                                          double* copy) {
    if (nf == 5) validate_body<5>(m, kind, src, bad, nonplanar, copy);
    else validate_body<14>(m, kind, src, bad, nonplanar, copy);
}

template <int NF>
__device__ __forceinline__ void setstate_body(const CellMap& m, int kind, const double* src,
                                              double* U) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[NF], W[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) V[k] = src[dense + k * dfs];
    if (kind == 0) {
        to_cons(V, W, NF);
    } else {
#pragma unroll
        for (int k = 0; k < NF; ++k) W[k] = V[k];
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) U[dev + k * fs] = W[k];
}

extern "C" __global__ void mxe_k_setstate(CellMap m, int nf, int kind, const double* src,
                                          double* U) {
    if (nf == 5) setstate_body<5>(m, kind, src, U);
    else setstate_body<14>(m, kind, src, U);
}

// kind 0 primitive, 1 conserved, 2 raw sigma (one field)
template <int NF>
__device__ __forceinline__ void getstate_body(const CellMap& m, int kind, const double* U,
                                              double* dst) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[NF], Q[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) V[k] = U[dev + k * fs];
    if (kind == 1) {
#pragma unroll
        for (int k = 0; k < NF; ++k) dst[dense + k * dfs] = V[k];
        return;
    }
    to_prim(V, Q, NF);
    if (kind == 0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) dst[dense + k * dfs] = Q[k];
        return;
    }
    dst[idx] = raw_sigma(Q, NF);
}

extern "C" __global__ void mxe_k_getstate(CellMap m, int nf, int kind, const double* U,
                                          double* dst) {
    if (nf == 5) getstate_body<5>(m, kind, U, dst);
    else getstate_body<14>(m, kind, U, dst);
}

// Boundary ghost states as the stencil sees them: prim -> conserved -> prim.
extern "C" __global__ void mxe_k_ghost(int nf, int n, const double* in, double* out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double Q[14], U[14];
    for (int k = 0; k < 14; ++k) Q[k] = in[s * 14 + k];
    to_cons(Q, U, nf);
    to_prim(U, Q, nf);
    for (int k = 0; k < 14; ++k) out[s * 14 + k] = k < nf ? Q[k] : 0.0;
}

// Diagnostics in two passes with a fixed summation order (the result does
// not depend on the scheduling of blocks).  Pass 1: each block writes
// DIAG_W partials: [0, nf) field sums over its cells, [16] min raw sigma,
// [17] sigma < sigma_lim, [18] sigma > 1, [19] non-positive, [20]
// non-finite cell counts (counts held exactly as doubles).
constexpr int DIAG_W = 24;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int NF>
__device__ __forceinline__ void diag_body(const CellMap& m, const double* U, double sigma_lim,
                                          double* part) {
    constexpr int nf = NF;
    __shared__ double sh[4][DIAG_W];
    double v[DIAG_W];
#pragma unroll
    for (int k = 0; k < DIAG_W; ++k) v[k] = 0.0;
    v[16] = INFINITY;
    long long dense, dfs, dev, fs, idx;
    if (cell_of(m, dense, dfs, dev, fs, idx)) {
        double V[NF], Q[NF];
#pragma unroll
        for (int k = 0; k < nf; ++k) V[k] = U[dev + k * fs];
        bool fin = true;
#pragma unroll
        for (int k = 0; k < nf; ++k) {
            fin &= isfinite(V[k]);
            v[k] = V[k];
        }
        if (!fin) {
            v[20] = 1.0;
        } else {
            to_prim(V, Q, nf);
            bool pos = Q[0] > 0.0 &&
                       (nf == 5 ? Q[2] > 0.0 : (Q[4] > 0.0 && Q[7] > 0.0 && Q[9] > 0.0));
            if (!pos) {
                v[19] = 1.0;
            } else {
                double sg = raw_sigma(Q, nf);
                v[17] = sg < sigma_lim ? 1.0 : 0.0;
                v[18] = sg > 1.0 ? 1.0 : 0.0;
                v[16] = sg;
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < DIAG_W; ++k) {
        double r = k == 16 ? warp_min_d(v[k]) : warp_sum_d(v[k]);
        if (lane == 0) sh[w][k] = r;
    }
    __syncthreads();
    if (threadIdx.x < DIAG_W) {
        int k = threadIdx.x;
        double r = sh[0][k];
        for (int q = 1; q < 4; ++q) r = k == 16 ? fmin(r, sh[q][k]) : r + sh[q][k];
        part[((long long)blockIdx.y * gridDim.x + blockIdx.x) * DIAG_W + k] = r;
    }
}

extern "C" __global__ void __launch_bounds__(128)
mxe_k_diag(CellMap m, int nf, const double* U, double sigma_lim, double* part) {
    if (nf == 5) diag_body<5>(m, U, sigma_lim, part);
    else diag_body<14>(m, U, sigma_lim, part);
}

// Pass 2 (one block of 256 threads): acc[k] = the partials combined, each
// thread over a fixed stride of blocks, then a fixed tree.
extern "C" __global__ void __launch_bounds__(256)
mxe_k_diag_reduce(const double* part, long long nblocks, double* acc) {
    __shared__ double sh[256];
    for (int k = 0; k < 21; ++k) {
        double r = k == 16 ? INFINITY : 0.0;
        for (long long b = threadIdx.x; b < nblocks; b += 256) {
            double x = part[b * DIAG_W + k];
            r = k == 16 ? fmin(r, x) : r + x;
        }
        sh[threadIdx.x] = r;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (threadIdx.x < h)
                sh[threadIdx.x] = k == 16 ? fmin(sh[threadIdx.x], sh[threadIdx.x + h])
                                          : sh[threadIdx.x] + sh[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) acc[k] = sh[0];
        __syncthreads();
    }
}

}  // namespace mxe
