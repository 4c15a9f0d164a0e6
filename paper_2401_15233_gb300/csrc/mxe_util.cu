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
    double s = raw_sigma(Q, nf);
    if (!(s <= 1.0 + 1e-9)) return 3;
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
extern "C" __global__ void mxe_k_validate(CellMap m, int nf, int kind, const double* src,
                                          unsigned long long* bad, unsigned* nonplanar) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[14], Q[14];
    for (int k = 0; k < nf; ++k) V[k] = src[dense + k * dfs];
    if (kind == 0) for (int k = 0; k < nf; ++k) Q[k] = V[k];
    else to_prim(V, Q, nf);
    int code = check_prim(Q, nf);
    if (code) atomicMin(bad, ((unsigned long long)idx << 2) | (unsigned long long)code);
    // planar iff the z-odd moments (u_z, P_xz, P_yz, q_z) vanish; on the
    // conserved side they are rho u_z, E_xz, E_yz, H_z (same positions)
    if (nf == 14 && (V[3] != 0.0 || V[6] != 0.0 || V[8] != 0.0 || V[12] != 0.0))
        atomicOr(nonplanar, 1u);
}

extern "C" __global__ void mxe_k_setstate(CellMap m, int nf, int kind, const double* src,
                                          double* U) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[14], W[14];
    for (int k = 0; k < nf; ++k) V[k] = src[dense + k * dfs];
    if (kind == 0) to_cons(V, W, nf);
    else for (int k = 0; k < nf; ++k) W[k] = V[k];
    for (int k = 0; k < nf; ++k) U[dev + k * fs] = W[k];
}

// kind 0 primitive, 1 conserved, 2 raw sigma (one field)
extern "C" __global__ void mxe_k_getstate(CellMap m, int nf, int kind, const double* U,
                                          double* dst) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[14], Q[14];
    for (int k = 0; k < nf; ++k) V[k] = U[dev + k * fs];
    if (kind == 1) {
        for (int k = 0; k < nf; ++k) dst[dense + k * dfs] = V[k];
        return;
    }
    to_prim(V, Q, nf);
    if (kind == 0) {
        for (int k = 0; k < nf; ++k) dst[dense + k * dfs] = Q[k];
        return;
    }
    dst[idx] = raw_sigma(Q, nf);
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

// Diagnostics: acc[0..nf) field sums, acc[16] min sigma;
// cnt[0] sigma<lim, cnt[1] sigma>1, cnt[2] non-positive, cnt[3] non-finite.
__device__ __forceinline__ void atomic_min_double(double* a, double v) {
    unsigned long long* p = (unsigned long long*)a;
    unsigned long long old = *p, assumed;
    do {
        assumed = old;
        if (__longlong_as_double((long long)assumed) <= v) return;
        old = atomicCAS(p, assumed, (unsigned long long)__double_as_longlong(v));
    } while (old != assumed);
}

extern "C" __global__ void mxe_k_diag(CellMap m, int nf, const double* U, double sigma_lim,
                                      double* acc, unsigned long long* cnt) {
    long long dense, dfs, dev, fs, idx;
    if (!cell_of(m, dense, dfs, dev, fs, idx)) return;
    double V[14], Q[14];
    bool fin = true;
    for (int k = 0; k < nf; ++k) {
        V[k] = U[dev + k * fs];
        fin &= isfinite(V[k]);
        atomicAdd(acc + k, V[k]);
    }
    if (!fin) { atomicAdd(cnt + 3, 1ull); return; }
    to_prim(V, Q, nf);
    bool pos = Q[0] > 0.0 && (nf == 5 ? Q[2] > 0.0 : (Q[4] > 0.0 && Q[7] > 0.0 && Q[9] > 0.0));
    if (!pos) { atomicAdd(cnt + 2, 1ull); return; }
    double s = raw_sigma(Q, nf);
    if (s < sigma_lim) atomicAdd(cnt + 0, 1ull);
    if (s > 1.0) atomicAdd(cnt + 1, 1ull);
    atomic_min_double(acc + 16, s);
}

}  // namespace mxe
