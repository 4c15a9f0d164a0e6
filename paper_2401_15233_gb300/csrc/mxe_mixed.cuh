// mxe_mixed.cuh -- pieces of the mixed-precision path shared by the 2D
// stage kernels and the batched tube kernel: the policy that sends an
// ill-conditioned closure back to FP64, and the face-state evaluation that
// applies it.
#pragma once
#include "mxe_policy.cuh"

namespace mxe {

// A face state is re-evaluated in FP64 when sigma lies in [sigma_lim,
// sig_lo) (near the Junk subspace), above sig_hi (near the realizability
// boundary), or when det P* < det_min.
struct MixedPolicy {
    float sig_lo, sig_hi, det_min;
};

// FP64 re-evaluation of one face state (kept out of line: rare path).  The
// state goes in and the result comes back by value, so that the caller's
// arrays never have their address taken and stay in registers.
template <int NF>
struct FaceIn {
    float q[NF];
};
template <int NF>
struct FaceOut {
    float v[2 * NF + 2];
};

template <class PH, int K>
__device__ __noinline__ FaceOut<PH::NF> face_fp64(FaceIn<PH::NF> in, double sl, double kw) {
    constexpr int NF = PH::NF;
    double Q[NF], U[NF], F[NF], lo, hi;
#pragma unroll
    for (int k = 0; k < NF; ++k) Q[k] = (double)in.q[k];
    PH::template face<double, K>(Q, sl, kw, U, F, lo, hi);
    FaceOut<NF> r;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        r.v[k] = (float)U[k];
        r.v[NF + k] = (float)F[k];
    }
    r.v[2 * NF] = (float)lo;
    r.v[2 * NF + 1] = (float)hi;
    return r;
}

// One face state: conserved U, flux F, wave speeds (out[2NF], out[2NF+1]);
// FP64 re-evaluation where the closure is ill-conditioned.
template <class PH, int K>
__device__ __forceinline__ bool face_state_m(const float* Qf, const ParamsT<float>& p,
                                             const MixedPolicy& mp, double sl64, double kw64,
                                             float* out) {
    constexpr int NF = PH::NF;
    float lo, hi;
    bool flag = false;
    if (mp.sig_lo > 0.0f || mp.sig_hi < 1.0f || mp.det_min > 0.0f) {
        // the conditioning comes out of the same evaluation
        float sig, det;
        PH::template face_c<float, K>(Qf, p.sigma_lim, p.k_ws, out, out + NF, lo, hi, sig, det);
        out[2 * NF] = lo;
        out[2 * NF + 1] = hi;
        flag = (sig >= p.sigma_lim && sig < mp.sig_lo) || sig > mp.sig_hi || det < mp.det_min ||
               !(sig == sig);
        if (__any_sync(__activemask(), flag)) {
            if (flag) {
                FaceIn<NF> in;
#pragma unroll
                for (int k = 0; k < NF; ++k) in.q[k] = Qf[k];
                FaceOut<NF> r = face_fp64<PH, K>(in, sl64, kw64);
#pragma unroll
                for (int n = 0; n < 2 * NF + 2; ++n) out[n] = r.v[n];
            }
        }
    } else {
        PH::template face<float, K>(Qf, p.sigma_lim, p.k_ws, out, out + NF, lo, hi);
        out[2 * NF] = lo;
        out[2 * NF + 1] = hi;
    }
    return flag;
}

}  // namespace mxe
