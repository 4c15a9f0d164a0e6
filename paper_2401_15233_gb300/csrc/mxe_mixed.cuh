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

// FP64 re-evaluation of one face state (kept out of line: rare path)
template <class PH, int K>
__device__ __noinline__ void face_fp64(const float* Qf, double sl, double kw, float* out) {
    constexpr int NF = PH::NF;
    double Q[NF], U[NF], F[NF], lo, hi;
#pragma unroll
    for (int k = 0; k < NF; ++k) Q[k] = (double)Qf[k];
    PH::template face<double, K>(Q, sl, kw, U, F, lo, hi);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        out[k] = (float)U[k];
        out[NF + k] = (float)F[k];
    }
    out[2 * NF] = (float)lo;
    out[2 * NF + 1] = (float)hi;
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
            if (flag) face_fp64<PH, K>(Qf, sl64, kw64, out);
        }
    } else {
        PH::template face<float, K>(Qf, p.sigma_lim, p.k_ws, out, out + NF, lo, hi);
        out[2 * NF] = lo;
        out[2 * NF + 1] = hi;
    }
    return flag;
}

}  // namespace mxe
