// mxe_noalloc.cu -- a 1D solve that allocates no device memory.
//
// Some callers cannot allocate device memory: a host program whose device
// memory is wholly owned by its own pool allocator (an outside cudaMalloc
// either fails under the pool's cap or breaks its accounting), or a
// time-critical loop that cannot pay for cudaMalloc/cudaFree, which
// synchronise the device.  mxe_tube_run_noalloc serves them: the caller
// passes the state, and every other buffer the persistent tube kernel needs
// (the RK stage buffer, the tube descriptor, the clock and the ghost states)
// lives in file-scope __device__ arrays of fixed size below.  Every GPU that
// loads the library holds these arrays until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/maxent.h"
#include "mxe_internal.h"

namespace mxe {
extern "C" __global__ void mxe_tubes5_f64(const TubeArgs a);
extern "C" __global__ void mxe_tubes14_f64(const TubeArgs a);
int tubes_threads();

constexpr int NOALLOC_MAX_CELLS = 16384;    // 14 x 16384 doubles = 1.75 MiB of stage buffer

static __device__ __align__(256) double g_stage[14 * NOALLOC_MAX_CELLS];
static __device__ __align__(256) TubeDesc g_tube[1];
static __device__ __align__(256) TubeClock g_clock[1];
static __device__ __align__(256) double g_ghost[2 * 14];

struct NoallocPtrs {
    bool ready = false;
    double* stage = nullptr;
    TubeDesc* tube = nullptr;
    TubeClock* clock = nullptr;
    double* ghost = nullptr;
};
constexpr int MAX_DEVICES = 64;
static NoallocPtrs g_ptrs[MAX_DEVICES];
static std::mutex g_mutex;

// Device addresses of the file-scope arrays for the current device.  In host
// code the array names are host-side stand-ins, not device addresses, so
// they are looked up once per device, with that device current.
static cudaError_t noalloc_ptrs(NoallocPtrs& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    NoallocPtrs& p = g_ptrs[dev];
    if (!p.ready) {
        if ((e = cudaGetSymbolAddress((void**)&p.stage, g_stage)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&p.tube, g_tube)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&p.clock, g_clock)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress((void**)&p.ghost, g_ghost)) != cudaSuccess) return e;
        p.ready = true;
    }
    out = p;
    return cudaSuccess;
}

// Writes the tube descriptor and a fresh clock into the fixed arrays.  Both
// arrive by value as kernel arguments, so no host buffer has to outlive the
// call (a cudaMemcpyAsync from a stack variable would).
__global__ void mxe_noalloc_init(const TubeDesc td, const TubeClock ck) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        g_tube[0] = td;
        g_clock[0] = ck;
    }
}

}  // namespace mxe

using namespace mxe;

extern "C" mxe_status mxe_tube_run_noalloc(const mxe_config* cfg, int bc_lo, int bc_hi,
                                           int tau_model, double tau_ref, double rho_ref,
                                           double T_ref, double* U, double t0, double t_end,
                                           int max_steps, double* t_out, int* steps_out,
                                           void* stream) {
    if (!cfg || !U) return MXE_EINVAL;
    if (cfg->system != 5 && cfg->system != 14) return MXE_EINVAL;
    if (cfg->ny != 1 || cfg->nx < 4 || !(cfg->x1 > cfg->x0)) return MXE_EINVAL;
    if (cfg->nx > NOALLOC_MAX_CELLS) return MXE_EINVAL;          // beyond the fixed scratch
    if (cfg->precision != MXE_FP64) return MXE_EINVAL;
    if (cfg->order != 1 && cfg->order != 2) return MXE_EINVAL;
    if (cfg->integrator != MXE_FE && cfg->integrator != MXE_RK2) return MXE_EINVAL;
    if (cfg->flux != MXE_FLUX_HLL && cfg->flux != MXE_FLUX_RUSANOV) return MXE_EINVAL;
    if (cfg->limiter != MXE_LIM_MINMOD && cfg->limiter != MXE_LIM_VANALBADA) return MXE_EINVAL;
    if (!(cfg->cfl > 0.0) || !(cfg->sigma_lim > 0.0 && cfg->sigma_lim < 1.0) ||
        !(cfg->k_ws >= 1.0))
        return MXE_EINVAL;
    if ((bc_lo != MXE_BC_TRANSMISSIVE && bc_lo != MXE_BC_PERIODIC) ||
        (bc_hi != MXE_BC_TRANSMISSIVE && bc_hi != MXE_BC_PERIODIC) ||
        ((bc_lo == MXE_BC_PERIODIC) != (bc_hi == MXE_BC_PERIODIC)))
        return MXE_EINVAL;
    if (tau_model < 0 || tau_model > 2 || (tau_model != 0 && !(tau_ref > 0.0))) return MXE_EINVAL;
    if (max_steps < 0) return MXE_EINVAL;

    NoallocPtrs p;
    if (noalloc_ptrs(p) != cudaSuccess) return MXE_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    TubeDesc td{};
    td.off = 0;
    td.n = cfg->nx;
    td.dx = (cfg->x1 - cfg->x0) / cfg->nx;
    td.rp = RelaxParams{tau_model, tau_ref, rho_ref, T_ref};
    TubeClock ck{};               // the clock must start from t0 with no steps and no status
    ck.t = t0;
    mxe_noalloc_init<<<1, 32, 0, st>>>(td, ck);
    if (cudaGetLastError() != cudaSuccess) return MXE_ECUDA;

    TubeArgs a{};
    a.U = U;
    a.Us = p.stage;
    a.tubes = p.tube;
    a.clk = p.clock;
    a.bc_type[0] = bc_lo;
    a.bc_type[1] = bc_hi;
    a.ghost = p.ghost;            // read only for Dirichlet sides, which are not offered here
    a.ntubes = 1;
    a.system = cfg->system;
    a.integrator = cfg->integrator;
    a.sp.sigma_lim = cfg->sigma_lim;
    a.sp.k_ws = cfg->k_ws;
    a.sp.flux = cfg->flux;
    a.sp.limiter = cfg->limiter;
    a.sp.order = cfg->order;
    a.cfl = cfg->cfl;
    a.t_end = t_end;
    a.max_steps = max_steps;
    if (cfg->system == 5) mxe_tubes5_f64<<<1, tubes_threads(), 0, st>>>(a);
    else mxe_tubes14_f64<<<1, tubes_threads(), 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return MXE_ECUDA;
    if (t_out || steps_out) {
        if (cudaMemcpyAsync(&ck, p.clock, sizeof ck, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return MXE_ECUDA;
        if (t_out) *t_out = ck.t;
        if (steps_out) *steps_out = (int)ck.steps;
        if (ck.status & ST_NONFINITE) return MXE_ENONFINITE;
    }
    return MXE_OK;
}
