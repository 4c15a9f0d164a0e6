// mxe_capi.cu -- host implementation of the C-ABI declared in include/maxent.h.
//
// A context owns its device buffers and a CUDA stream.  2D grids advance
// with one fused tile kernel per RK stage (dt formed on the device from the
// previous step's CFL reduction, so a step needs no host round trip); 1D
// problems and batches of tubes advance inside one persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/maxent.h"
#include "mxe_internal.h"

#include "mxe_mixed.cuh"

namespace mxe {
// kernels defined in the other translation units
extern "C" __global__ void mxe_stage14_2d_f64(const Stage2DArgs a);
extern "C" __global__ void mxe_stage14_2d_f64_planar(const Stage2DArgs a);
extern "C" __global__ void mxe_rate14_2d(const double* U, Grid2D g, SchemeParams sp,
                                         DevClock* clk, int slot);
extern "C" __global__ void mxe_rate14_2d_planar(const double* U, Grid2D g, SchemeParams sp,
                                                DevClock* clk, int slot);
extern "C" __global__ void mxe_tubes5_f64(const TubeArgs a);
extern "C" __global__ void mxe_tubes14_f64(const TubeArgs a);
size_t stage14_2d_f64_smem(bool planar);
extern "C" __global__ void mxe_stage14_2d_mixed(const Stage2DArgs a, const ParamsT<float> p,
                                                const MixedPolicy mp);
extern "C" __global__ void mxe_stage14_2d_mixed_planar(const Stage2DArgs a,
                                                       const ParamsT<float> p,
                                                       const MixedPolicy mp);
extern "C" __global__ void mxe_stage14_2d_mixed_b3(const Stage2DArgs a, const ParamsT<float> p,
                                                   const MixedPolicy mp);
extern "C" __global__ void mxe_stage14_2d_mixed_planar_b3(const Stage2DArgs a,
                                                          const ParamsT<float> p,
                                                          const MixedPolicy mp);
extern "C" __global__ void mxe_stage14_2d_mixed_planar_x2(const Stage2DArgs a,
                                                          const ParamsT<float> p,
                                                          const MixedPolicy mp);
extern "C" __global__ void mxe_resync14_2d(const double* U, float* W, Grid2D g);
extern "C" __global__ void mxe_resync14_2d_planar(const double* U, float* W, Grid2D g);
extern "C" __global__ void mxe_rate14_2d_mixed(const float* W, Grid2D g, ParamsT<float> p,
                                               float idxf, float idyf, DevClock* clk, int slot);
extern "C" __global__ void mxe_rate14_2d_mixed_planar(const float* W, Grid2D g,
                                                      ParamsT<float> p, float idxf, float idyf,
                                                      DevClock* clk, int slot);
size_t stage14_2d_mixed_smem(bool planar, int blocks_per_sm);
size_t stage14_2d_mixed_x2_smem();
int stage14_2d_mixed_x2_tile_x();
int stage14_2d_mixed_x2_tile_y();
const void* tubes_mixed_kernel(bool planar, int nt);
cudaError_t adj_stage(const double* U, const double* V, double coef, const double* b1,
                      const double* b2, double* out, double* P, double* Cx, double* Cy,
                      double* gbar, double* taubar, const Grid2D& g, const ParamsT<double>& p,
                      bool f32, float* f32buf, bool frozen_phi, cudaStream_t st);
long long adj_f32_floats(const Grid2D& g);
extern "C" __global__ void mxe_adj_pack(const double* dense, double* pitched, Grid2D g, int to_pitched,
                                        unsigned long long* nonfinite);
size_t tubes_mixed_smem(bool planar, int nt);
void tube_rates(bool planar, const double* U, const TubeDesc* tubes, int ntubes, float sl,
                float kw, float* rates, cudaStream_t st);
int tile_x();
int tile_y();
int tubes_threads();

extern "C" __global__ void mxe_k_validate(CellMap m, int nf, int kind, const double* src,
                                          unsigned long long* bad, unsigned* nonplanar,
                                          double* copy);
extern "C" __global__ void mxe_k_setstate(CellMap m, int nf, int kind, const double* src,
                                          double* U);
extern "C" __global__ void mxe_k_getstate(CellMap m, int nf, int kind, const double* U,
                                          double* dst);
extern "C" __global__ void mxe_k_ghost(int nf, int n, const double* in, double* out);
extern "C" __global__ void mxe_k_diag(CellMap m, int nf, const double* U, double sigma_lim,
                                      double* part);
extern "C" __global__ void mxe_k_diag_reduce(const double* part, long long nblocks,
                                             double* acc);
constexpr int DIAG_W = 24;
}  // namespace mxe

using namespace mxe;

struct mxe_ctx {
    mxe_config cfg;
    int nf = 14;
    bool tubes = false;               // 1D problems (single or batched)
    int ntubes = 0;
    long long ncell = 0;              // cells in total
    long long nelem = 0;              // device elements per state buffer
    // 2D grid
    Grid2D g{};
    int slot = 0;
    DevClock* clk = nullptr;
    // tubes
    std::vector<TubeDesc> tdesc;
    std::vector<int> tn;
    TubeDesc* tdesc_d = nullptr;
    TubeClock* tclk = nullptr;
    int* order_d = nullptr;           // mixed tubes: hand-out order (longest work first)
    std::vector<int> order_h;         // the same order on the host
    int* queue_d = nullptr;           // mixed tubes: work counters of the team and fill launches
    cudaStream_t fill_stream = nullptr;    // the fill launch (forked from and joined to the work stream)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    float* rates_d = nullptr;         // per-tube CFL rate (step estimates of the split)
    int lay_teams = 0, lay_nA = 0, lay_fill = 0;   // layout of the last mixed tube launch
    int g_lay_teams = 0, g_lay_nA = 0, g_lay_fill = 0;   // layout captured in the graph
    int tune_nt = 128, tune_cl = 1;   // block shape of the mixed tube launch
    bool tuned = false;
    int nsm = 0;
    cudaStream_t cap_stream = nullptr;     // graph capture only (never executes work)
    cudaGraphExec_t gexec = nullptr;       // captured [queue reset, persistent launch]
    double g_tend = -1.0;
    int g_steps = -1, g_nt = 0, g_cl = 0;
    bool g_planar = false;
    long long g_gen = -1;
    long long gen = 0;                // bumped whenever launch arguments change
    // dt history of 2D grids (steps counted from set_state)
    double* dth = nullptr;
    long long dth_cap = 0;
    // discrete adjoint: tape of (U^n, U*) per recorded step, scratch
    double* tape = nullptr;
    long long tape_cap = 0;           // states the tape can hold
    int tape_n = 0;                   // recorded steps
    std::vector<double> tape_dt;
    double* adjP = nullptr;           // primitives (NP fields, pitched)
    double* adjCx = nullptr;          // face contributions
    double* adjCy = nullptr;
    double* adjA = nullptr;           // adjoint state buffers (pitched)
    double* adjB = nullptr;
    double* adjG = nullptr;           // [4][GHOST_SLOTS][14] imposed-state adjoint, then tau_ref's
    bool adj_f32 = false;             // face-state reverse in FP32 (MXE_MIXED adjoint)
    bool adj_frozen = false;          // shared limiter held constant in the derivative
    float* adjF = nullptr;            // FP32 per-cell data of that reverse
    // state
    double* U = nullptr;
    double* Us = nullptr;
    float* W = nullptr;               // mixed: FP32 primitives of U
    float* Ws = nullptr;              // mixed: FP32 primitives of the stage state
    double* diag_part = nullptr;      // diagnostics: per-block partials
    long long diag_part_n = 0;
    bool mixed = false;
    MixedPolicy mp{0.0f, 0.999f, 1e-3f};
    int resync_every = 16;
    int stage_occ = 3;                // mixed stage kernels: blocks per SM (2 or 3)
    int face_packed = 1;              // planar mixed, 3 blocks/SM: face-state pairs in f32x2
    long long launched = 0;           // steps launched since set_state
    bool state_planar = false;        // z-odd moments exactly zero (and kept so)
    bool w_planar = false;            // layout of W (mixed): compact planar fields
    double* stage = nullptr;          // dense staging buffer (nf * ncell)
    double* dts_d = nullptr;          // prescribed dt sequence
    int dts_cap = 0;
    unsigned long long* scratch = nullptr;  // validation / diagnostics counters
    double* accd = nullptr;
    // boundary conditions
    int bc_type[4] = {0, 0, 0, 0};
    int nspans[4] = {0, 0, 0, 0};
    double span_lo[4][MAX_SPANS], span_hi[4][MAX_SPANS];
    double ghost_h[4][GHOST_SLOTS][14];
    double* ghost_in = nullptr;       // raw prim states (device)
    double* ghost_d = nullptr;        // round-tripped (device)
    RelaxParams rp{0, 1.0, 1.0, 1.0};
    SchemeParams sp{};
    bool have_state = false;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    std::string err;
};

static mxe_status fail(mxe_ctx* c, mxe_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, MXE_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                            \
    } while (0)

static CellMap cellmap(const mxe_ctx* c) {
    CellMap m{};
    m.nf = c->nf;
    if (c->tubes) {
        m.mode = 1;
        m.tubes = c->tdesc_d;
        m.ntubes = c->ntubes;
    } else {
        m.mode = 0;
        m.nx = c->g.nx;
        m.ny = c->g.ny;
        m.pitch = c->g.pitch;
        m.fstride = c->g.fstride;
    }
    return m;
}

static dim3 cellgrid(const mxe_ctx* c, int threads) {
    if (c->tubes) {
        int mx = *std::max_element(c->tn.begin(), c->tn.end());
        return dim3((mx + threads - 1) / threads, c->ntubes);
    }
    return dim3((c->g.nx + threads - 1) / threads, c->g.ny);
}

static mxe_status check_cfg(mxe_ctx* c, const mxe_config* cfg, bool batch) {
    if (!cfg) return fail(c, MXE_EINVAL, "cfg is NULL");
    if (cfg->system != 5 && cfg->system != 14)
        return fail(c, MXE_EINVAL, "system must be 5 or 14 (got %d)", cfg->system);
    if (!batch) {
        if (cfg->nx < 4 || cfg->ny < 1) return fail(c, MXE_EINVAL, "need nx >= 4 and ny >= 1");
        if (cfg->ny > 1 && cfg->ny < 4) return fail(c, MXE_EINVAL, "2D grids need ny >= 4");
        if (!(cfg->x1 > cfg->x0)) return fail(c, MXE_EINVAL, "need x1 > x0");
        if (cfg->ny > 1 && !(cfg->y1 > cfg->y0)) return fail(c, MXE_EINVAL, "need y1 > y0");
    }
    if (cfg->system == 5 && cfg->ny != 1)
        return fail(c, MXE_EINVAL, "the 5-moment (1D1V) system needs ny == 1");
    if (cfg->precision != MXE_FP64 && cfg->precision != MXE_MIXED)
        return fail(c, MXE_EINVAL, "precision must be MXE_FP64 or MXE_MIXED");
    if (cfg->precision == MXE_MIXED && cfg->system != 14)
        return fail(c, MXE_EINVAL, "MXE_MIXED is available for the 14-moment system");
    if (cfg->flux != MXE_FLUX_HLL && cfg->flux != MXE_FLUX_RUSANOV)
        return fail(c, MXE_EINVAL, "unknown flux %d", cfg->flux);
    if (cfg->limiter != MXE_LIM_MINMOD && cfg->limiter != MXE_LIM_VANALBADA)
        return fail(c, MXE_EINVAL, "unknown limiter %d", cfg->limiter);
    if (cfg->order != 1 && cfg->order != 2) return fail(c, MXE_EINVAL, "order must be 1 or 2");
    if (cfg->integrator != MXE_FE && cfg->integrator != MXE_RK2)
        return fail(c, MXE_EINVAL, "integrator must be MXE_FE or MXE_RK2");
    if (!(cfg->cfl > 0.0)) return fail(c, MXE_EINVAL, "cfl must be > 0");
    if (!(cfg->sigma_lim > 0.0 && cfg->sigma_lim < 1.0))
        return fail(c, MXE_EINVAL, "sigma_lim must lie in (0, 1)");
    if (!(cfg->k_ws >= 1.0)) return fail(c, MXE_EINVAL, "k_ws must be >= 1");
    return MXE_OK;
}

static mxe_status alloc_common(mxe_ctx* c) {
    CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    c->stream = c->own_stream;
    CK(cudaMalloc(&c->U, sizeof(double) * c->nelem));
    CK(cudaMemset(c->U, 0, sizeof(double) * c->nelem));
    if (c->mixed) {
        CK(cudaMalloc(&c->W, sizeof(float) * c->nelem));
        CK(cudaMalloc(&c->Ws, sizeof(float) * c->nelem));
        CK(cudaMemset(c->W, 0, sizeof(float) * c->nelem));
        CK(cudaMemset(c->Ws, 0, sizeof(float) * c->nelem));
    } else {
        CK(cudaMalloc(&c->Us, sizeof(double) * c->nelem));
        CK(cudaMemset(c->Us, 0, sizeof(double) * c->nelem));
    }
    CK(cudaMalloc(&c->stage, sizeof(double) * c->nf * c->ncell));
    CK(cudaMalloc(&c->scratch, sizeof(unsigned long long) * 8));
    CK(cudaMalloc(&c->accd, sizeof(double) * 32));
    CK(cudaMalloc(&c->ghost_in, sizeof(double) * 4 * GHOST_SLOTS * 14));
    CK(cudaMalloc(&c->ghost_d, sizeof(double) * 4 * GHOST_SLOTS * 14));
    memset(c->ghost_h, 0, sizeof c->ghost_h);
    CK(cudaMemset(c->ghost_d, 0, sizeof(double) * 4 * GHOST_SLOTS * 14));
    c->sp.sigma_lim = c->cfg.sigma_lim;
    c->sp.k_ws = c->cfg.k_ws;
    c->sp.flux = c->cfg.flux;
    c->sp.limiter = c->cfg.limiter;
    c->sp.order = c->cfg.order;
    return MXE_OK;
}

// Tube contexts: device descriptors and clocks; for the mixed path also the
// work queue, its hand-out order (largest n/dx first: a tube's work grows as
// cells x steps ~ n^2 / length), the capture stream and the kernel
// attributes of every block shape.
static mxe_status tubes_setup(mxe_ctx* c) {
    const int n = c->ntubes;
    CK(cudaMalloc(&c->tdesc_d, sizeof(TubeDesc) * n));
    CK(cudaMalloc(&c->tclk, sizeof(TubeClock) * n));
    CK(cudaMemset(c->tclk, 0, sizeof(TubeClock) * n));
    CK(cudaMemcpy(c->tdesc_d, c->tdesc.data(), sizeof(TubeDesc) * n, cudaMemcpyHostToDevice));
    if (!c->mixed) return MXE_OK;
    std::vector<int> order(n);
    for (int b = 0; b < n; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return c->tdesc[x].n / c->tdesc[x].dx > c->tdesc[y].n / c->tdesc[y].dx;
    });
    CK(cudaMalloc(&c->order_d, sizeof(int) * n));
    CK(cudaMemcpy(c->order_d, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    c->order_h = order;
    CK(cudaMalloc(&c->rates_d, sizeof(float) * n));
    CK(cudaMalloc(&c->queue_d, 2 * sizeof(int)));
    CK(cudaMemset(c->queue_d, 0, 2 * sizeof(int)));
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->fill_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
    for (int pl = 0; pl < 2; ++pl)
        for (int nt = 128; nt <= 256; nt *= 2)
            CK(cudaFuncSetAttribute(tubes_mixed_kernel(pl, nt),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tubes_mixed_smem(pl, nt)));
    return MXE_OK;
}

extern "C" mxe_status mxe_create(const mxe_config* cfg, mxe_ctx** out) {
    if (!out) return MXE_EINVAL;
    *out = nullptr;
    mxe_ctx* c = new (std::nothrow) mxe_ctx();
    if (!c) return MXE_ENOMEM;
    mxe_status s = check_cfg(c, cfg, false);
    if (s != MXE_OK) {
        delete c;
        return s;
    }
    c->cfg = *cfg;
    c->nf = cfg->system;
    c->mixed = cfg->precision == MXE_MIXED;
    if (cfg->ny == 1) {                 // 1D: a batch of one tube
        c->tubes = true;
        c->ntubes = 1;
        TubeDesc td{};
        td.off = 0;
        td.n = cfg->nx;
        td.dx = (cfg->x1 - cfg->x0) / cfg->nx;
        td.rp = c->rp;
        c->tdesc.push_back(td);
        c->tn.push_back(cfg->nx);
        c->ncell = cfg->nx;
        c->nelem = (long long)c->nf * cfg->nx;
    } else {
        c->g.nx = cfg->nx;
        c->g.ny = cfg->ny;
        c->g.pitch = (cfg->nx + 31) / 32 * 32;
        c->g.fstride = (long long)c->g.pitch * cfg->ny;
        c->g.dx = (cfg->x1 - cfg->x0) / cfg->nx;
        c->g.dy = (cfg->y1 - cfg->y0) / cfg->ny;
        c->g.idx = 1.0 / c->g.dx;
        c->g.idy = 1.0 / c->g.dy;
        c->ncell = (long long)cfg->nx * cfg->ny;
        c->nelem = (long long)c->nf * c->g.fstride;
    }
    s = alloc_common(c);
    if (s == MXE_OK && c->tubes) {
        s = tubes_setup(c);
    } else if (s == MXE_OK) {
        cudaError_t e = cudaMalloc(&c->clk, sizeof(DevClock));
        if (e == cudaSuccess) e = cudaMemset(c->clk, 0, sizeof(DevClock));
        if (e != cudaSuccess) s = fail(c, MXE_ECUDA, "clock: %s", cudaGetErrorString(e));
    }
    if (s != MXE_OK) {
        mxe_destroy(c);
        return s;
    }
    c->g.ghost = c->ghost_d;
    if (!c->tubes) {
        cudaError_t e = c->mixed
            ? cudaFuncSetAttribute(mxe_stage14_2d_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)stage14_2d_mixed_smem(false, 2))
            : cudaFuncSetAttribute(mxe_stage14_2d_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)stage14_2d_f64_smem(false));
        if (e == cudaSuccess)
            e = c->mixed ? cudaFuncSetAttribute(mxe_stage14_2d_mixed_planar,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)stage14_2d_mixed_smem(true, 2))
                         : cudaFuncSetAttribute(mxe_stage14_2d_f64_planar,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)stage14_2d_f64_smem(true));
        if (e == cudaSuccess && c->mixed)
            e = cudaFuncSetAttribute(mxe_stage14_2d_mixed_planar_b3,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stage14_2d_mixed_smem(true, 3));
        if (e == cudaSuccess && c->mixed)
            e = cudaFuncSetAttribute(mxe_stage14_2d_mixed_planar_x2,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stage14_2d_mixed_x2_smem());
        if (e == cudaSuccess && c->mixed)
            e = cudaFuncSetAttribute(mxe_stage14_2d_mixed_b3,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)stage14_2d_mixed_smem(false, 3));
        if (e != cudaSuccess) {
            fail(c, MXE_ECUDA, "smem attribute: %s", cudaGetErrorString(e));
            mxe_destroy(c);
            return MXE_ECUDA;
        }
    }
    *out = c;
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_create(const mxe_config* cfg, int n, const int* ncells,
                                       const double* length, mxe_ctx** out) {
    if (!out) return MXE_EINVAL;
    *out = nullptr;
    mxe_ctx* c = new (std::nothrow) mxe_ctx();
    if (!c) return MXE_ENOMEM;
    mxe_status s = check_cfg(c, cfg, true);
    if (s == MXE_OK && cfg->ny != 1) s = fail(c, MXE_EINVAL, "batched tubes need ny == 1");
    if (s == MXE_OK && (n < 1 || !ncells || !length)) s = fail(c, MXE_EINVAL, "bad tube list");
    if (s != MXE_OK) {
        delete c;
        return s;
    }
    c->cfg = *cfg;
    c->nf = cfg->system;
    c->mixed = cfg->precision == MXE_MIXED;
    c->tubes = true;
    c->ntubes = n;
    long long off = 0;
    for (int b = 0; b < n; ++b) {
        if (ncells[b] < 4 || !(length[b] > 0.0)) {
            delete c;
            return MXE_EINVAL;
        }
        TubeDesc td{};
        td.off = off;
        td.coff = c->ncell;
        td.n = ncells[b];
        td.dx = length[b] / ncells[b];
        td.rp = c->rp;
        c->tdesc.push_back(td);
        c->tn.push_back(ncells[b]);
        off += (long long)c->nf * ncells[b];
        c->ncell += ncells[b];
    }
    c->nelem = off;
    s = alloc_common(c);
    if (s == MXE_OK) s = tubes_setup(c);
    if (s != MXE_OK) {
        mxe_destroy(c);
        return s;
    }
    *out = c;
    return MXE_OK;
}

extern "C" void mxe_destroy(mxe_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->U);
    cudaFree(c->Us);
    cudaFree(c->W);
    cudaFree(c->Ws);
    cudaFree(c->diag_part);
    cudaFree(c->stage);
    cudaFree(c->scratch);
    cudaFree(c->accd);
    cudaFree(c->ghost_in);
    cudaFree(c->ghost_d);
    cudaFree(c->clk);
    cudaFree(c->tdesc_d);
    cudaFree(c->tclk);
    cudaFree(c->dts_d);
    cudaFree(c->order_d);
    cudaFree(c->queue_d);
    cudaFree(c->rates_d);
    cudaFree(c->dth);
    cudaFree(c->tape);
    cudaFree(c->adjP);
    cudaFree(c->adjCx);
    cudaFree(c->adjCy);
    cudaFree(c->adjA);
    cudaFree(c->adjB);
    cudaFree(c->adjG);
    cudaFree(c->adjF);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->fill_stream) cudaStreamDestroy(c->fill_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

extern "C" mxe_status mxe_set_stream(mxe_ctx* c, void* stream) {
    if (!c) return MXE_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    return MXE_OK;
}

extern "C" void* mxe_get_stream(const mxe_ctx* c) { return c ? (void*)c->stream : nullptr; }

extern "C" const char* mxe_last_error(const mxe_ctx* c) { return c ? c->err.c_str() : ""; }

// ---------------------------------------------------------------- planar states
// The z-odd moments (u_z, P_xz, P_yz, q_z) of a 14-moment 2D state stay
// exactly zero when they are zero initially and in every boundary state;
// the planar kernels then carry the ten remaining moments only.
static bool bc_planar(const mxe_ctx* c) {
    const int zodd[4] = {3, 6, 8, 12};
    for (int s = 0; s < 4; ++s)
        for (int n = 0; n < GHOST_SLOTS; ++n) {
            bool used = (n == 0 && c->bc_type[s] == MXE_BC_DIRICHLET) || (n > 0 && n <= c->nspans[s]);
            if (!used) continue;
            for (int z : zodd)
                if (c->ghost_h[s][n][z] != 0.0) return false;
        }
    return true;
}

static bool use_planar(mxe_ctx* c) {
    if (c->tubes || c->nf != 14) return false;
    if (c->state_planar && !bc_planar(c)) c->state_planar = false;   // stays off until set_state
    return c->state_planar;
}

static ParamsT<float> fparams(const mxe_ctx* c) { return make_params<float>(c->sp, c->rp); }

static void launch_resync(mxe_ctx* c, bool planar) {
    dim3 rg((c->g.nx + 255) / 256, c->g.ny);
    if (planar) mxe_resync14_2d_planar<<<rg, 256, 0, c->stream>>>(c->U, c->W, c->g);
    else mxe_resync14_2d<<<rg, 256, 0, c->stream>>>(c->U, c->W, c->g);
    c->w_planar = planar;
}

// ---------------------------------------------------------------- clocks
static mxe_status reset_clock(mxe_ctx* c) {
    if (c->tubes) {
        std::vector<TubeClock> z(c->ntubes);
        memset(z.data(), 0, sizeof(TubeClock) * c->ntubes);
        CK(cudaMemcpyAsync(c->tclk, z.data(), sizeof(TubeClock) * c->ntubes,
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return MXE_OK;
    }
    CK(cudaMemsetAsync(c->clk, 0, sizeof(DevClock), c->stream));
    c->slot = 0;
    c->launched = 0;
    int nt = 256;
    dim3 grid((c->g.nx + nt - 1) / nt, c->g.ny);
    bool pl = use_planar(c);
    if (c->mixed) {
        launch_resync(c, pl);
        if (pl)
            mxe_rate14_2d_mixed_planar<<<grid, nt, 0, c->stream>>>(c->W, c->g, fparams(c),
                                                                   (float)c->g.idx, (float)c->g.idy,
                                                                   c->clk, 0);
        else
            mxe_rate14_2d_mixed<<<grid, nt, 0, c->stream>>>(c->W, c->g, fparams(c), (float)c->g.idx,
                                                            (float)c->g.idy, c->clk, 0);
    } else {
        if (pl) mxe_rate14_2d_planar<<<grid, nt, 0, c->stream>>>(c->U, c->g, c->sp, c->clk, 0);
        else mxe_rate14_2d<<<grid, nt, 0, c->stream>>>(c->U, c->g, c->sp, c->clk, 0);
    }
    CK(cudaGetLastError());
    return MXE_OK;
}

// ---------------------------------------------------------------- state I/O
// Device address of a page-locked (pinned or registered) host buffer, which
// kernels read and write directly over the host link; nullptr for pageable
// memory (then the data moves through the context's stage buffer).
static void* pinned_alias(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

extern "C" mxe_status mxe_set_state(mxe_ctx* c, int kind, const double* soa, int on_device) {
    if (!c) return MXE_EINVAL;
    if (!soa) return fail(c, MXE_EINVAL, "soa is NULL");
    if (kind != MXE_PRIMITIVE && kind != MXE_CONSERVED && kind != MXE_CONSERVED_RESTORE)
        return fail(c, MXE_EINVAL, "kind must be PRIMITIVE, CONSERVED or CONSERVED_RESTORE");
    const bool restore = kind == MXE_CONSERVED_RESTORE;
    if (restore) kind = MXE_CONSERVED;
    size_t bytes = sizeof(double) * c->nf * c->ncell;
    const double* src = soa;
    const double* vsrc = soa;        // what the validation kernel reads
    double* copy = nullptr;          // where it leaves a device copy
    if (!on_device) {
        src = c->stage;
        vsrc = (const double*)pinned_alias(soa);
        if (vsrc) {
            copy = c->stage;         // one pass over the host link, fused with the checks
        } else {
            CK(cudaMemcpyAsync(c->stage, soa, bytes, cudaMemcpyHostToDevice, c->stream));
            vsrc = c->stage;
        }
    }
    unsigned long long init[2] = {~0ull, 0ull};
    CK(cudaMemcpyAsync(c->scratch, init, sizeof init, cudaMemcpyHostToDevice, c->stream));
    CellMap m = cellmap(c);
    dim3 grid = cellgrid(c, 128);
    mxe_k_validate<<<grid, 128, 0, c->stream>>>(m, c->nf, kind, vsrc, c->scratch,
                                                (unsigned*)(c->scratch + 1), copy);
    CK(cudaGetLastError());
    unsigned long long res[2] = {0, 0};
    CK(cudaMemcpyAsync(res, c->scratch, sizeof res, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    unsigned long long bad = res[0];
    if (bad != ~0ull && !restore) {
        unsigned long long idx = bad >> 2;
        int code = (int)(bad & 3);
        const char* why = code == 1 ? "non-finite value"
                        : code == 2 ? "rho <= 0 or pressure tensor not positive definite"
                                    : "sigma > 1 (outside the realizability boundary)";
        return fail(c, code == 1 ? MXE_ENONFINITE : MXE_EUNREALIZABLE,
                    "input cell %llu: %s", idx, why);
    }
    mxe_k_setstate<<<grid, 128, 0, c->stream>>>(m, c->nf, kind, src, c->U);
    CK(cudaGetLastError());
    c->state_planar = (res[1] == 0ull);
    if (!c->tubes && c->Us) CK(cudaMemsetAsync(c->Us, 0, sizeof(double) * c->nelem, c->stream));
    mxe_status s = reset_clock(c);
    if (s != MXE_OK) return s;
    c->have_state = true;
    return MXE_OK;
}

extern "C" mxe_status mxe_get_moments(mxe_ctx* c, int kind, double* soa, int on_device) {
    if (!c) return MXE_EINVAL;
    if (!soa) return fail(c, MXE_EINVAL, "soa is NULL");
    if (kind < 0 || kind > 2) return fail(c, MXE_EINVAL, "bad kind %d", kind);
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    int nfo = kind == MXE_SIGMA ? 1 : c->nf;
    // device array, page-locked host array (written directly by the kernel)
    // or pageable host array (through the stage buffer)
    double* pinned = on_device ? nullptr : (double*)pinned_alias(soa);
    double* dst = on_device ? soa : (pinned ? pinned : c->stage);
    CellMap m = cellmap(c);
    mxe_k_getstate<<<cellgrid(c, 128), 128, 0, c->stream>>>(m, c->nf, kind, c->U, dst);
    CK(cudaGetLastError());
    if (!on_device && !pinned)
        CK(cudaMemcpyAsync(soa, c->stage, sizeof(double) * nfo * c->ncell, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MXE_OK;
}

// ---------------------------------------------------------------- BCs, tau
static mxe_status upload_ghosts(mxe_ctx* c) {
    CK(cudaMemcpyAsync(c->ghost_in, c->ghost_h, sizeof c->ghost_h, cudaMemcpyHostToDevice,
                       c->stream));
    // Dirichlet ghosts carry the imposed primitive state itself (the
    // reconstruction acts on primitives), so no conversion is applied.
    CK(cudaMemcpyAsync(c->ghost_d, c->ghost_in, sizeof c->ghost_h, cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // 2D side descriptors: index ranges of the slots along each side
    if (!c->tubes) {
        for (int s = 0; s < 4; ++s) {
            SideDesc& sd = c->g.side[s];
            sd.type = c->bc_type[s];
            sd.nspans = 0;
            int ncell_side = s < 2 ? c->g.ny : c->g.nx;
            double o = s < 2 ? c->cfg.y0 : c->cfg.x0;
            double h = s < 2 ? (c->cfg.y1 - c->cfg.y0) / c->cfg.ny : (c->cfg.x1 - c->cfg.x0) / c->cfg.nx;
            for (int n2 = 0; n2 < c->nspans[s]; ++n2) {
                int lo = -1, hi = -2;
                for (int j = 0; j < ncell_side; ++j) {
                    double xt = o + ((double)j + 0.5) * h;
                    if (xt >= c->span_lo[s][n2] && xt <= c->span_hi[s][n2]) {
                        if (lo < 0) lo = j;
                        hi = j;
                    }
                }
                sd.lo[sd.nspans] = lo < 0 ? 1 : lo;
                sd.hi[sd.nspans] = lo < 0 ? 0 : hi;      // empty range if no cell
                ++sd.nspans;
            }
        }
        c->g.ghost = c->ghost_d;
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_set_bc(mxe_ctx* c, int side, int type, double lo, double hi,
                                 const double* prim) {
    if (!c) return MXE_EINVAL;
    ++c->gen;
    int nsides = c->tubes ? 2 : 4;
    if (side < 0 || side >= nsides) return fail(c, MXE_EINVAL, "bad side %d", side);
    if (type < 0 || type > 2) return fail(c, MXE_EINVAL, "bad BC type %d", type);
    if (type == MXE_BC_DIRICHLET && !prim) return fail(c, MXE_EINVAL, "Dirichlet needs a state");
    if (type == MXE_BC_DIRICHLET) {
        // the imposed state must itself be admissible
        for (int k = 0; k < c->nf; ++k)
            if (!std::isfinite(prim[k])) return fail(c, MXE_EINVAL, "non-finite BC state");
        if (!(prim[0] > 0.0)) return fail(c, MXE_EUNREALIZABLE, "BC state with rho <= 0");
    }
    if (type == MXE_BC_DIRICHLET && lo < hi) {
        if (c->tubes) return fail(c, MXE_EINVAL, "inflow slots need a 2D grid");
        if (c->nspans[side] >= MAX_SPANS) return fail(c, MXE_EINVAL, "at most %d slots", MAX_SPANS);
        int n = c->nspans[side]++;
        c->span_lo[side][n] = lo;
        c->span_hi[side][n] = hi;
        for (int k = 0; k < 14; ++k) c->ghost_h[side][1 + n][k] = k < c->nf ? prim[k] : 0.0;
    } else {
        c->bc_type[side] = type;
        c->nspans[side] = 0;
        if (type == MXE_BC_DIRICHLET)
            for (int k = 0; k < 14; ++k) c->ghost_h[side][0][k] = k < c->nf ? prim[k] : 0.0;
    }
    return upload_ghosts(c);
}

extern "C" mxe_status mxe_set_relaxation(mxe_ctx* c, int model, double tau_ref, double rho_ref,
                                         double T_ref) {
    if (!c) return MXE_EINVAL;
    if (model < 0 || model > 2) return fail(c, MXE_EINVAL, "bad relaxation model %d", model);
    if (model != 0 && !(tau_ref > 0.0)) return fail(c, MXE_EINVAL, "tau_ref must be > 0");
    if (model == 2 && !(rho_ref > 0.0 && T_ref > 0.0))
        return fail(c, MXE_EINVAL, "rho_ref and T_ref must be > 0");
    c->rp = RelaxParams{model, tau_ref, rho_ref, T_ref, c->rp.implicit};
    ++c->gen;
    if (c->tubes) {
        for (auto& td : c->tdesc) td.rp = c->rp;
        CK(cudaMemcpyAsync(c->tdesc_d, c->tdesc.data(), sizeof(TubeDesc) * c->ntubes,
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_set_relaxation(mxe_ctx* c, int tube, int model, double tau_ref,
                                               double rho_ref, double T_ref) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes) return fail(c, MXE_ESTATE, "not a batch context");
    if (tube < 0 || tube >= c->ntubes) return fail(c, MXE_EINVAL, "bad tube %d", tube);
    if (model < 0 || model > 2) return fail(c, MXE_EINVAL, "bad relaxation model %d", model);
    if (model != 0 && !(tau_ref > 0.0)) return fail(c, MXE_EINVAL, "tau_ref must be > 0");
    c->tdesc[tube].rp = RelaxParams{model, tau_ref, rho_ref, T_ref, c->rp.implicit};
    CK(cudaMemcpyAsync(c->tdesc_d + tube, &c->tdesc[tube], sizeof(TubeDesc),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MXE_OK;
}

extern "C" mxe_status mxe_set_source_scheme(mxe_ctx* c, int scheme) {
    if (!c) return MXE_EINVAL;
    if (scheme != MXE_SOURCE_EXPLICIT && scheme != MXE_SOURCE_POINT_IMPLICIT)
        return fail(c, MXE_EINVAL, "bad source scheme %d", scheme);
    c->rp.implicit = scheme;
    ++c->gen;
    if (c->tubes) {
        for (auto& td : c->tdesc) td.rp.implicit = scheme;
        CK(cudaMemcpyAsync(c->tdesc_d, c->tdesc.data(), sizeof(TubeDesc) * c->ntubes,
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return MXE_OK;
}

// ---------------------------------------------------------------- stepping
static mxe_status periodic_ok(mxe_ctx* c) {
    int ns = c->tubes ? 2 : 4;
    for (int s = 0; s < ns; s += 2)
        if ((c->bc_type[s] == MXE_BC_PERIODIC) != (c->bc_type[s + 1] == MXE_BC_PERIODIC))
            return fail(c, MXE_EINVAL, "periodic BCs must be set on both opposite sides");
    return MXE_OK;
}

// One step of a 2D grid.  ustar (FP64 RK2 only, optional): where stage 1
// writes U* (default: the context's stage buffer).
static mxe_status launch_2d_step(mxe_ctx* c, double t_end, double dt_fixed,
                                 double* ustar = nullptr, bool skip_rate = false) {
    Stage2DArgs a{};
    a.skip_rate = skip_rate && !c->mixed;
    a.dt_hist = c->dth;
    a.dt_hist_cap = c->dth_cap;
    a.g = c->g;
    for (int s = 0; s < 4; ++s) a.g.side[s].type = c->bc_type[s];
    a.sp = c->sp;
    a.rp = c->rp;
    a.cfl = c->cfg.cfl;
    a.t_end = t_end;
    a.dt_fixed = dt_fixed;
    a.slot = c->slot;
    a.clk = c->clk;
    a.idxf = (float)c->g.idx;
    a.idyf = (float)c->g.idy;
    dim3 grid((c->g.nx + tile_x() - 1) / tile_x(), (c->g.ny + tile_y() - 1) / tile_y());
    const bool pl = use_planar(c);
    if (c->mixed) {
        if (c->w_planar != pl) launch_resync(c, pl);       // W layout follows the kernel
        // three blocks per SM (L2 prefetch) or two (planar: with the final
        // stage's shared-memory prefetch); the same kernel for both stages
        const bool b3 = c->stage_occ == 3;
        const bool packed = pl && b3 && c->face_packed;
        const auto kern = pl ? (b3 ? mxe_stage14_2d_mixed_planar_b3 : mxe_stage14_2d_mixed_planar)
                             : (b3 ? mxe_stage14_2d_mixed_b3 : mxe_stage14_2d_mixed);
        const size_t smem = stage14_2d_mixed_smem(pl, c->stage_occ);
        // packed planar stage: its own kernel and tile
        auto launch = [&]() {
            if (!packed) {
                kern<<<grid, 256, smem, c->stream>>>(a, fparams(c), c->mp);
                return;
            }
            const int tx = stage14_2d_mixed_x2_tile_x(), ty = stage14_2d_mixed_x2_tile_y();
            dim3 gp((c->g.nx + tx - 1) / tx, (c->g.ny + ty - 1) / ty);
            mxe_stage14_2d_mixed_planar_x2<<<gp, 256, stage14_2d_mixed_x2_smem(), c->stream>>>(
                a, fparams(c), c->mp);
        };
        a.Ubase = c->U;
        a.Uout = c->U;
        a.resync = (c->launched + 1) % c->resync_every == 0;
        if (c->cfg.integrator == MXE_RK2) {
            a.Win = c->W; a.Wout = c->Ws; a.Wbase = c->W; a.coef = 0.5; a.final_stage = 0;
            launch();
            a.Win = c->Ws; a.Wout = c->W; a.Wbase = c->W; a.coef = 1.0; a.final_stage = 1;
            launch();
        } else {
            a.Win = c->W; a.Wout = c->Ws; a.Wbase = c->W; a.coef = 1.0; a.final_stage = 1;
            launch();
            std::swap(c->W, c->Ws);
        }
        CK(cudaGetLastError());
        c->slot = (c->slot + 1) % 3;
        ++c->launched;
        return MXE_OK;
    }
    auto kern = pl ? mxe_stage14_2d_f64_planar : mxe_stage14_2d_f64;
    size_t smem = stage14_2d_f64_smem(pl);
    if (c->cfg.integrator == MXE_RK2) {
        double* us = ustar ? ustar : c->Us;
        a.Uin = c->U; a.Ubase = c->U; a.Uout = us; a.coef = 0.5; a.final_stage = 0;
        kern<<<grid, 256, smem, c->stream>>>(a);
        a.Uin = us; a.Ubase = c->U; a.Uout = c->U; a.coef = 1.0; a.final_stage = 1;
        kern<<<grid, 256, smem, c->stream>>>(a);
    } else {
        a.Uin = c->U; a.Ubase = c->U; a.Uout = c->Us; a.coef = 1.0; a.final_stage = 1;
        kern<<<grid, 256, smem, c->stream>>>(a);
        std::swap(c->U, c->Us);
    }
    CK(cudaGetLastError());
    c->slot = (c->slot + 1) % 3;
    return MXE_OK;
}

static mxe_status read_clock_2d(mxe_ctx* c, DevClock* h) {
    CK(cudaMemcpyAsync(h, c->clk, sizeof(DevClock), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MXE_OK;
}

// ---------------------------------------------------------------- mixed tubes
static bool tubes_planar(mxe_ctx* c) { return c->nf == 14 && c->state_planar && bc_planar(c); }

static mxe_status upload_dts(mxe_ctx* c, const double* dts, int ndts) {
    if (ndts > c->dts_cap) {
        cudaFree(c->dts_d);
        c->dts_d = nullptr;
        CK(cudaMalloc(&c->dts_d, sizeof(double) * ndts));
        c->dts_cap = ndts;
    }
    CK(cudaMemcpyAsync(c->dts_d, dts, sizeof(double) * ndts, cudaMemcpyHostToDevice, c->stream));
    return MXE_OK;
}

static TubeMixedArgs tubes_mixed_args(mxe_ctx* c, int max_steps, double t_end) {
    TubeMixedArgs a{};
    a.U = c->U;
    a.W = c->W;
    a.Ws = c->Ws;
    a.tubes = c->tdesc_d;
    a.order = c->order_d;
    a.queue = c->queue_d;
    a.clk = c->tclk;
    a.bc_type[0] = c->bc_type[0];
    a.bc_type[1] = c->bc_type[1];
    a.ghost = c->ghost_d;
    a.ntubes = c->ntubes;
    a.integrator = c->cfg.integrator;
    a.max_steps = max_steps;
    a.resync_every = c->resync_every;
    a.cfl = c->cfg.cfl;
    a.t_end = t_end;
    a.sl64 = c->sp.sigma_lim;
    a.kw64 = c->sp.k_ws;
    return a;
}

// Launch shape of the persistent tube kernel with nt threads per CTA and
// teams of cl CTAs (a cluster when cl > 1): as many teams as can be
// resident at once, at most one per tube.  Clusters are placed whole within
// a GPU processing cluster, so a cluster launch can leave CTA slots unused
// (on the GB300, 36 teams of 8 CTAs at two CTAs per SM occupy 144 of the 152
// SMs).  Those slots run a second, concurrent launch of single CTAs ("fill")
// that takes the smallest tubes, the tail of the work order: `nA` tubes go to
// the teams, the rest to the fill CTAs.
struct TubeLaunch {
    const void* kern;
    size_t smem;
    int nt, cl, teams;
    int nA;              // tubes handed to the teams (order[0, nA))
    int fill;            // single-CTA fill launch over order[nA, ntubes), 0 for none
};

// Estimated steps of every tube in a run (indexed by tube): the prescribed
// count, or min(max_steps, (t_end - t) m / CFL) with m the CFL rate of the
// tube's current state (one small kernel; synchronises the stream).
static mxe_status tube_steps(mxe_ctx* c, int max_steps, double t_end, int n_fixed,
                             std::vector<double>& steps) {
    const int n = c->ntubes;
    steps.assign(n, (double)(n_fixed > 0 ? n_fixed : max_steps));
    if (n_fixed > 0) return MXE_OK;
    std::vector<float> rate(n);
    std::vector<TubeClock> ck(n);
    tube_rates(tubes_planar(c), c->U, c->tdesc_d, n, (float)c->sp.sigma_lim, (float)c->sp.k_ws,
               c->rates_d, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(rate.data(), c->rates_d, sizeof(float) * n, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(ck.data(), c->tclk, sizeof(TubeClock) * n, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < n; ++b) {
        const double left = std::max(t_end - ck[b].t, 0.0) * (double)rate[b] / c->cfg.cfl;
        if (std::isfinite(left)) steps[b] = std::min(steps[b], std::ceil(left));
    }
    return MXE_OK;
}

// The fill launch's share: the largest tail of the work order whose estimated
// time on the fill CTAs stays within the teams' estimated time, and no tube of
// which would take longer alone.  Tubes in work order (cells[q], steps[q]);
// estimates in CTA passes over a chunk of C cells times the tube's steps: a
// team of cl CTAs spends cl * ceil(chunks / cl) CTA passes on a step, one CTA
// `chunks`.  Returns the number of tubes for the teams (the rest go to the
// fill CTAs) and the estimated time of the run, max(teams, fill).
static int plan_fill(int n, const int* cells, const double* steps, int C, int cl, int teams,
                     int fill, double* time_out) {
    std::vector<double> team(n), solo(n);
    double TA = 0.0;
    for (int q = 0; q < n; ++q) {
        const int ch = (cells[q] + C - 1) / C;
        team[q] = (double)((ch + cl - 1) / cl) * steps[q] / teams;
        solo[q] = (double)ch * steps[q];
        TA += team[q];
    }
    double TB = 0.0;
    int nA = n;
    while (fill > 0 && nA > 1) {
        const int q = nA - 1;
        const double ta = TA - team[q], tb = TB + solo[q] / fill;
        if (tb > ta || solo[q] > ta) break;
        TA = ta;
        TB = tb;
        nA = q;
    }
    if (time_out) *time_out = std::max(TA, TB);
    return nA;
}

extern "C" mxe_status mxe_batch_plan_fill(int n, const int* cells, const double* steps,
                                          int chunk, int cl, int teams, int fill, int* team_tubes,
                                          double* est_time) {
    if (n < 1 || !cells || !steps || chunk < 1 || cl < 1 || teams < 1 || fill < 0)
        return MXE_EINVAL;
    for (int q = 0; q < n; ++q)
        if (cells[q] < 1 || !(steps[q] >= 0.0) || !std::isfinite(steps[q])) return MXE_EINVAL;
    const int nA = plan_fill(n, cells, steps, chunk, cl, teams, fill, est_time);
    if (team_tubes) *team_tubes = nA;
    return MXE_OK;
}

// The division for launch L from per-tube step estimates (indexed by tube);
// sets L->nA and trims L->fill.  Without estimates (est == NULL) there is no
// fill launch.
static void tube_fill_split(const mxe_ctx* c, TubeLaunch* L, const std::vector<double>* est) {
    const int n = c->ntubes;
    L->nA = n;
    if (L->fill <= 0 || n < 2 || !est) {
        L->fill = 0;
        return;
    }
    std::vector<int> cells(n);
    std::vector<double> steps(n);
    for (int q = 0; q < n; ++q) {
        cells[q] = c->tdesc[c->order_h[q]].n;
        steps[q] = (*est)[c->order_h[q]];
    }
    const int nA = plan_fill(n, cells.data(), steps.data(), L->nt - 2, L->cl, L->teams, L->fill,
                             nullptr);
    L->nA = nA;
    L->fill = nA < n ? std::min(L->fill, n - nA) : 0;
}

static mxe_status tube_launch_shape(mxe_ctx* c, int nt, int cl, TubeLaunch* L,
                                    const std::vector<double>* est = nullptr) {
    const bool pl = tubes_planar(c);
    L->kern = tubes_mixed_kernel(pl, nt);
    L->smem = tubes_mixed_smem(pl, nt);
    L->nt = nt;
    L->cl = cl;
    int per = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, L->kern, nt, L->smem));
    int teams = 0;
    if (cl > 1) {
        cudaLaunchConfig_t lc = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        lc.blockDim = dim3(nt, 1, 1);
        lc.dynamicSmemBytes = L->smem;
        lc.gridDim = dim3(cl * c->ntubes, 1, 1);
        CK(cudaOccupancyMaxActiveClusters(&teams, L->kern, &lc));
    } else {
        teams = per * c->nsm;
    }
    if (teams < 1) return fail(c, MXE_ECUDA, "tube block shape %d x %d does not fit", nt, cl);
    L->teams = std::min(teams, c->ntubes);
    L->fill = cl > 1 && teams < c->ntubes ? per * c->nsm - cl * teams : 0;
    tube_fill_split(c, L, est);
    L->teams = std::min(L->teams, L->nA);
    return MXE_OK;
}

static cudaError_t launch_tube_grid(cudaStream_t st, const TubeLaunch& L, int cl, int nblocks,
                                    const TubeMixedArgs& a, const ParamsT<float>& p,
                                    const MixedPolicy& mp) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    lc.blockDim = dim3(L.nt, 1, 1);
    lc.gridDim = dim3(nblocks, 1, 1);
    lc.dynamicSmemBytes = L.smem;
    lc.stream = st;
    if (cl > 1) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
    }
    void* args[] = {(void*)&a, (void*)&p, (void*)&mp};
    return cudaLaunchKernelExC(&lc, L.kern, args);
}

// Queue reset + the persistent team launch on `st`, and the fill launch on
// the fill stream, forked after the reset and joined back into `st` (runtime
// calls that can be captured into a graph).  The two launches share no data
// but their tubes' disjoint state and never wait on each other.
static mxe_status launch_tubes_mixed(mxe_ctx* c, cudaStream_t st, const TubeMixedArgs& a,
                                     const TubeLaunch& L) {
    const ParamsT<float> p = fparams(c);
    const MixedPolicy mp = c->mp;
    c->lay_teams = L.teams;
    c->lay_nA = L.nA;
    c->lay_fill = L.fill;
    CK(cudaMemsetAsync(c->queue_d, 0, 2 * sizeof(int), st));
    if (L.fill > 0) {
        CK(cudaEventRecord(c->ev_fork, st));
        CK(cudaStreamWaitEvent(c->fill_stream, c->ev_fork, 0));
    }
    TubeMixedArgs aA = a;
    aA.ntubes = L.nA;
    CK(launch_tube_grid(st, L, L.cl, L.cl * L.teams, aA, p, mp));
    if (L.fill > 0) {
        TubeMixedArgs aB = a;
        aB.order = a.order + L.nA;
        aB.ntubes = a.ntubes - L.nA;
        aB.queue = a.queue + 1;
        CK(launch_tube_grid(c->fill_stream, L, 1, L.fill, aB, p, mp));
        CK(cudaEventRecord(c->ev_join, c->fill_stream));
        CK(cudaStreamWaitEvent(st, c->ev_join, 0));
    }
    return MXE_OK;
}

// Run through the cached CUDA graph [queue reset, persistent launch]; the
// graph is captured again when t_end, max_steps, the block shape or any
// launch argument changed.
static mxe_status run_tubes_mixed(mxe_ctx* c, int max_steps, double t_end, const double* dts,
                                  int ndts) {
    TubeLaunch L;
    std::vector<double> est;
    mxe_status s;
    if (dts) {                                   // prescribed steps: direct launch
        s = tube_steps(c, ndts, INFINITY, ndts, est);
        if (s == MXE_OK) s = tube_launch_shape(c, c->tune_nt, c->tune_cl, &L, &est);
        if (s == MXE_OK) s = upload_dts(c, dts, ndts);
        if (s != MXE_OK) return s;
        TubeMixedArgs a = tubes_mixed_args(c, ndts, INFINITY);
        a.dt_fixed = c->dts_d;
        a.n_fixed = ndts;
        return launch_tubes_mixed(c, c->stream, a, L);
    }
    if (!c->gexec || c->g_tend != t_end || c->g_steps != max_steps || c->g_nt != c->tune_nt ||
        c->g_cl != c->tune_cl || c->g_gen != c->gen || c->g_planar != tubes_planar(c)) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        // the team / fill division of the captured launch, from the current
        // state's step estimates
        s = tube_steps(c, max_steps, t_end, 0, est);
        if (s == MXE_OK) s = tube_launch_shape(c, c->tune_nt, c->tune_cl, &L, &est);
        if (s != MXE_OK) return s;
        TubeMixedArgs a = tubes_mixed_args(c, max_steps, t_end);
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        s = launch_tubes_mixed(c, c->cap_stream, a, L);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (s != MXE_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(c, MXE_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->gexec = nullptr;
            return fail(c, MXE_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        c->g_tend = t_end;
        c->g_steps = max_steps;
        c->g_nt = c->tune_nt;
        c->g_cl = c->tune_cl;
        c->g_gen = c->gen;
        c->g_planar = tubes_planar(c);
        c->g_lay_teams = c->lay_teams;
        c->g_lay_nA = c->lay_nA;
        c->g_lay_fill = c->lay_fill;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->lay_teams = c->g_lay_teams;
    c->lay_nA = c->g_lay_nA;
    c->lay_fill = c->g_lay_fill;
    return MXE_OK;
}

static mxe_status run_tubes(mxe_ctx* c, int max_steps, double t_end, const double* dts,
                            int ndts) {
    if (c->mixed) return run_tubes_mixed(c, max_steps, t_end, dts, ndts);
    TubeArgs a{};
    a.U = c->U;
    a.Us = c->Us;
    a.tubes = c->tdesc_d;
    a.clk = c->tclk;
    a.bc_type[0] = c->bc_type[0];
    a.bc_type[1] = c->bc_type[1];
    a.ghost = c->ghost_d;
    a.ntubes = c->ntubes;
    a.system = c->nf;
    a.integrator = c->cfg.integrator;
    a.sp = c->sp;
    a.cfl = c->cfg.cfl;
    a.t_end = t_end;
    a.max_steps = max_steps;
    if (dts) {
        mxe_status s = upload_dts(c, dts, ndts);
        if (s != MXE_OK) return s;
        a.dt_fixed = c->dts_d;
        a.n_fixed = ndts;
        a.max_steps = ndts;
    }
    if (c->nf == 5) mxe_tubes5_f64<<<c->ntubes, tubes_threads(), 0, c->stream>>>(a);
    else mxe_tubes14_f64<<<c->ntubes, tubes_threads(), 0, c->stream>>>(a);
    CK(cudaGetLastError());
    return MXE_OK;
}

static mxe_status tube_status(mxe_ctx* c, double* t0, long long* steps0) {
    std::vector<TubeClock> h(c->ntubes);
    CK(cudaMemcpyAsync(h.data(), c->tclk, sizeof(TubeClock) * c->ntubes, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (t0) *t0 = h[0].t;
    if (steps0) *steps0 = h[0].steps;
    for (int b = 0; b < c->ntubes; ++b) {
        if (h[b].status & ST_NONFINITE)
            return fail(c, MXE_ENONFINITE, "tube %d: non-finite state at t = %g", b, h[b].t);
        if (h[b].status & ST_NONPOSITIVE)
            return fail(c, MXE_EUNREALIZABLE,
                        "tube %d: a cell lost positivity (rho <= 0 or a diagonal pressure <= 0) "
                        "at t = %g", b, h[b].t);
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_step(mxe_ctx* c, int max_steps, double t_end, double* t_out,
                               int* steps_out) {
    if (!c) return MXE_EINVAL;
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    if (max_steps < 0) return fail(c, MXE_EINVAL, "max_steps < 0");
    mxe_status s = periodic_ok(c);
    if (s != MXE_OK) return s;
    if (c->tubes) {
        long long st0 = 0, st1 = 0;
        if (steps_out) {
            s = tube_status(c, nullptr, &st0);
            if (s != MXE_OK) return s;
        }
        s = run_tubes(c, max_steps, t_end, nullptr, 0);
        if (s != MXE_OK) return s;
        if (t_out || steps_out) {
            double t;
            s = tube_status(c, &t, &st1);
            if (t_out) *t_out = t;
            if (steps_out) *steps_out = (int)(st1 - st0);
            return s;
        }
        return MXE_OK;
    }
    DevClock h{};
    long long st0 = 0;
    bool want = t_out || steps_out;
    if (want) {
        s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        st0 = h.steps;
    }
    // launch in chunks; a step past t_end is a no-op on the device, and so
    // is a step whose CFL size is zero (a non-finite wave speed somewhere)
    int done = 0, chunk = 4;
    bool have = false, stalled = false;
    long long prev = -1;
    while (done < max_steps) {
        int n = std::min(chunk, max_steps - done);
        for (int i = 0; i < n; ++i) {
            s = launch_2d_step(c, t_end, 0.0);
            if (s != MXE_OK) return s;
        }
        done += n;
        if (done >= max_steps) break;
        s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        have = true;
        if (h.status & (ST_NONFINITE | ST_NONPOSITIVE)) break;
        if (!(h.t[c->slot] < t_end)) break;
        if (h.steps == prev) {                // no step advanced the clock
            stalled = true;
            break;
        }
        prev = h.steps;
        chunk = std::min(chunk * 2, 256);
    }
    if (want) {
        s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        have = true;
        if (t_out) *t_out = h.t[c->slot];
        if (steps_out) *steps_out = (int)(h.steps - st0);
        if (h.steps - st0 < done && h.t[c->slot] < t_end) stalled = true;
    }
    if (have) {
        if (h.status & ST_NONFINITE) return fail(c, MXE_ENONFINITE, "non-finite state");
        if (h.status & ST_NONPOSITIVE)
            return fail(c, MXE_EUNREALIZABLE,
                        "a cell lost positivity (rho <= 0 or a diagonal pressure <= 0) by t = %g "
                        "after %lld steps; its wave speeds are undefined", h.t[c->slot], h.steps);
        if (stalled)
            return fail(c, MXE_EUNREALIZABLE,
                        "the CFL step size collapsed to zero at t = %g after %lld steps (a wave "
                        "speed is not finite)", h.t[c->slot], h.steps);
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_step_dt(mxe_ctx* c, int n, const double* dts) {
    if (!c) return MXE_EINVAL;
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    if (n < 0 || (n > 0 && !dts)) return fail(c, MXE_EINVAL, "bad dt list");
    for (int i = 0; i < n; ++i)
        if (!(dts[i] > 0.0) || !std::isfinite(dts[i])) return fail(c, MXE_EINVAL, "dt[%d] <= 0", i);
    mxe_status s = periodic_ok(c);
    if (s != MXE_OK) return s;
    if (n == 0) return MXE_OK;
    if (c->tubes) {
        s = run_tubes(c, n, INFINITY, dts, n);
        if (s != MXE_OK) return s;
        return tube_status(c, nullptr, nullptr);
    }
    for (int i = 0; i < n; ++i) {
        s = launch_2d_step(c, INFINITY, dts[i]);
        if (s != MXE_OK) return s;
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_set_mixed_policy(mxe_ctx* c, double sigma_lo, double sigma_hi,
                                           double det_min, int resync_every) {
    if (!c) return MXE_EINVAL;
    if (!c->mixed) return fail(c, MXE_ESTATE, "context is not MXE_MIXED");
    if (!(std::isfinite(sigma_lo) && std::isfinite(sigma_hi) && std::isfinite(det_min)) ||
        resync_every < 1)
        return fail(c, MXE_EINVAL, "bad mixed-precision policy");
    c->mp = MixedPolicy{(float)sigma_lo, (float)sigma_hi, (float)det_min};
    c->resync_every = resync_every;
    ++c->gen;
    return MXE_OK;
}

extern "C" mxe_status mxe_set_stage_occupancy(mxe_ctx* c, int blocks_per_sm) {
    if (!c) return MXE_EINVAL;
    if (!c->mixed || c->tubes) return fail(c, MXE_ESTATE, "not a 2D MXE_MIXED context");
    if (blocks_per_sm != 2 && blocks_per_sm != 3)
        return fail(c, MXE_EINVAL, "blocks_per_sm must be 2 or 3");
    c->stage_occ = blocks_per_sm;
    return MXE_OK;
}

extern "C" mxe_status mxe_set_face_packing(mxe_ctx* c, int packed) {
    if (!c) return MXE_EINVAL;
    if (!c->mixed || c->tubes) return fail(c, MXE_ESTATE, "not a 2D MXE_MIXED context");
    if (packed != 0 && packed != 1) return fail(c, MXE_EINVAL, "packed must be 0 or 1");
    c->face_packed = packed;
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_run(mxe_ctx* c, int max_steps, double t_end) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes) return fail(c, MXE_ESTATE, "not a batch context");
    return mxe_step(c, max_steps, t_end, nullptr, nullptr);
}

extern "C" mxe_status mxe_batch_get_clock(mxe_ctx* c, double* t, long long* steps) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes) return fail(c, MXE_ESTATE, "not a batch context");
    std::vector<TubeClock> h(c->ntubes);
    CK(cudaMemcpyAsync(h.data(), c->tclk, sizeof(TubeClock) * c->ntubes, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < c->ntubes; ++b) {
        if (t) t[b] = h[b].t;
        if (steps) steps[b] = h[b].steps;
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_autotune(mxe_ctx* c, double t_probe, int* nt_out, int* cl_out,
                                         double* ms_out) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes || !c->mixed) return fail(c, MXE_ESTATE, "autotuning needs an MXE_MIXED 1D context");
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    if (!(t_probe > 0.0) || !std::isfinite(t_probe)) return fail(c, MXE_EINVAL, "t_probe must be > 0");
    mxe_status s = periodic_ok(c);
    if (s != MXE_OK) return s;
    // save the state and the clocks; every candidate starts from them
    std::vector<TubeClock> ck(c->ntubes);
    CK(cudaMemcpyAsync(ck.data(), c->tclk, sizeof(TubeClock) * c->ntubes, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double t0 = 0.0;
    for (const TubeClock& k : ck) t0 = std::max(t0, k.t);
    double* Usave = nullptr;
    CK(cudaMalloc(&Usave, sizeof(double) * c->nelem));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Usave, c->U, sizeof(double) * c->nelem, cudaMemcpyDeviceToDevice,
                            c->stream);
    std::vector<double> est;
    if (e == cudaSuccess && tube_steps(c, 1 << 30, t0 + t_probe, 0, est) != MXE_OK)
        e = cudaErrorUnknown;
    const int nts[2] = {128, 256}, cls[4] = {1, 2, 4, 8};
    float best = INFINITY;
    int bnt = c->tune_nt, bcl = c->tune_cl;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        for (int j = 0; j < 4 && e == cudaSuccess; ++j) {
            TubeLaunch L;
            if (tube_launch_shape(c, nts[i], cls[j], &L, &est) != MXE_OK) {
                cudaGetLastError();
                continue;                       // shape does not fit on this device
            }
            e = cudaMemcpyAsync(c->U, Usave, sizeof(double) * c->nelem, cudaMemcpyDeviceToDevice,
                                c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->tclk, ck.data(), sizeof(TubeClock) * c->ntubes,
                                    cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            if (e != cudaSuccess) break;
            TubeMixedArgs a = tubes_mixed_args(c, 1 << 30, t0 + t_probe);
            if (launch_tubes_mixed(c, c->stream, a, L) != MXE_OK) {
                cudaGetLastError();
                continue;
            }
            e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                bnt = nts[i];
                bcl = cls[j];
            }
        }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->U, Usave, sizeof(double) * c->nelem, cudaMemcpyDeviceToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->tclk, ck.data(), sizeof(TubeClock) * c->ntubes,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(Usave);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(c, MXE_ECUDA, "autotune: %s", cudaGetErrorString(e));
    if (!(best < INFINITY)) return fail(c, MXE_ECUDA, "autotune: no block shape could be launched");
    c->tune_nt = bnt;
    c->tune_cl = bcl;
    c->tuned = true;
    c->lay_nA = 0;                   // the layout of the next launch is not known yet
    if (nt_out) *nt_out = bnt;
    if (cl_out) *cl_out = bcl;
    if (ms_out) *ms_out = best;
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_get_layout(mxe_ctx* c, int* teams, int* team_tubes,
                                           int* fill_ctas) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes || !c->mixed) return fail(c, MXE_ESTATE, "layout of an MXE_MIXED 1D context only");
    if (c->lay_nA == 0) {            // nothing launched yet: the teams alone
        TubeLaunch L;
        mxe_status s = tube_launch_shape(c, c->tune_nt, c->tune_cl, &L);
        if (s != MXE_OK) return s;
        c->lay_teams = L.teams;
        c->lay_nA = L.nA;
        c->lay_fill = L.fill;
    }
    if (teams) *teams = c->lay_teams;
    if (team_tubes) *team_tubes = c->lay_nA;
    if (fill_ctas) *fill_ctas = c->lay_fill;
    return MXE_OK;
}

extern "C" mxe_status mxe_batch_set_shape(mxe_ctx* c, int nt, int cl) {
    if (!c) return MXE_EINVAL;
    if (!c->tubes || !c->mixed) return fail(c, MXE_ESTATE, "block shapes apply to MXE_MIXED 1D contexts");
    if ((nt != 128 && nt != 256) || (cl != 1 && cl != 2 && cl != 4 && cl != 8))
        return fail(c, MXE_EINVAL, "shape must be nt in {128, 256}, cl in {1, 2, 4, 8}");
    c->tune_nt = nt;
    c->tune_cl = cl;
    c->lay_nA = 0;                   // the layout of the next launch is not known yet
    return MXE_OK;
}

extern "C" mxe_status mxe_get_diagnostics(mxe_ctx* c, mxe_diag* out) {
    if (!c || !out) return MXE_EINVAL;
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    memset(out, 0, sizeof *out);
    double acc[32];
    dim3 dg = cellgrid(c, 128);
    long long nb = (long long)dg.x * dg.y;
    if (c->diag_part_n < nb) {
        cudaFree(c->diag_part);
        c->diag_part = nullptr;
        c->diag_part_n = 0;
        CK(cudaMalloc(&c->diag_part, sizeof(double) * DIAG_W * nb));
        c->diag_part_n = nb;
    }
    mxe_k_diag<<<dg, 128, 0, c->stream>>>(cellmap(c), c->nf, c->U, c->cfg.sigma_lim,
                                          c->diag_part);
    mxe_k_diag_reduce<<<1, 256, 0, c->stream>>>(c->diag_part, nb, c->accd);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(acc, c->accd, sizeof(double) * 21, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->nf; ++k) out->sums[k] = acc[k];
    out->min_sigma = acc[16];
    out->n_sigma_below_lim = (long long)acc[17];
    out->n_sigma_above_one = (long long)acc[18];
    out->n_nonpositive = (long long)acc[19];
    out->n_nonfinite = (long long)acc[20];
    if (c->tubes) {
        std::vector<TubeClock> h(c->ntubes);
        CK(cudaMemcpy(h.data(), c->tclk, sizeof(TubeClock) * c->ntubes, cudaMemcpyDeviceToHost));
        out->t = h[0].t;
        out->last_dt = h[0].last_dt;
        out->steps = h[0].steps;
        out->max_rate = h[0].rate;
        for (const TubeClock& k : h) {
            out->n_fp64_closures += (long long)k.n_face64;
            out->n_closures += (long long)k.n_face;
        }
        out->planar = (c->mixed && tubes_planar(c)) ? 1 : 0;
    } else {
        DevClock h{};
        mxe_status s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        out->t = h.t[c->slot];
        out->last_dt = h.last_dt;
        out->steps = h.steps;
        memcpy(&out->max_rate, &h.rate[c->slot], sizeof(double));
        out->n_fp64_closures = (long long)h.n_face64;
        out->n_closures = (long long)h.n_face;
        out->planar = use_planar(c) ? 1 : 0;
    }
    return MXE_OK;
}

// ---------------------------------------------------------------- dt history
extern "C" mxe_status mxe_set_dt_history(mxe_ctx* c, long long capacity) {
    if (!c) return MXE_EINVAL;
    if (c->tubes) return fail(c, MXE_ESTATE, "dt history is kept for 2D grids");
    if (capacity < 0) return fail(c, MXE_EINVAL, "capacity < 0");
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->dth);
    c->dth = nullptr;
    c->dth_cap = 0;
    if (capacity > 0) {
        CK(cudaMalloc(&c->dth, sizeof(double) * capacity));
        CK(cudaMemset(c->dth, 0, sizeof(double) * capacity));
        c->dth_cap = capacity;
    }
    return MXE_OK;
}

extern "C" mxe_status mxe_get_dt_history(mxe_ctx* c, long long n, double* out) {
    if (!c || !out) return MXE_EINVAL;
    if (n < 0 || n > c->dth_cap) return fail(c, MXE_EINVAL, "n outside the history capacity");
    if (n == 0) return MXE_OK;
    CK(cudaMemcpyAsync(out, c->dth, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MXE_OK;
}

// ---------------------------------------------------------------- adjoint
static mxe_status adjoint_ready(mxe_ctx* c) {
    if (c->tubes || c->nf != 14 || c->mixed)
        return fail(c, MXE_ESTATE, "the adjoint needs an MXE_FP64 2D 14-moment context");
    if (!c->have_state) return fail(c, MXE_ESTATE, "no state set");
    if (!use_planar(c))
        return fail(c, MXE_ESTATE, "the adjoint needs a planar state (u_z, P_xz, P_yz, q_z zero)");
    if (c->rp.implicit)
        return fail(c, MXE_ESTATE, "the adjoint covers the explicit BGK source only");
    mxe_status s = periodic_ok(c);
    if (s != MXE_OK) return s;
    const long long fs = c->g.fstride;
    if (!c->adjP) {
        CK(cudaMalloc(&c->adjP, sizeof(double) * NP * fs));
        CK(cudaMalloc(&c->adjCx, sizeof(double) * 4 * NP * c->g.ny * (long long)(c->g.nx + 1)));
        CK(cudaMalloc(&c->adjCy, sizeof(double) * 4 * NP * (long long)(c->g.ny + 1) * c->g.nx));
        CK(cudaMalloc(&c->adjA, sizeof(double) * c->nelem));
        CK(cudaMalloc(&c->adjB, sizeof(double) * c->nelem));
        CK(cudaMalloc(&c->adjG, sizeof(double) * (4 * GHOST_SLOTS * 14 + 2)));   // + tau, flag
    }
    if (c->adj_f32 && !c->adjF) CK(cudaMalloc(&c->adjF, sizeof(float) * adj_f32_floats(c->g)));
    return MXE_OK;
}

static Grid2D adj_grid(const mxe_ctx* c) {
    Grid2D g = c->g;
    for (int s = 0; s < 4; ++s) g.side[s].type = c->bc_type[s];
    return g;
}

extern "C" mxe_status mxe_adjoint_record(mxe_ctx* c, int n, const double* dts) {
    if (!c) return MXE_EINVAL;
    if (n < 1) return fail(c, MXE_EINVAL, "need n >= 1 steps");
    if (dts)
        for (int i = 0; i < n; ++i)
            if (!(dts[i] > 0.0) || !std::isfinite(dts[i]))
                return fail(c, MXE_EINVAL, "dt[%d] <= 0", i);
    mxe_status s = adjoint_ready(c);
    if (s != MXE_OK) return s;
    // dts == NULL: n steps at the CFL step size, recorded as they are taken;
    // their sizes come back through the dt history
    long long steps0 = 0;
    if (!dts) {
        DevClock h{};
        s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        steps0 = h.steps;
        if (!c->dth || steps0 + n > c->dth_cap)
            return fail(c, MXE_ESTATE, "recording CFL steps needs a dt history of at least "
                                       "%lld entries (mxe_set_dt_history)", steps0 + n);
        if (h.status & (ST_NONFINITE | ST_NONPOSITIVE))
            return fail(c, MXE_EUNREALIZABLE, "the state is not finite or not positive");
    }
    const bool rk2 = c->cfg.integrator == MXE_RK2;
    const long long need = (long long)n * (rk2 ? 2 : 1);
    if (need > c->tape_cap) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->tape);
        c->tape = nullptr;
        c->tape_cap = 0;
        CK(cudaMalloc(&c->tape, sizeof(double) * c->nelem * need));
        c->tape_cap = need;
    }
    for (int i = 0; i < n; ++i) {
        double* un = c->tape + c->nelem * (long long)(rk2 ? 2 * i : i);
        CK(cudaMemcpyAsync(un, c->U, sizeof(double) * c->nelem, cudaMemcpyDeviceToDevice,
                           c->stream));
        s = dts ? launch_2d_step(c, INFINITY, dts[i], rk2 ? un + c->nelem : nullptr, true)
                : launch_2d_step(c, INFINITY, 0.0, rk2 ? un + c->nelem : nullptr, false);
        if (s != MXE_OK) return s;
    }
    if (dts) {
        // the replay skipped the CFL rate: form it once for the final state
        DevClock* ck = c->clk;
        CK(cudaMemsetAsync(&ck->rate[c->slot], 0, sizeof(unsigned long long), c->stream));
        dim3 grid((c->g.nx + 255) / 256, c->g.ny);
        mxe_rate14_2d_planar<<<grid, 256, 0, c->stream>>>(c->U, c->g, c->sp, c->clk, c->slot);
        CK(cudaGetLastError());
        c->tape_dt.assign(dts, dts + n);
    } else {
        DevClock h{};
        s = read_clock_2d(c, &h);
        if (s != MXE_OK) return s;
        if (h.status & ST_NONFINITE) return fail(c, MXE_ENONFINITE, "non-finite state");
        if (h.status & ST_NONPOSITIVE)
            return fail(c, MXE_EUNREALIZABLE, "a cell lost positivity while recording");
        if (h.steps - steps0 != n)
            return fail(c, MXE_EUNREALIZABLE, "the CFL step size collapsed to zero while "
                                              "recording (%lld of %d steps)", h.steps - steps0, n);
        c->tape_dt.resize(n);
        CK(cudaMemcpy(c->tape_dt.data(), c->dth + steps0, sizeof(double) * n,
                      cudaMemcpyDeviceToHost));
    }
    c->tape_n = n;
    return MXE_OK;
}

extern "C" mxe_status mxe_adjoint_run(mxe_ctx* c, double* ubar, int on_device, double* gbar,
                                      double* taubar) {
    if (!c) return MXE_EINVAL;
    if (!ubar) return fail(c, MXE_EINVAL, "ubar is NULL");
    mxe_status s = adjoint_ready(c);
    if (s != MXE_OK) return s;
    if (c->tape_n < 1) return fail(c, MXE_ESTATE, "no recorded steps");
    const size_t bytes = sizeof(double) * 14 * c->ncell;
    const double* src = ubar;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->stage, ubar, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->stage;
    }
    const Grid2D g = adj_grid(c);
    const dim3 pg((g.nx + 127) / 128, g.ny);
    CK(cudaMemsetAsync(c->adjA, 0, sizeof(double) * c->nelem, c->stream));
    mxe_adj_pack<<<pg, 128, 0, c->stream>>>(src, c->adjA, g, 1, nullptr);
    CK(cudaMemsetAsync(c->adjG, 0, sizeof(double) * (4 * GHOST_SLOTS * 14 + 2), c->stream));
    double* gb = c->adjG;
    double* tb = c->adjG + 4 * GHOST_SLOTS * 14;
    unsigned long long* nonfinite = (unsigned long long*)(c->adjG + 4 * GHOST_SLOTS * 14 + 1);
    const ParamsT<double> p = make_params<double>(c->sp, c->rp);
    const bool rk2 = c->cfg.integrator == MXE_RK2;
    for (int i = c->tape_n - 1; i >= 0; --i) {
        const double dt = c->tape_dt[i];
        const double* un = c->tape + c->nelem * (long long)(rk2 ? 2 * i : i);
        cudaError_t e;
        if (rk2) {
            // U^{n+1} = U^n + dt L(U*): B = dt L'(U*)^T A
            e = adj_stage(un + c->nelem, c->adjA, dt, nullptr, nullptr, c->adjB, c->adjP,
                          c->adjCx, c->adjCy, gb, tb, g, p, c->adj_f32, c->adjF,
                          c->adj_frozen, c->stream);
            // U* = U^n + dt/2 L(U^n): A = A + B + dt/2 L'(U^n)^T B
            if (e == cudaSuccess)
                e = adj_stage(un, c->adjB, 0.5 * dt, c->adjA, c->adjB, c->adjA, c->adjP,
                              c->adjCx, c->adjCy, gb, tb, g, p, c->adj_f32, c->adjF,
                          c->adj_frozen, c->stream);
        } else {
            e = adj_stage(un, c->adjA, dt, c->adjA, nullptr, c->adjA, c->adjP, c->adjCx,
                          c->adjCy, gb, tb, g, p, c->adj_f32, c->adjF,
                          c->adj_frozen, c->stream);
        }
        if (e != cudaSuccess) return fail(c, MXE_ECUDA, "adjoint stage: %s", cudaGetErrorString(e));
    }
    double* dst = on_device ? ubar : c->stage;
    mxe_adj_pack<<<pg, 128, 0, c->stream>>>(dst, c->adjA, g, 0, nonfinite);
    CK(cudaGetLastError());
    if (!on_device)
        CK(cudaMemcpyAsync(ubar, c->stage, bytes, cudaMemcpyDeviceToHost, c->stream));
    double hg[4 * GHOST_SLOTS * 14 + 2];
    CK(cudaMemcpyAsync(hg, c->adjG, sizeof hg, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    bool finite = std::isfinite(hg[4 * GHOST_SLOTS * 14]);
    for (int k = 0; k < 4 * GHOST_SLOTS * 14; ++k) finite = finite && std::isfinite(hg[k]);
    unsigned long long flag;
    std::memcpy(&flag, &hg[4 * GHOST_SLOTS * 14 + 1], sizeof flag);
    if (flag || !finite)     // gbar, taubar untouched: the caller may sweep again
        return fail(c, MXE_ENONFINITE, "the adjoint left the finite range");
    if (gbar)
        for (int k = 0; k < 4 * GHOST_SLOTS * 14; ++k) gbar[k] += hg[k];
    if (taubar) *taubar += hg[4 * GHOST_SLOTS * 14];
    return MXE_OK;
}

extern "C" mxe_status mxe_adjoint_residual(mxe_ctx* c, const double* U, const double* V,
                                           double* out, int on_device, double* gbar,
                                           double* taubar) {
    if (!c) return MXE_EINVAL;
    if (!U || !V || !out) return fail(c, MXE_EINVAL, "NULL array");
    mxe_status s = adjoint_ready(c);
    if (s != MXE_OK) return s;
    const size_t bytes = sizeof(double) * 14 * c->ncell;
    const Grid2D g = adj_grid(c);
    const dim3 pg((g.nx + 127) / 128, g.ny);
    // U and V staged in the adjoint buffers, the result in a temporary
    double* Up = c->adjB;
    double* Vp = c->adjA;
    const double* su = U;
    const double* sv = V;
    double* tmpU = nullptr;
    if (!on_device) {
        CK(cudaMalloc(&tmpU, 2 * bytes));
        CK(cudaMemcpyAsync(tmpU, U, bytes, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(tmpU + 14 * c->ncell, V, bytes, cudaMemcpyHostToDevice, c->stream));
        su = tmpU;
        sv = tmpU + 14 * c->ncell;
    }
    CK(cudaMemsetAsync(Up, 0, sizeof(double) * c->nelem, c->stream));
    CK(cudaMemsetAsync(Vp, 0, sizeof(double) * c->nelem, c->stream));
    mxe_adj_pack<<<pg, 128, 0, c->stream>>>(su, Up, g, 1, nullptr);
    mxe_adj_pack<<<pg, 128, 0, c->stream>>>(sv, Vp, g, 1, nullptr);
    CK(cudaMemsetAsync(c->adjG, 0, sizeof(double) * (4 * GHOST_SLOTS * 14 + 2), c->stream));
    const ParamsT<double> p = make_params<double>(c->sp, c->rp);
    double* Op = nullptr;
    CK(cudaMalloc(&Op, sizeof(double) * c->nelem));
    cudaError_t e = adj_stage(Up, Vp, 1.0, nullptr, nullptr, Op, c->adjP, c->adjCx, c->adjCy,
                              c->adjG, c->adjG + 4 * GHOST_SLOTS * 14, g, p, c->adj_f32,
                              c->adjF, c->adj_frozen, c->stream);
    if (e == cudaSuccess) {
        double* dst = on_device ? out : tmpU;
        mxe_adj_pack<<<pg, 128, 0, c->stream>>>(dst, Op, g, 0, nullptr);
        e = cudaGetLastError();
        if (e == cudaSuccess && !on_device)
            e = cudaMemcpyAsync(out, tmpU, bytes, cudaMemcpyDeviceToHost, c->stream);
    }
    double hg[4 * GHOST_SLOTS * 14 + 1];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg, c->adjG, sizeof hg, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(Op);
    cudaFree(tmpU);
    if (e != cudaSuccess) return fail(c, MXE_ECUDA, "adjoint residual: %s", cudaGetErrorString(e));
    if (gbar)
        for (int k = 0; k < 4 * GHOST_SLOTS * 14; ++k) gbar[k] += hg[k];
    if (taubar) *taubar += hg[4 * GHOST_SLOTS * 14];
    return MXE_OK;
}

extern "C" mxe_status mxe_set_adjoint_precision(mxe_ctx* c, int precision) {
    if (!c) return MXE_EINVAL;
    if (precision != MXE_FP64 && precision != MXE_MIXED)
        return fail(c, MXE_EINVAL, "precision must be MXE_FP64 or MXE_MIXED");
    c->adj_f32 = precision == MXE_MIXED;
    return MXE_OK;
}

extern "C" mxe_status mxe_set_adjoint_limiter(mxe_ctx* c, int frozen) {
    if (!c) return MXE_EINVAL;
    if (frozen != 0 && frozen != 1) return fail(c, MXE_EINVAL, "frozen must be 0 or 1");
    c->adj_frozen = frozen == 1;
    return MXE_OK;
}
