// mxe_internal.h -- host/device shared descriptors of the CUDA library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mxe_physics.cuh"

namespace mxe {

constexpr int MAX_SPANS = 4;
constexpr int GHOST_SLOTS = 1 + MAX_SPANS;     // base state + slots

// status bits (device status word)
constexpr unsigned ST_NONFINITE = 1u;
constexpr unsigned ST_NONPOSITIVE = 2u;

// Boundary side: base type and Dirichlet slots as inclusive index ranges of
// the cells along the side (computed on the host from [lo, hi]).
struct SideDesc {
    int type;                 // 0 transmissive, 1 periodic, 2 dirichlet
    int nspans;
    int lo[MAX_SPANS], hi[MAX_SPANS];
};

// Clock of one grid: triple-buffered time and CFL rate so that a step
// reads slot s, accumulates slot s+1 and clears slot s+2 (mod 3).
struct DevClock {
    double t[3];
    unsigned long long rate[3];     // bit pattern of a non-negative double
    double last_dt;
    long long steps;
    unsigned status;
    unsigned pad;
    unsigned long long n_face, n_face64;   // mixed-precision counters
};

struct Grid2D {
    int nx, ny, pitch;              // pitch: row stride in elements
    long long fstride;              // field stride (ny * pitch)
    double dx, dy;
    double idx, idy;                // 1/dx, 1/dy
    SideDesc side[4];
    const double* ghost;            // [4][GHOST_SLOTS][14] primitive ghost states
};

struct Stage2DArgs {
    const double* Uin;              // FP64 path: state the residual is evaluated on
    const double* Ubase;            // U^n
    double* Uout;
    const float* Win;               // mixed path: FP32 primitive stencil state
    float* Wout;                    // mixed path: FP32 primitives of the result
    const float* Wbase;             // mixed path: FP32 primitives of U^n
    Grid2D g;
    SchemeParams sp;
    RelaxParams rp;
    double cfl, t_end, coef, dt_fixed;
    float idxf, idyf;               // 1/dx, 1/dy for the FP32 path
    int slot, final_stage;
    DevClock* clk;
    double* dt_hist;                // optional: dt of step s at dt_hist[s] (s < dt_hist_cap)
    long long dt_hist_cap;
    int skip_rate;                  // FP64 final stage: no CFL rate (prescribed dt follows)
    int resync;                     // mixed final stage: W^{n+1} = prim(U^{n+1}) in FP64
};

// ---- 1D tubes ----
struct TubeDesc {
    long long off;                  // element offset of the tube's field 0
    long long coff;                 // cell offset (cells of the tubes before it)
    int n;                          // cells
    int pad;
    double dx;
    RelaxParams rp;
};

struct TubeClock {
    double t, last_dt, rate;
    long long steps;
    unsigned status;
    unsigned pad;
    unsigned long long n_face, n_face64;
};

struct TubeArgs {
    double* U;                      // all tubes, FP64 conserved
    double* Us;                     // stage buffer (same layout)
    const TubeDesc* tubes;
    TubeClock* clk;
    int bc_type[2];                 // xlo, xhi: 0 transmissive, 1 periodic, 2 dirichlet
    const double* ghost;            // [2][14] primitive ghost states (round-tripped)
    int ntubes, system;
    int integrator;                 // 0 FE, 1 RK2
    SchemeParams sp;
    double cfl, t_end;
    int max_steps;
    const double* dt_fixed;         // NULL, or n_fixed prescribed steps
    int n_fixed;
};

// Mixed-precision batched tubes (one persistent launch, work queue)
struct TubeMixedArgs {
    double* U;                      // all tubes, FP64 conserved (14 fields per tube)
    float* W;                       // FP32 primitives, NF fields per tube at NF * coff
    float* Ws;                      // FP32 primitives of the stage state (same layout)
    const TubeDesc* tubes;
    const int* order;               // tube indices in the order they are handed out
    int* queue;                     // next position in `order` (zero at launch)
    TubeClock* clk;
    int bc_type[2];
    const double* ghost;            // [2][14] primitive ghost states
    int ntubes;
    int integrator;                 // 0 FE, 1 RK2
    int max_steps;
    int resync_every;               // W = prim(U) in FP64 every this many steps
    double cfl, t_end;
    double sl64, kw64;              // sigma_lim and k for the FP64 re-evaluation
    const double* dt_fixed;         // NULL, or n_fixed prescribed steps
    int n_fixed;
};

// Addressing of the cells of a context: a pitched 2D grid, or concatenated
// 1D tubes (per tube: fields of n cells one after another).
struct CellMap {
    int mode;                   // 0 grid, 1 tubes
    int nx, ny, pitch;
    long long fstride;
    const TubeDesc* tubes;
    int ntubes;
    int nf;
};

}  // namespace mxe
