// engine.h -- host-side launch interface between the C ABI (capi.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "pic_internal.cuh"

namespace pic {

// Device buffers and launch geometry of the grid (field-solve) kernels.
struct FieldArgs {
    const GridDev* grids;   // [ngrids]
    const int* blk_grid;    // [nblk] simulation of each field block
    int ngrids, nblk;
    long long ntot;         // total cells over all simulations
    double* F;              // 6 * ntot: Ex Ey Ez Bx By Bz (component-major)
    const double* J64;      // 3 * ntot, FP64 current (FP64 particle path) or nullptr
    const long long* Jfix;  // 3 * ntot, fixed-point current (MIXED32 particle path) or nullptr
    float* F32;             // 6 * ntot FP32 copy of the fields for MIXED32 gathers, or nullptr
    double* Fn;             // 6 * ntot FP64 node-averaged fields (FP64 with PIC_GATHER_NODAL) or nullptr
    int any_nodal;          // some simulation gathers node-averaged fields
    int coop;               // the cooperative solve follows (it reads the FP32 copy of r only)
    int quads;              // every simulation's nx is a multiple of 4: the MIXED32 E and B
                            // updates take quads of cells with vector loads
    double *x, *r, *p, *q;  // 3 * ntot each: dB (solution), residual, direction, A p
    CgState* cg;            // [ngrids]
    double* part;           // 4 * nblk block partials
    unsigned int* done;     // [ngrids] block-completion counters
    DevStatus* st;
    cudaGraphConditionalHandle cond;  // WHILE-node handle of the PCG loop
    int use_cond;                      // 1 when running inside the captured step graph
    // mixed-precision refinement (MIXED32 only; nullptr otherwise)
    double* b;                         // 3 * ntot right-hand side of Eq. (7)
    float *r32, *p32, *q32, *e32;      // 3 * ntot each, inner FP32 CG vectors
    float *r32b, *z32;                 // 3 * ntot each: second residual buffer, z = M r
    cudaGraphConditionalHandle cond_in;  // WHILE-node handle of the inner loop
};

// Mixed-precision PCG pieces (see fields.cu): inner start, one inner iteration, and the
// FP64 refinement x += e, r = b - A x.
void launch_mp_inner_begin(const FieldArgs& a, cudaStream_t s);
void launch_mp_inner_iteration(const FieldArgs& a, cudaStream_t s);
void launch_mp_refine(const FieldArgs& a, cudaStream_t s);

// Per-step prologue (deferred stop, step counter, accumulators) and epilogue.
void launch_step_begin(const FieldArgs& a, cudaStream_t s);
void launch_step_end(const FieldArgs& a, cudaStream_t s);
// b of Eq. (7), initial residual, energies at time level n.
void launch_rhs(const FieldArgs& a, cudaStream_t s);
// r = b - A x for an initial guess x written after launch_rhs (the learned guess).
void launch_guess_residual(const FieldArgs& a, cudaStream_t s);
// The same in FP32 for the cooperative solve, from the guess's FP32 copy in a.e32 into
// a.r32 (which holds the FP32 copy of b): the first inner solve needs no more.
void launch_guess_residual32(const FieldArgs& a, cudaStream_t s);
// One PCG iteration: A-product and direction update, then solution/residual update.
void launch_cg_iteration(const FieldArgs& a, cudaStream_t s);
// E, B from Eqs. (5)-(6) with dB; FP32 copies when a.F32 is set.
void launch_field_update(const FieldArgs& a, cudaStream_t s);
// Explicit FDTD field step, Eqs. (3)-(4) (PIC_EXPLICIT): three kernels, no solve.
void launch_explicit_fields(const FieldArgs& a, cudaStream_t s);
// Node-averaged gather copies (PIC_GATHER_NODAL): into F32 (MIXED32) or Fn (FP64).
void launch_nodal(const FieldArgs& a, cudaStream_t s);
// FP32 copy of the FP64 fields (after pic_set_fields / init), node-averaged where asked.
void launch_fields_to_f32(const FieldArgs& a, cudaStream_t s);

// The MIXED32 solve as one cooperative persistent kernel (solve_coop.cu), used when the
// device supports cooperative launches and a handle holds at most kCoopMaxGrids
// simulations; otherwise the WHILE-node solve above runs.
constexpr int kCoopMaxGrids = 64;
struct CoopSolve {
    int2* gchunk = nullptr;       // per simulation: first chunk, chunk count
    int* chunk_grid = nullptr;    // per chunk: simulation
    int* tile_grid = nullptr;     // per 32 x 64 Chebyshev tile: simulation
    int2* tile_xy = nullptr;      // per tile: first cell (x, y)
    double* part = nullptr;       // 2 buffers x 2 values x nchunks chunk partial sums
    unsigned int* bar = nullptr;  // grid barrier: arrivals, generation
    int nchunks = 0, nblocks = 0, ngrids = 0, ntiles = 0, cg_inner = 0;
    int cheb = 0;                 // some simulation takes the Chebyshev inner solve
};
// PIC_OK, PIC_EINVAL (not applicable: keep the WHILE-node solve) or PIC_ECUDA. cg_inner:
// the inner solve is always the CG (PIC_CG_INNER).
int coop_create(CoopSolve* cs, const GridDev* hgrids, int ngrids, bool cg_inner, std::string& err);
// Dynamic shared memory of the cooperative solve's launch.
size_t coop_smem(const CoopSolve& cs);
void coop_free(CoopSolve* cs);
// The solve after launch_rhs (and a learned guess): needs a.b, a.x, a.r and the FP32 vectors.
cudaError_t launch_mp_coop(const CoopSolve& cs, const FieldArgs& a, cudaStream_t s);

// Arguments of the FP64 particle kernel.
struct Fp64PushArgs {
    const GridDev* grids;
    const SegDev* segs;
    const int* blk_seg;   // [nblk] segment of each block
    int nblk;
    int nsegs;
    long long ntot;
    const double* F;      // 6 * ntot
    double* J;            // 3 * ntot
    double *x, *y, *ux, *uy, *uz;  // positions in grid units (x/dx, y/dy)
    CgState* cg;          // kinetic energy accumulates into cg[g].uk
    DevStatus* st;
};
// One launch over all blocks of the table; every segment must have shape order `order`.
void launch_push_fp64(const Fp64PushArgs& a, int order, cudaStream_t s);

// The moving injector's pairs of the current step for the FP64 particle arrays (one
// simulation; segment counts grow on the device).
struct Fp64InjectArgs {
    const GridDev* grids;
    SegDev* segs;          // [2], count incremented
    long long cap[2];      // allocated slots per species
    double *x[2], *y[2], *ux[2], *uy[2], *uz[2];
    DevStatus* st;
    int ny;
    long long kmax;        // most pairs per row in one step
};
void launch_inject_fp64(const Fp64InjectArgs& a, cudaStream_t s);

// Diagnostics of FP64 particles (positions in grid units): rho += node charge density of
// n particles of charge density q each (one simulation's nx * ny array; G by value), and
// out[0..2] += w * sum of the momenta.
void launch_rho_fp64(const GridDev& G, const double* x, const double* y, long long n, double q, double* rho,
                     cudaStream_t s);
void launch_momentum_fp64(const double* ux, const double* uy, const double* uz, long long n, double w,
                          double* out, cudaStream_t s);

// Amplitude spectrum |F^(p, q)| / (nx ny) of an (ny, nx) FP64 grid quantity F (device)
// into out (device), both in the fields' layout (spectrum.cu).
int spectrum_2d(const double* F, int nx, int ny, double* out, cudaStream_t st, std::string& err);

}  // namespace pic
