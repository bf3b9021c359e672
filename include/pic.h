/*
 * pic.h -- C ABI of the GB300 implicit-FDTD particle-in-cell library.
 *
 * The library advances 2D electromagnetic PIC simulations of relativistic pair
 * plasmas with the particle cycle of Ikeya & Matsumoto, "Stability Property of
 * Numerical Cherenkov Radiation and its Application to Relativistic Shock
 * Simulations" (PASJ 2015, arXiv:1412.2480):
 *   - momentum-conserving field gather (Sec. 1, Sec. 3) at shape order 1, 2 or 3;
 *   - relativistic Buneman-Boris push (the paper gives no pusher; standard scheme);
 *   - density-decomposition (Esirkepov) charge-conserving current deposit (Sec. 1, 3);
 *   - implicit theta-FDTD Maxwell update, Eqs. (5)-(6), with the elliptic equation
 *     Eq. (7) for dB = B^{n+1} - B^n solved by preconditioned conjugate gradient
 *     (or, with PIC_EXPLICIT, the explicit FDTD update of Eqs. (3)-(4)).
 * Around it: on-demand diagnostics (densities, conservation moments, Fourier spectra
 * and the resonance line of Eq. 17), checkpoints, batches of simulations per handle,
 * and a learned initial guess for the solve.
 *
 * Units: Gaussian, c = 1. Lengths in physical units with cell sizes dx, dy; the time
 * step is dt = cfl * dx (CFL number sigma = c dt / dx, Sec. 3.1). Species 0 are
 * positrons (q/m = +1), species 1 electrons (q/m = -1); each macro-particle carries
 * charge +-w and mass w, with w fixed by the plasma frequency in the flow frame
 * (Sec. 4): omega_pe^2 = 4 pi n q^2 / (m gamma0), n = ppc/(dx dy), omega_pe = 1/skin_depth.
 *
 * Grid storage (every grid quantity, nx*ny values, index k = j*nx + i) follows the
 * 2D Yee arrangement (Sec. 2, Fig. 1): Ez, Jz, rho at (i, j); Ex, Jx, By at (i+1/2, j);
 * Ey, Jy, Bx at (i, j+1/2); Bz at (i+1/2, j+1/2). Boundaries are periodic in y, and in x
 * periodic or conducting, reflecting walls (PIC_BC_WALLS).
 *
 * Conventions for every call:
 *   - return value PIC_OK (0) or a negative PIC_E* code; nothing aborts or exits;
 *     pic_last_error() gives a message for the last failure on that handle;
 *   - pointers passed in may be host or device memory (CUDA unified addressing
 *     decides); the library copies and never keeps a caller pointer;
 *   - the handle owns all device memory it allocates; pic_free releases it;
 *   - a handle is not thread-safe; calls on one handle must not overlap.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

/* ---- return codes ---- */
#define PIC_OK 0
#define PIC_EINVAL (-1)      /* invalid argument or parameter */
#define PIC_ENOMEM (-2)      /* device or host allocation failed */
#define PIC_ECUDA (-3)       /* a CUDA call failed (message has the CUDA error) */
#define PIC_ECG_NOCONV (-4)  /* PCG reached cg_max_iter before cg_rtol */
#define PIC_ECFL (-5)        /* a particle moved one cell or more in one step */
#define PIC_ENAN (-6)        /* a non-finite particle momentum or position appeared */
#define PIC_ETIMEOUT (-7)    /* a bounded wait inside a kernel gave up (see pic_set_wait_limit) */
#define PIC_ESTATE (-8)      /* call not valid in the handle's current state */

/* ---- precision of the particle half (the field solve is always FP64) ----
 * PIC_MIXED32 runs are bit-for-bit reproducible: the same inputs and parameters give the
 * same fields, currents and particle sets on every run, alone or inside a batch, whatever
 * the order particles are stored in and whichever of them overflow their bins (the
 * current is summed in fixed point). PIC_FP64 sums its current with FP64 atomics and
 * reproduces a run to rounding only. */
#define PIC_FP64 0    /* positions, momenta, gather, push and deposit in FP64 */
#define PIC_MIXED32 1 /* int cell + FP32 offset, FP32 momenta, FP32 gather/push/deposit */

/* ---- initial guess of the PCG solve of Eq. (7) ---- */
#define PIC_WS_ZERO 0 /* dB_0 = 0 */
#define PIC_WS_PREV 1 /* dB_0 = the previous step's dB */
#define PIC_WS_LEARNED 2 /* dB_0 from the learned network set by pic_set_cnn (PIC_MIXED32 only) */

/* ---- flags ---- */
#define PIC_NO_DEPOSIT 1   /* test-particle mode: particles feel the fields, J = 0 */
#define PIC_NO_GRAPH 2     /* launch kernels directly instead of a captured CUDA graph */
#define PIC_NO_COOP 4      /* PIC_MIXED32: run the PCG loop as graph-driven kernel launches instead
                              of one cooperative persistent kernel (same arithmetic) */
#define PIC_EXPLICIT 8     /* explicit FDTD field update, Eqs. (3)-(4), instead of the implicit
                              theta scheme (theta and the PCG settings are not used); B is kept
                              at integer time levels by two half steps of Eq. (3) around Eq. (4).
                              Needs (c dt)^2 (1/dx^2 + 1/dy^2) <= 1 (Courant limit, Eq. 16) */
#define PIC_GATHER_NODAL 16 /* the alternative reading of the momentum-conserving gather: E and B
                              are first averaged from their staggered lattices to the nodes (Ex, By
                              over two x-neighbours, Ey, Bx over two y-neighbours, Bz over four
                              cells) and every component is then gathered with the node weights
                              of the charge deposit; periodic boundaries only */
#define PIC_CG_INNER 32    /* PIC_MIXED32 cooperative solve: the FP32 inner solve of every
                              refinement by preconditioned CG. Without it the inner solve is a
                              Chebyshev iteration of at most 13 steps on A's spectrum interval,
                              tile by tile (no grid-wide step), with the refinement's residual
                              in FP32-pair arithmetic: sigma = c0 / (2 (cx + cy)) >= 5/4 for
                              every theta in [1/2, 1] and CFL in (0, 1], so 13 steps always
                              reduce the error by 4e3 at least. A simulation asking for
                              cg_rtol < 1e-13 keeps the CG (the pairs resolve about 1e-14 of
                              ||b||). The same FP64-class test ||r|| <= rtol ||b|| ends the
                              solve either way. NO_GRAPH, NO_COOP, EXPLICIT and CG_INNER are
                              per handle: every simulation of a batch gives the same. */

/* ---- x boundaries ----
 * PIC_BC_WALLS closes the box in x with two perfectly conducting walls at x = 0 and
 * x = nx dx that reflect particles specularly (x -> -x, ux -> -ux), as the shock
 * configuration does at its reflecting wall (Sec. 4). Fields take the images of a
 * perfect conductor: Ey = Ez = Bx = 0 on the wall nodes (the x = 0 column; the x = nx
 * nodes are not stored), Ex, By, Bz even about the walls; Eq. (7) then has Dirichlet
 * rows for Bx and Neumann rows for By, Bz and stays symmetric positive definite. A
 * particle's deposit folds back at a wall as its mirror image's (Jx odd, Jy, Jz even);
 * the conductor carries the current of its wall nodes. Loaded positions must lie in
 * [0, nx dx). pic_set_fields zeroes Ey, Ez, Bx on the wall column. With PIC_WS_LEARNED
 * the network's stencil is applied to the conductor's images of the right-hand side
 * near the walls (the network itself is trained on periodic grids). */
#define PIC_BC_PERIODIC 0
#define PIC_BC_WALLS 1

/* ---- the moving injector (PIC_BC_WALLS, inject_x0 >= 0) ----
 * The shock set-up feeds the wall at x = 0 with a pair beam from a plane that starts at
 * x_f(0) = inject_x0 (cells) and moves toward +x at c: x_f(n) = inject_x0 + n cfl. The
 * paper injects from a fixed boundary (Sec. 4); a plane moving at c keeps every
 * injected and reflected particle behind it, so no particle ever leaves the box. At the
 * end of step n (n = steps completed before it, counted from pic_init) the slab
 * [x_f(n+1) - (1 + v) cfl, x_f(n+1)) of every row j, which the beam has uncovered by
 * moving at -v while the plane moved at +c, receives N_n = floor(ppc w (n+1)) -
 * floor(ppc w n) co-located pairs, w = (1 + v) cfl the slab width: the beam's density
 * ppc per cell per species over time. Pair k of row j at step n sits at
 * x = x_f(n+1) - w U0, y = j + U1; species s gets rest-frame momenta u_th (z0, z1, z2)
 * from Box-Muller pairs (U2, U3) and (U4, U5), boosted toward -x: ux = -gamma0
 * (u_th z0 + beta0 gamma'), uy = u_th z1, uz = u_th z2, gamma' = sqrt(1 + u_th^2 |z|^2).
 * U_d = ((h >> 11) + 1/2) 2^-53, h = splitmix64 (Steele, Lea & Flood 2014) of the counter
 * seed K0 + n K1 + j K2 + k K3 + s K4 + d (mod 2^64), with K0..K4 = 0xD1B54A32D192ED03,
 * 0xABC98388FB8FAC03, 0x8CB92BA72F3D8DD7, 0x9E3779B97F4A7C15, 0xC2B2AE3D27D4EB4F
 * (positions use s = 0). Injection stops once x_f(n+1) > nx. The fields ahead of the
 * plane are whatever the caller set (a uniform Bz and the beam's motional Ey make a
 * static vacuum solution). */

/* ---- grid quantity ids for pic_fields / pic_set_fields ---- */
#define PIC_EX 0
#define PIC_EY 1
#define PIC_EZ 2
#define PIC_BX 3
#define PIC_BY 4
#define PIC_BZ 5
#define PIC_JX 6 /* J^{n+1/2} of the last step */
#define PIC_JY 7
#define PIC_JZ 8
#define PIC_DBX 9 /* dB of the last step's solve (x, y, z) */
#define PIC_DBY 10
#define PIC_DBZ 11
#define PIC_RHSX 12 /* right-hand side b of Eq. (7) of the last step (PIC_MIXED32 only) */
#define PIC_RHSY 13
#define PIC_RHSZ 14
#define PIC_RHO 15  /* node charge density of the current particles (computed on demand) */
#define PIC_DENSITY_P 16  /* positron number density (macro-particles per unit area) on the nodes,
                             deposited with the particle shape; ppc/(dx dy) in a uniform plasma */
#define PIC_DENSITY_E 17  /* electron number density, likewise */

typedef struct pic_params {
    int32_t nx, ny;        /* cells (Sec. 3: 128 x 128; Sec. 4: 5650 x 990); >= 8 each */
    double dx, dy;         /* cell size, default 1 */
    double cfl;            /* CFL number sigma = c dt / dx (Sec. 3.1), 0 < cfl <= 1 */
    double theta;          /* implicitness factor of Eqs. (5)-(6), 0.5 <= theta <= 1 */
    int32_t shape_order;   /* particle shape order 1, 2 or 3 (Sec. 3.3) */
    double gamma0;         /* drift Lorentz factor of the flow (Sec. 3) */
    int32_t ppc;           /* macro-particles per cell per species (sets w and capacity) */
    double skin_depth;     /* c / omega_pe in length units (Sec. 4 definition), default 10 */
    int32_t precision;     /* PIC_FP64 or PIC_MIXED32 */
    double cg_rtol;        /* stop when ||r||_2 <= cg_rtol ||b||_2, default 1e-10 */
    int32_t cg_max_iter;   /* default 200 */
    int32_t warm_start;    /* PIC_WS_ZERO, PIC_WS_PREV or PIC_WS_LEARNED */
    int32_t flags;         /* PIC_NO_DEPOSIT | PIC_NO_GRAPH | PIC_NO_COOP | PIC_EXPLICIT |
                              PIC_GATHER_NODAL */
    int32_t tile_x, tile_y;/* MIXED32 tile size in cells; 0 = chosen by the library */
    double bin_slack;      /* MIXED32 bin capacity factor over ppc * tile cells; 0 = 1.25 */
    int32_t bc_x;          /* PIC_BC_PERIODIC or PIC_BC_WALLS (x boundaries; y is periodic) */
    double inject_x0;      /* PIC_BC_WALLS: start of the moving injector in cells (< 0: none) */
    double u_th;           /* injector: rest-frame thermal momentum spread (units of c) */
    uint64_t seed;         /* injector: seed of its counter-based random numbers */
} pic_params;

typedef struct pic_moments_t {
    int64_t step;            /* completed steps */
    double time;             /* step * dt */
    double U_E, U_B;         /* field energies sum |E|^2 dx dy / 8 pi, same for B (at step n) */
    double U_K;              /* kinetic energy sum w (gamma - 1) with u^{n-1/2} of the last step */
    double macro_weight;     /* w */
    int64_t n_particles[2];  /* live macro-particles per species */
    int32_t cg_iters_last;   /* PCG iterations of the last step */
    int32_t cg_iters_max;    /* largest PCG iteration count since the last pic_moments */
    int64_t cg_iters_total;  /* all PCG iterations so far */
    double cg_rel_resid;     /* ||r|| / ||b|| at the end of the last solve */
    int64_t cfl_violations;  /* moves of one cell or more seen so far (should stay 0; handle-wide) */
    int64_t overflow_moves;  /* MIXED32: particles routed through the overflow path so far (handle-wide) */
    int64_t rebins;          /* MIXED32: full re-sorts performed so far */
    int64_t cg_refinements;  /* MIXED32: FP64 residual refinements (outer PCG iterations) so far */
    int64_t loop_iters;      /* handle-wide: CG iterations the PCG loop ran (in a batch, as many
                                per step as its slowest simulation needed) */
    int64_t loop_refinements;/* handle-wide, MIXED32: FP64 refinements the PCG loop ran */
    int64_t kernel_launches; /* handle-wide: kernels of this library launched by pic_step and
                                pic_profile so far (the PCG loop's included) */
} pic_moments_t;

typedef struct pic_sim pic_sim;

/* Fill *p with the defaults above (64 x 64, dx = dy = 1, cfl 1, theta 0.5, order 1,
 * gamma0 20, ppc 8, skin_depth 10, FP64, rtol 1e-10, 200 iterations, zero warm start). */
PIC_API void pic_params_default(pic_params* p);

/* Create one simulation on the current CUDA device. Validates *p (PIC_EINVAL with a
 * message if out of range), allocates all device memory, zeroes the fields. The new
 * handle is written to *out; the caller releases it with pic_free. On failure *out is
 * NULL and the last-error message is available through pic_last_error(NULL). */
PIC_API int pic_init(const pic_params* p, pic_sim** out);

/* ---- batched parameter scan ----------------------------------------------------------
 * One handle can hold n independent simulations, each with its own grid size, cell
 * size, CFL number, theta, shape order, gamma0, ppc, skin depth, PCG settings and tile
 * shape (the paper's scan over sigma, theta and shape order, Sec. 3.2-3.3). pic_step
 * advances all of them together: every kernel of the step covers every simulation, the
 * particle tiles of each shape order are one persistent launch whose CTAs take tiles from
 * a device work counter (largest first), and the PCG loop runs until the last simulation
 * has converged, each simulation stopping its own iterations at its own tolerance.
 *
 * pic_init_batch: like pic_init for the n parameter sets p[0..n), 1 <= n <= 4096. A batch
 * of more than one simulation requires PIC_MIXED32 in every set and the same
 * PIC_NO_GRAPH and PIC_EXPLICIT flags. Simulation 0 is selected.
 * pic_select: per-simulation calls (pic_load_particles, pic_set_fields, pic_fields,
 * pic_moments, pic_particle_count, pic_particles, and the PCG iteration count of
 * pic_profile) address simulation k from now on. The counters cfl_violations and
 * overflow_moves of pic_moments, and error returns of pic_step, are handle-wide.
 * pic_batch_size: number of simulations of the handle (0 for NULL). */
PIC_API int pic_init_batch(const pic_params* p, int32_t n, pic_sim** out);
PIC_API int pic_select(pic_sim* s, int32_t k);
PIC_API int pic_batch_size(const pic_sim* s);

/* Tile-shape autotuner for PIC_MIXED32 (the paper has no counterpart: tiles are a
 * storage detail of this library and do not change the method). For each shape order
 * present in p[0..n), it builds a scratch batch of those simulations for each candidate
 * tile shape (32x16, 16x16, 32x8, 64x8, 64x16, 16x8, 32x32 cells, clamped to each grid),
 * fills it with a synthetic drifting pair plasma of each set's ppc and gamma0, runs two
 * warm-up steps and `steps` timed steps (1..1000), and writes the fastest shape into
 * tile_x, tile_y of those sets. best_ms (NULL allowed, else 3 doubles) receives the
 * tile-kernel milliseconds per step of the chosen shape for orders 1, 2, 3 (0 if the
 * order is absent). The scratch handles are freed before returning; the simulations
 * described by p are not touched. Errors: PIC_EINVAL (bad sets), PIC_ECUDA (no shape
 * could be run); the message is in pic_last_error(NULL). */
PIC_API int pic_autotune_tiles(pic_params* p, int32_t n, int32_t steps, double* best_ms);

/* Run subsequent work of this handle on the given CUDA stream (cudaStream_t, passed as
 * void*). NULL selects the handle's own non-blocking stream, which is also the default.
 * The legacy default stream cannot be used (steps are captured into CUDA graphs).
 * Waits for work already enqueued on the previous stream; drops the captured graph. */
PIC_API int pic_set_stream(pic_sim* s, void* cuda_stream);

/* Replace the particles of one species (0 = positrons, 1 = electrons) with n
 * macro-particles: physical positions x in [0, nx dx), y in [0, ny dy) and momenta
 * u = gamma v (units of c). Arrays are FP64, host or device; they are copied. Positions
 * outside the box are wrapped periodically. MIXED32 converts to cell + FP32 offset and
 * FP32 momenta and sorts into tiles; its temporaries (about 56 bytes per particle:
 * the FP64 copy, the staged FP32 form, the sort keys) come from a stream-ordered pool
 * of the library's that keeps its memory for the next load, re-sort or diagnostic call
 * of any handle in the process. Returns PIC_EINVAL for bad species, n < 0, NULL arrays
 * with n > 0, or non-finite values. */
PIC_API int pic_load_particles(pic_sim* s, int32_t species, const double* x, const double* y,
                       const double* ux, const double* uy, const double* uz, int64_t n);

/* Overwrite one field component (PIC_EX..PIC_BZ) with nx*ny FP64 values (host or
 * device). The caller keeps ownership of data. */
PIC_API int pic_set_fields(pic_sim* s, int32_t which, const double* data, size_t len);

/* Advance n >= 0 steps of the particle cycle (Sec. 2, Sec. 3): for each step, gather
 * E^n, B^n; push; move; deposit J^{n+1/2}; solve Eq. (7) by PCG; update E, B by
 * Eqs. (5)-(6) (with PIC_EXPLICIT: Eqs. (3)-(4), no solve). Work is enqueued on the handle's stream and the call returns after the
 * stream has finished (one host synchronisation per call, not per step; MIXED32 also
 * synchronises every 32 steps, to re-sort particles that found no room in their tile's
 * bin into larger bins). Errors
 * detected on the device (PIC_ECG_NOCONV, PIC_ECFL, PIC_ENAN) stop the remaining
 * steps of the call; the fields and particles then hold the state after the failing
 * step and pic_moments reports its step count. PIC_ESTATE if warm_start is
 * PIC_WS_LEARNED and no network has been set with pic_set_cnn. */
PIC_API int pic_step(pic_sim* s, int32_t n);

/* Advance n >= 1 steps like pic_step, timing each with CUDA events recorded on the
 * handle's stream inside the step graph, and synchronising after every step. Writes up
 * to n_out averages (milliseconds per step unless noted) into out:
 *   out[0] whole step; out[1] particle half (J reset, push, deposit, migration);
 *   out[2] the dominant particle kernel alone (the FP64 push kernels, or the MIXED32
 *          tile kernel); out[3] field solve (rhs of Eq. (7), PCG, Eqs. (5)-(6) update);
 *   out[4] PCG iterations per step (count, not ms).
 * Device-detected errors are reported as by pic_step. */
PIC_API int pic_profile(pic_sim* s, int32_t n, double* out, int32_t n_out);

/* Copy grid quantity `which` (PIC_EX..PIC_DENSITY_E) into out (len >= nx*ny FP64 values,
 * host or device, caller-owned). */
PIC_API int pic_fields(pic_sim* s, int32_t which, double* out, size_t len);

/* Fill *out with diagnostics at the current step (energies, PCG statistics, counts). */
PIC_API int pic_moments(pic_sim* s, pic_moments_t* out);

/* Number of live macro-particles of a species. */
PIC_API int64_t pic_particle_count(pic_sim* s, int32_t species);

/* Copy the particles of a species into out: 5 arrays of n FP64 values laid out as
 * [x(n), y(n), ux(n), uy(n), uz(n)] (host or device, caller-owned); n must equal
 * pic_particle_count. FP64 mode keeps the load order; MIXED32 returns tile order. */
PIC_API int pic_particles(pic_sim* s, int32_t species, double* out5xn, int64_t n);

/* ---- allocation-free field solve ----------------------------------------------------
 * The paper has no counterpart to this entry point: it is a service of this library.
 *
 * Some callers cannot allocate device memory: an application whose device memory is
 * already reserved by another allocator's pool (a framework that takes the GPU's memory
 * at start-up), a long-running service that forbids allocation after start-up because
 * an allocation can fail under fragmentation or stall the device mid-run, or a caller
 * that has no access to the CUDA allocation calls at all. pic_field_solve_noalloc gives
 * them the field solve of pic_step without any allocation: it builds the right-hand side
 * b of Eq. (7) from the fields F and the current J, then runs the same Jacobi-PCG, from a
 * zero initial guess, until ||r||_2 <= cg_rtol ||b||_2, and writes dB. It solves the
 * periodic operator only (the grid is periodic in x and y; a handle with PIC_BC_WALLS
 * solves a different operator), with dt = cfl * dx as in pic_params.
 *
 * Its scratch (three solver vectors of 3*nx*ny FP64 values, reduction partials, solver
 * state) is a fixed array in the library's device memory, sized for
 * PIC_NOALLOC_MAX_CELLS cells (about 4.7 MB). Every GPU that loads the library holds it
 * until the process exits. The call makes no cudaMalloc, cudaFree or other allocating
 * call; it enqueues copies, sets and kernels on `stream` and synchronises that stream
 * before returning.
 *
 *   nx, ny          grid size; nx, ny >= 8 and nx*ny <= PIC_NOALLOC_MAX_CELLS
 *   dx, dy, cfl, theta, cg_rtol, cg_max_iter   as in pic_params
 *   F               device pointer (memory of the current device, or managed memory),
 *                   6*nx*ny FP64: Ex, Ey, Ez, Bx, By, Bz (the layout of
 *                   pic_fields, component-major, index j*nx + i)
 *   J               device pointer, 3*nx*ny FP64: Jx, Jy, Jz
 *   dB              device pointer, 3*nx*ny FP64, written: dBx, dBy, dBz
 *   iters, rel_resid  optional outputs (NULL allowed): PCG iterations and ||r||/||b||
 *   stream          cudaStream_t as void* (NULL = the legacy default stream)
 *   errbuf, errlen  optional caller-owned buffer for a message (NULL allowed)
 * The library cannot see the lengths of F, J and dB: they must hold at least the counts
 * above (the Python binding checks them). Returns PIC_OK, PIC_EINVAL (sizes beyond the
 * maximum, bad parameters, or a pointer that is not memory of the current device),
 * PIC_ECUDA, or PIC_ECG_NOCONV.
 *
 * The first call on a device does a one-time set-up on that device (it looks up the
 * device address of the scratch array); make that first call before any stream capture
 * on the device. With CUDA's lazy module loading (the default since CUDA 12.2) that
 * set-up is also when the array is reserved and the solver's kernels are loaded, so it
 * can itself need device memory: make the first call before the caller's allocator
 * takes the GPU's memory. Later calls need none. All calls on a device share the one array and each starts by clearing
 * what must start at zero: calls that overlap on the GPU (on different streams or from
 * different host threads) race and produce wrong results, so serialise them. */
#define PIC_NOALLOC_MAX_CELLS 65536
PIC_API int pic_field_solve_noalloc(int32_t nx, int32_t ny, double dx, double dy, double cfl,
                                    double theta, double cg_rtol, int32_t cg_max_iter,
                                    const double* F, const double* J, double* dB,
                                    int32_t* iters, double* rel_resid, void* stream,
                                    char* errbuf, size_t errlen);

/* ---- learned warm start --------------------------------------------------------------
 * The paper solves Eq. (7) by PCG from a plain initial guess; this library can start it
 * from a guess made by a small convolutional network instead (PIC_WS_LEARNED). The CG
 * still iterates to the same tolerance cg_rtol, so the solution is the plain solver's;
 * the network only changes how many iterations that takes.
 *
 * Network: four 3x3 convolutions with periodic padding and biases, 3 -> 32 -> 32 ->
 * 32 -> 3 channels, no activation (the map b -> dB = A^{-1} b it approximates is
 * linear). Its input is b / rms(b) with the three components of b as channels on the
 * cell grid (rms over the 3 nx ny values), its output dB_0 / rms(b). Convolutions run
 * on the tensor cores with BF16 operands and FP32 accumulation: the input, the weights
 * and every hidden activation and back-propagated gradient are rounded to BF16 (to
 * nearest even); the output and loss are FP32.
 *
 * In the solver (PIC_WS_LEARNED) the network is not run layer by layer: being linear,
 * its four layers compose exactly into one 9x9 stencil from the 3 channels to the 3
 * channels plus a bias, which pic_set_cnn computes in FP64 from the FP32 parameters and
 * the step applies in FP32 to b (x0 = K * b + bias rms(b)): about 1.5 kFLOP per cell
 * instead of 40 kFLOP, and no BF16 rounding. pic_cnn_stencil returns that stencil.
 *
 * Parameters (PIC_CNN_NPARAMS FP32 values), layer by layer (cin, cout) = (3, 32),
 * (32, 32), (32, 32), (32, 3): W[cout][tap][cin] with tap = 3 (dy + 1) + (dx + 1) for
 * the neighbour at (i + dx, j + dy), then b[cout].
 *
 * Image arrays (in, out, target) hold nimg images of [3][ny][nx] FP32 values, host or
 * device; nx*ny must be a multiple of 128. Every call synchronises the network's own
 * stream. Errors: PIC_EINVAL (sizes, NULL arrays), PIC_ENOMEM, PIC_ECUDA, PIC_ETIMEOUT (a
 * tensor-core completion wait ran out); pic_cnn_last_error gives the message. */
typedef struct pic_cnn pic_cnn;
#define PIC_CNN_NPARAMS 20259
PIC_API int pic_cnn_create(pic_cnn** out); /* all parameters zero */
PIC_API void pic_cnn_free(pic_cnn* c);
PIC_API const char* pic_cnn_last_error(const pic_cnn* c); /* c == NULL: last create failure */
PIC_API int pic_cnn_set_params(pic_cnn* c, const float* p, int64_t n); /* resets Adam state */
PIC_API int pic_cnn_get_params(pic_cnn* c, float* p, int64_t n);
/* out = network(in). */
PIC_API int pic_cnn_forward(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in, float* out);
/* Gradient of the loss L = mean over images, channels and pixels of (network(in) -
 * target)^2 with respect to the parameters (grad: PIC_CNN_NPARAMS values, layout as
 * above), and L itself (loss may be NULL). */
PIC_API int pic_cnn_gradient(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in,
                             const float* target, float* grad, double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on that loss. */
PIC_API int pic_cnn_train_step(pic_cnn* c, int32_t nimg, int32_t nx, int32_t ny, const float* in,
                               const float* target, float lr, double* loss);
/* The collapsed stencil of the current parameters: PIC_CNN_STENCIL FP32 values,
 * K[co][ci][dy + 4][dx + 4] for the neighbour (i + dx, j + dy), then bias[co] (host or
 * device). */
#define PIC_CNN_STENCIL 732
PIC_API int pic_cnn_stencil(pic_cnn* c, float* out, int64_t n);
/* Collapse the network's current parameters into the handle's learned guess for
 * PIC_WS_LEARNED. Later training of c does not affect the handle until the next
 * pic_set_cnn. */
PIC_API int pic_set_cnn(pic_sim* s, const pic_cnn* c);
/* The tensor-core building block: D = A B^T with A [M x K], B [N x K] row-major BF16
 * bit patterns and D [M x N] FP32 (host or device; M a multiple of 128, N and K
 * multiples of 16 in [16, 256]). Errors are reported through pic_cnn_last_error(NULL). */
PIC_API int pic_tc_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, const uint16_t* B,
                             float* D);

/* Fourier diagnostics (the k-space maps of Sec. 3.1, Fig. 3): the amplitude spectrum of
 * grid quantity `which` (PIC_EX..PIC_DENSITY_E) of the selected simulation,
 *   out[q nx + p] = |sum_{l,m} F(l, m) exp(-2 pi i (p l / nx + q m / ny))| / (nx ny),
 * p, q in FFT order (p >= nx/2 stands for the wave number 2 pi (p - nx) / (nx dx)). len
 * >= nx*ny FP64 values (host or device). FP64 FFTs on the GPU (radices 2, 3, 4, 5; other
 * lengths by the direct sum). Growth maps follow from two spectra: the rate of mode
 * (p, q) between steps n1 < n2 is ln(out2 / out1) / ((n2 - n1) dt). */
PIC_API int pic_spectrum(pic_sim* s, int32_t which, double* out, size_t len);

/* The resonance line of numerical Cherenkov radiation, Eq. (17): for a flow at
 * beta = V/c in (0, 1) and k_x dx in (0, pi], the k_y dy >= 0 at which the flow's mode
 * omega = V k_x meets the vacuum dispersion surface of the theta = 1/2 scheme, Eq. (15),
 * with cfl_x = c dt/dx, cfl_y = c dt/dy. Returns PIC_OK and *ky_dy (the line is symmetric:
 * -ky_dy too), or PIC_EINVAL when no real k_y exists for this k_x (the flow does not
 * overtake those waves) or an argument is out of range. Host only; needs no handle. */
PIC_API int pic_resonance_ky(double cfl_x, double cfl_y, double beta, double kx_dx, double* ky_dy);

/* Conservation diagnostics of the selected simulation, computed on demand from the
 * particles and fields (a pass over all particles: not for every step): up to n_out of
 *   out[0..2] total momentum sum w u of both species (units of m c),
 *   out[3]    total charge sum rho dx dy,
 *   out[4]    max |div E - 4 pi rho| over the nodes (off the wall column with walls),
 *   out[5]    its root mean square.
 * With charge-conserving deposits out[4] stays at its initial value to round-off. */
PIC_API int pic_conservation(pic_sim* s, double* out, int32_t n_out);

/* Checkpoints. pic_save writes every simulation of the handle to `path`: its parameters,
 * E, B, the last dB (the previous-step warm start), both species' particles (FP64
 * physical positions and momenta) and the step counters (the injector's schedule
 * follows them). pic_restore reads such a file into a handle created with the same
 * parameters (same precision and number of simulations; PIC_EINVAL otherwise) and
 * replaces its state. The file is read and checked in full first: an unreadable,
 * truncated or mismatched file gives PIC_EINVAL and leaves the handle unchanged.
 * MIXED32 particles round-trip exactly when dx = dy = 1. PCG statistics and a learned
 * network are not saved. */
PIC_API int pic_save(pic_sim* s, const char* path);
PIC_API int pic_restore(pic_sim* s, const char* path);

/* Message of the last failure on this handle (or of the last failed pic_init when s
 * is NULL). The string stays valid until the next call on the handle. */
PIC_API const char* pic_last_error(const pic_sim* s);

/* ---- bounded device-side waits -----------------------------------------------------
 * The paper has no counterpart: these are services of this library for testing its
 * failure paths. Every wait inside the library's kernels is bounded. The grid barriers
 * of the cooperative PCG (a persistent kernel whose blocks meet through global memory)
 * poll at most 2^22 times; the tensor-core completion waits of the network's kernels
 * at most 2^24 times. A wait that runs out makes the kernel record the failure and
 * return (a tensor-core wait that gave up first waits, with the default bound, for the
 * matrix operations it has in flight, and only then frees its tensor memory); the call
 * reports PIC_ETIMEOUT and the device stays usable.
 *
 * These calls lower the bound so that a test can make the waits run out on purpose:
 * spins >= 1 polls per wait, 0 restores the default. pic_set_wait_limit applies to the
 * handle's cooperative solve (MIXED32) from the next step on; a handle that solves
 * without it is unaffected. pic_cnn_set_wait_limit applies to the network's next calls
 * (forward, gradient, training). Both return PIC_OK or PIC_EINVAL (spins < 0). */
PIC_API int pic_set_wait_limit(pic_sim* s, int32_t spins);
PIC_API int pic_cnn_set_wait_limit(pic_cnn* c, int32_t spins);

/* Release the handle and all its device memory. NULL is a no-op. */
PIC_API void pic_free(pic_sim* s);

/* ---- check of the FP32-pair arithmetic ------------------------------------------------
 * The MIXED32 right-hand side of Eq. (7), its E update and the refinements of the
 * Chebyshev solve compute in pairs of FP32 numbers h + l (47 significant bits) instead
 * of FP64 (the paper fixes no precision; this part's FP64 pipe is slow). This entry runs
 * the device's building blocks on n inputs so that a test can hold them against exact
 * host arithmetic. With a = x[i], b = x[(i + 1) mod n], k = d[i], for i < n:
 *   out[10 i + 0], out[10 i + 1]  the pair of a (h, l)
 *   out[10 i + 2]                 a rounded to FP32 (to nearest, ties to even)
 *   out[10 i + 3], out[10 i + 4]  the pair of the integer k
 *   out[10 i + 5], out[10 i + 6]  pair(a) + pair(b)
 *   out[10 i + 7], out[10 i + 8]  pair(a) x pair(b)
 *   out[10 i + 9]                 (pair(a) joined back to FP64) - a, rounded to FP32
 * x, d and out are host arrays of n, n and 10 n values; 1 <= n <= 2^24. Returns PIC_OK,
 * PIC_EINVAL (n out of range or a NULL pointer) or PIC_ECUDA, with the message in
 * pic_last_error(NULL). No handle is needed; the call uses the current device. */
PIC_API int pic_dword_check(const double* x, const int64_t* d, int64_t n, float* out);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
