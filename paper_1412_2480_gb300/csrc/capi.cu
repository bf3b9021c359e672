// capi.cu -- the C ABI (include/pic.h): handle lifecycle, parameter validation, particle
// and field I/O, and the step sequence.
//
// One step (Sec. 2, Sec. 3 of Ikeya & Matsumoto 2015):
//   step_begin -> J = 0 -> particle half (gather E^n,B^n; push; move; deposit J^{n+1/2})
//   -> rhs of Eq. (7) -> WHILE(any simulation active) { PCG iteration } -> E,B update
//   (Eqs. (5)-(6)) -> step_end.
// The step is captured once into a CUDA graph whose PCG loop is a WHILE conditional
// node driven from the device, so pic_step(n) launches n graphs and synchronises once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cnn.h"
#include "dword.cuh"
#include "engine.h"
#include "mixed.h"
#include "pic.h"

using namespace pic;

struct pic_sim {
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;      // stream all work of the handle is enqueued on
    cudaStream_t own_stream = nullptr;  // the handle's own non-blocking stream (default)
    pic_params prm{};                // the first simulation's parameters (handle-wide settings)
    std::vector<pic_params> prms;    // every simulation's parameters
    int ngrids = 1;
    int sel = 0;                     // simulation addressed by per-simulation calls
    std::vector<GridDev> hgrids;
    GridDev* dgrids = nullptr;
    std::vector<int> hblk_grid;
    int* dblk_grid = nullptr;
    int nblk = 0;
    long long ntot = 0;
    // grid arrays
    double* F = nullptr;    // 6 ntot
    double* J64 = nullptr;  // 3 ntot (FP64)
    long long* Jfix = nullptr;  // 3 ntot fixed-point current (MIXED32)
    float* F32 = nullptr;   // 6 ntot (MIXED32)
    double* Fn = nullptr;   // 6 ntot node-averaged fields (FP64 with PIC_GATHER_NODAL)
    bool any_nodal = false;
    bool quads = false;  // every simulation's nx is a multiple of 4
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    double* part = nullptr;
    CgState* cg = nullptr;
    unsigned int* done = nullptr;
    DevStatus* st = nullptr;
    double* tmp = nullptr;  // ntot scratch for conversions (pic_fields of J in MIXED32)
    // FP64 particles, one set of arrays per species (grid units)
    double* pa[2][5] = {{nullptr}};
    long long np[2] = {0, 0};
    long long pcap[2] = {0, 0};
    SegDev* dsegs = nullptr;   // [2]
    int* dblk_seg[2] = {nullptr, nullptr};
    int nblk_push[2] = {0, 0};
    // MIXED32 particles
    MixedState* mixed = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // profiling: one graph per part of the step, CUDA events recorded between them
    cudaEvent_t ev[6] = {nullptr};
    cudaGraph_t pgraph[5] = {nullptr};
    cudaGraphExec_t pexec[5] = {nullptr};
    long long graph_gen = 0;  // MIXED32 buffer generation the captured graphs point into
    cudaStream_t body_stream = nullptr;
    cudaStream_t body_stream2 = nullptr;  // captures the inner loop of the MIXED32 solve
    // MIXED32 mixed-precision PCG: FP64 right-hand side and FP32 inner vectors
    double* bvec = nullptr;
    float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *e32 = nullptr;
    float *r32b = nullptr, *z32 = nullptr;  // second inner residual buffer, z = M r
    // learned warm start: the network's forward weights and its buffers
    bool learned = false;
    bool has_cnn = false;
    CnnGuess guess;
    // MIXED32 solve as one cooperative kernel
    bool use_coop = false;
    CoopSolve coop;
    // bookkeeping
    long long steps = 0;
    long long kernels = 0;         // kernels of this library launched by pic_step / pic_profile
    long long graph_kernels = -1;  // kernel nodes of the step graph outside its PCG loop
    unsigned long long seen_cfl = 0, seen_nan = 0, seen_lost = 0;
    unsigned int seen_noconv = 0, seen_sync = 0;
};

namespace {

enum { kPartPre = 0, kPartPush = 1, kPartPost = 2, kPartField = 3, kPartEnd = 4, kNumParts = 5 };

std::string g_init_err;

int fail(pic_sim* s, int code, const std::string& msg) {
    if (s) s->err = msg;
    else g_init_err = msg;
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(s, PIC_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

int validate(const pic_params* p, std::string& why) {
    char buf[256];
    auto bad = [&](const char* m) {
        why = m;
        return PIC_EINVAL;
    };
    if (!p) return bad("params is NULL");
    if (p->nx < 8 || p->ny < 8 || p->nx > 32768 || p->ny > 32768)
        return bad("nx and ny must lie in [8, 32768]");
    if (!(p->dx > 0) || !(p->dy > 0)) return bad("dx and dy must be > 0");
    if (!(p->cfl > 0) || p->cfl > 1.0) return bad("cfl must lie in (0, 1]");
    if (p->cfl * p->dx > p->dy * (1.0 + 1e-12))
        return bad("dt = cfl*dx must not exceed dy (a move must stay below one cell)");
    if (!(p->theta >= 0.5) || p->theta > 1.0) return bad("theta must lie in [0.5, 1]");
    if (p->shape_order < 1 || p->shape_order > 3) return bad("shape_order must be 1, 2 or 3");
    if (!(p->gamma0 >= 1.0)) return bad("gamma0 must be >= 1");
    if (p->ppc < 1) return bad("ppc must be >= 1");
    if (!(p->skin_depth > 0)) return bad("skin_depth must be > 0");
    if (p->precision != PIC_FP64 && p->precision != PIC_MIXED32)
        return bad("precision must be PIC_FP64 or PIC_MIXED32");
    if (!(p->cg_rtol > 0) || p->cg_rtol >= 1) return bad("cg_rtol must lie in (0, 1)");
    if (p->cg_max_iter < 1 || p->cg_max_iter > 100000) return bad("cg_max_iter must lie in [1, 1e5]");
    if (p->warm_start != PIC_WS_ZERO && p->warm_start != PIC_WS_PREV && p->warm_start != PIC_WS_LEARNED)
        return bad("warm_start must be PIC_WS_ZERO, PIC_WS_PREV or PIC_WS_LEARNED");
    if (p->warm_start == PIC_WS_LEARNED && p->precision != PIC_MIXED32)
        return bad("PIC_WS_LEARNED requires PIC_MIXED32");
    if ((p->flags & PIC_GATHER_NODAL) && p->bc_x == PIC_BC_WALLS)
        return bad("PIC_GATHER_NODAL needs periodic boundaries");
    if (p->flags & PIC_EXPLICIT) {
        // Eq. (16): real frequencies for every mode need (c dt)^2 (1/dx^2 + 1/dy^2) <= 1
        const double dt = p->cfl * p->dx;
        if (dt * dt * (1.0 / (p->dx * p->dx) + 1.0 / (p->dy * p->dy)) > 1.0 + 1e-12)
            return bad("PIC_EXPLICIT needs (c dt)^2 (1/dx^2 + 1/dy^2) <= 1 (Courant limit of Eq. 16)");
        if (p->warm_start == PIC_WS_LEARNED) return bad("PIC_EXPLICIT has no solve to warm-start");
    }
    if (p->tile_x < 0 || p->tile_y < 0) return bad("tile sizes must be >= 0");
    const int tx = std::min(p->tile_x > 0 ? p->tile_x : 32, p->nx);
    const int ty = std::min(p->tile_y > 0 ? p->tile_y : 16, p->ny);
    if ((tx + 5) * (ty + 5) > kMaxWinCells) {
        snprintf(buf, sizeof buf, "(tile_x+5)*(tile_y+5) must not exceed %d", kMaxWinCells);
        return bad(buf);
    }
    if (p->bin_slack < 0) return bad("bin_slack must be >= 0");
    if (p->bc_x != PIC_BC_PERIODIC && p->bc_x != PIC_BC_WALLS) return bad("bc_x must be PIC_BC_PERIODIC or PIC_BC_WALLS");
    if (p->inject_x0 >= 0.0) {
        if (p->bc_x != PIC_BC_WALLS) return bad("the injector needs PIC_BC_WALLS");
        if (p->inject_x0 < 2.0 * p->cfl || p->inject_x0 > p->nx) return bad("inject_x0 must lie in [2 cfl, nx]");
        if (!(p->u_th >= 0.0) || p->u_th > 1.0) return bad("u_th must lie in [0, 1]");
    }
    return PIC_OK;
}

void fill_grid(const pic_params& p, GridDev& G) {
    memset(&G, 0, sizeof G);
    G.nx = p.nx;
    G.ny = p.ny;
    G.order = p.shape_order;
    G.ncell = p.nx * p.ny;
    G.dx = p.dx;
    G.dy = p.dy;
    G.dt = p.cfl * p.dx;
    G.theta = (p.flags & PIC_EXPLICIT) ? 1.0 : p.theta;  // explicit: E sees the whole half step
    G.idx = 1.0 / p.dx;
    G.idy = 1.0 / p.dy;
    G.a = (p.theta * G.dt) * (p.theta * G.dt);
    G.cx = G.a / (p.dx * p.dx);
    G.cy = G.a / (p.dy * p.dy);
    G.c0 = 1.0 + 2.0 * G.cx + 2.0 * G.cy;
    {
        // Chebyshev-optimal degree-1 preconditioner p(A) on A's spectrum [l1, l2] =
        // [c0 - 2cx - 2cy, c0 + 2cx + 2cy] = [1, 1 + 4cx + 4cy] (Gershgorin; the periodic
        // and the wall operators alike): with d = (l1 + l2)/2 = c0 and hw = (l2 - l1)/2,
        // p(lambda) = 2 (2d - lambda) / (2 d^2 - hw^2), so that 1 - lambda p(lambda) is the
        // scaled Chebyshev polynomial T2 (at most 1 / T2(d / hw) in magnitude); p(A) =
        // (2 / D) (c0 I + cx (E + W) + cy (N + S)), D = 2 c0^2 - hw^2.
        const double hw = 2.0 * (G.cx + G.cy);
        const double D = 2.0 * G.c0 * G.c0 - hw * hw;
        G.pc0 = 2.0 * G.c0 / D;
        G.pcx = 2.0 * G.cx / D;
        G.pcy = 2.0 * G.cy / D;
    }
    // omega_pe^2 = 4 pi n q^2 / (m gamma0), n = ppc/(dx dy), q = m = w (Sec. 4 definition)
    const double wpe = 1.0 / p.skin_depth;
    G.w = wpe * wpe * p.gamma0 * p.dx * p.dy / (4.0 * kPi * p.ppc);
    G.qm[0] = 1.0;
    G.qm[1] = -1.0;
    G.qw[0] = G.w;
    G.qw[1] = -G.w;
    // MIXED32 fixed-point current: a single particle adds at most u/2 to one node, with
    // u = 2 max(q/(dt dy), q/(dt dx), q/(dx dy)); u maps to 2^40, so one unit is 9e-13 u
    // (far below FP32 rounding) and 2^23 u fits in int64.
    const double u = 2.0 * G.w * std::max(std::max(1.0 / (G.dt * p.dy), 1.0 / (G.dt * p.dx)),
                                          1.0 / (p.dx * p.dy));
    G.jscale = std::ldexp(1.0, 40) / u;
    G.jinv = 1.0 / G.jscale;
    const double area = G.dx * G.dy;
    for (int s = 0; s < 2; s++) {
        G.pk_h[s] = (float)(0.5 * G.qm[s] * G.dt);
        G.pk_fx[s] = (float)(G.qw[s] * G.dx / (G.dt * area));
        G.pk_fy[s] = (float)(G.qw[s] * G.dy / (G.dt * area));
        G.pk_fz[s] = (float)(G.qw[s] / area);
    }
    G.pk_dtx = (float)(G.dt * G.idx);
    G.pk_dty = (float)(G.dt * G.idy);
    G.js40 = (float)(G.jscale * std::ldexp(1.0, -40));
    {
        const auto pair = [](double v, float out[2]) {
            out[0] = (float)v;
            out[1] = (float)(v - (double)out[0]);
        };
        const double th_dt2 = G.theta * G.dt * G.dt;
        pair(th_dt2 * G.idx * G.idx, G.dw_ax);
        pair(th_dt2 * G.idy * G.idy, G.dw_ay);
        pair(4.0 * kPi * th_dt2 * G.jinv * G.idx, G.dw_kjx);
        pair(4.0 * kPi * th_dt2 * G.jinv * G.idy, G.dw_kjy);
        pair(G.dt * G.idx, G.dw_dtx);
        pair(G.dt * G.idy, G.dw_dty);
        pair(G.c0, G.dw_c0);
        pair(G.cx, G.dw_cx);
        pair(G.cy, G.dw_cy);
        pair(4.0 * kPi * G.dt * G.jinv, G.dw_fj);
        pair(G.theta, G.dw_th);
    }
    G.rtol = p.cg_rtol;
    G.maxit = p.cg_max_iter;
    G.warm = p.warm_start == PIC_WS_PREV ? 1 : (p.warm_start == PIC_WS_LEARNED ? 2 : 0);
    G.deposit = (p.flags & PIC_NO_DEPOSIT) ? 0 : 1;
    G.walls = p.bc_x == PIC_BC_WALLS ? 1 : 0;
    G.nodal = (p.flags & PIC_GATHER_NODAL) ? 1 : 0;
    G.inject = (G.walls && p.inject_x0 >= 0.0) ? 1 : 0;
    G.ppc = p.ppc;
    G.inj_x0 = p.inject_x0;
    G.cfl = p.cfl;
    G.gamma0 = p.gamma0;
    G.u_th = p.u_th;
    G.inj_seed = p.seed;
}

FieldArgs field_args(pic_sim* s, int use_cond, cudaGraphConditionalHandle cond) {
    FieldArgs a{};
    a.grids = s->dgrids;
    a.blk_grid = s->dblk_grid;
    a.ngrids = s->ngrids;
    a.nblk = s->nblk;
    a.ntot = s->ntot;
    a.F = s->F;
    a.J64 = s->prm.precision == PIC_FP64 ? s->J64 : nullptr;
    a.Jfix = s->prm.precision == PIC_MIXED32 ? s->Jfix : nullptr;
    a.F32 = s->F32;
    a.Fn = s->Fn;
    a.any_nodal = s->any_nodal ? 1 : 0;
    a.coop = s->use_coop ? 1 : 0;
    a.quads = s->quads ? 1 : 0;
    a.x = s->x;
    a.r = s->r;
    a.p = s->p;
    a.q = s->q;
    a.cg = s->cg;
    a.part = s->part;
    a.done = s->done;
    a.st = s->st;
    a.cond = cond;
    a.use_cond = use_cond;
    a.b = s->bvec;
    a.r32 = s->r32;
    a.p32 = s->p32;
    a.q32 = s->q32;
    a.e32 = s->e32;
    a.r32b = s->r32b;
    a.z32 = s->z32;
    return a;
}

void drop_graph(pic_sim* s);

// Graphs hold buffer pointers as kernel arguments: drop them once MIXED32 re-binning
// has reallocated its buffers.
void check_graph_generation(pic_sim* s) {
    if (s->mixed && mixed_generation(s->mixed) != s->graph_gen) {
        drop_graph(s);
        s->graph_gen = mixed_generation(s->mixed);
    }
}

void drop_graph(pic_sim* s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->graph) cudaGraphDestroy(s->graph);
    s->gexec = nullptr;
    s->graph = nullptr;
    for (int k = 0; k < kNumParts; k++) {
        if (s->pexec[k]) cudaGraphExecDestroy(s->pexec[k]);
        if (s->pgraph[k]) cudaGraphDestroy(s->pgraph[k]);
        s->pexec[k] = nullptr;
        s->pgraph[k] = nullptr;
    }
}

// The step in five parts: [step_begin, J = 0, (overflow push)] [dominant particle
// kernel] [migration] [field solve: rhs, PCG loop, E/B update] [step_end].
void enqueue_part(pic_sim* s, int part, cudaStream_t st) {
    const FieldArgs a = field_args(s, 0, 0);
    const bool fp64 = s->prm.precision == PIC_FP64;
    switch (part) {
    case kPartPre:
        launch_step_begin(a, st);
        if (fp64) cudaMemsetAsync(s->J64, 0, 3 * s->ntot * sizeof(double), st);
        else cudaMemsetAsync(s->Jfix, 0, 3 * s->ntot * sizeof(long long), st);
        if (!fp64) mixed_enqueue(s->mixed, st, 0);
        break;
    case kPartPush:
        if (!fp64) {
            mixed_enqueue(s->mixed, st, 1);
            break;
        }
        for (int sp = 0; sp < 2; sp++) {
            if (s->nblk_push[sp] == 0) continue;
            Fp64PushArgs p{};
            p.grids = s->dgrids;
            p.segs = s->dsegs + sp;
            p.blk_seg = s->dblk_seg[sp];
            p.nblk = s->nblk_push[sp];
            p.nsegs = 1;
            p.ntot = s->ntot;
            p.F = s->Fn ? s->Fn : s->F;  // node-averaged copy for the nodal gather
            p.J = s->J64;
            p.x = s->pa[sp][0];
            p.y = s->pa[sp][1];
            p.ux = s->pa[sp][2];
            p.uy = s->pa[sp][3];
            p.uz = s->pa[sp][4];
            p.cg = s->cg;
            p.st = s->st;
            launch_push_fp64(p, s->prm.shape_order, st);
        }
        break;
    case kPartPost:
        if (!fp64) {
            mixed_enqueue(s->mixed, st, 2);  // the injector's pairs, then the bin swap
        } else if (s->hgrids[0].inject) {
            Fp64InjectArgs in{};
            in.grids = s->dgrids;
            in.segs = s->dsegs;
            for (int sp = 0; sp < 2; sp++) {
                in.cap[sp] = s->pcap[sp];
                in.x[sp] = s->pa[sp][0];
                in.y[sp] = s->pa[sp][1];
                in.ux[sp] = s->pa[sp][2];
                in.uy[sp] = s->pa[sp][3];
                in.uz[sp] = s->pa[sp][4];
            }
            in.st = s->st;
            in.ny = s->hgrids[0].ny;
            const GridDev& G = s->hgrids[0];
            in.kmax = (long long)std::ceil(G.ppc * (1.0 + std::sqrt(1.0 - 1.0 / (G.gamma0 * G.gamma0))) * G.cfl) + 1;
            launch_inject_fp64(in, st);
        }
        break;
    case kPartEnd:
        launch_step_end(a, st);
        break;
    default:
        break;
    }
}

// A conditional handle on the graph that stream `st` is capturing into.
cudaError_t new_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cap = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cap, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(h, cap, 0, cudaGraphCondAssignDefault);
    return e;
}

// Append WHILE(h) { body } at the capture position of `st`; the body is captured on
// stream `bs` into the conditional node's body graph.
template <typename Body>
cudaError_t add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaStream_t bs, Body body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t cap = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cap, &deps, nullptr, &nd);
    cudaGraphNode_t wnode{};
    cudaGraphNodeParams cp{};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, cap, deps, nullptr, nd, &cp);
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t eb = body(bs);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(bs, &out);
            if (e == cudaSuccess) e = eb;
        }
    }
    return e;
}

// Capture the parts in `mask` (in order) into one graph. The field-solve part becomes
// rhs -> WHILE(any simulation active){PCG iteration} -> E/B update, the WHILE condition
// being set on the device by the rhs and PCG kernels.
int capture(pic_sim* s, int mask, cudaGraph_t* gout, cudaGraphExec_t* xout) {
    cudaStream_t st = s->stream;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int part = 0; part < kNumParts && e == cudaSuccess; part++) {
        if (!(mask & (1 << part))) continue;
        if (part != kPartField) {
            enqueue_part(s, part, st);
            continue;
        }
        if (s->prm.flags & PIC_EXPLICIT) {
            launch_explicit_fields(field_args(s, 0, 0), st);
            launch_nodal(field_args(s, 0, 0), st);
            continue;
        }
        if (s->use_coop) {
            // rhs -> (learned guess) -> one cooperative kernel for the whole PCG -> update
            launch_rhs(field_args(s, 0, 0), st);
            if (s->learned) {
                // the guess from b's FP32 copy, into the FP64 solution (the refinements'
                // base) and an FP32 copy (in e32) for its residual, formed in FP32: that
                // residual only starts the first inner solve
                launch_learned_guess(s->guess, s->dgrids, s->cg, s->ntot, s->bvec, s->r32, s->x, s->e32, st);
                launch_guess_residual32(field_args(s, 0, 0), st);
            }
            e = launch_mp_coop(s->coop, field_args(s, 0, 0), st);
            if (e == cudaSuccess) launch_field_update(field_args(s, 0, 0), st);
            launch_nodal(field_args(s, 0, 0), st);
            continue;
        }
        cudaGraphConditionalHandle h{};
        e = new_handle(st, &h);
        if (e == cudaSuccess) launch_rhs(field_args(s, 1, h), st);
        if (e == cudaSuccess && s->learned) {
            launch_learned_guess(s->guess, s->dgrids, s->cg, s->ntot, s->bvec, nullptr, s->x, nullptr, st);
            launch_guess_residual(field_args(s, 1, h), st);
        }
        if (e == cudaSuccess && s->prm.precision == PIC_FP64) {
            e = add_while(st, h, s->body_stream,
                          [&](cudaStream_t bs) { launch_cg_iteration(field_args(s, 1, h), bs); return cudaSuccess; });
        } else if (e == cudaSuccess) {
            // mixed precision: WHILE(outer) { inner begin; WHILE(inner) { FP32 iteration };
            // x += e, r = b - A x }
            e = add_while(st, h, s->body_stream, [&](cudaStream_t bs) {
                cudaGraphConditionalHandle hin{};
                cudaError_t ei = new_handle(bs, &hin);
                if (ei != cudaSuccess) return ei;
                FieldArgs a = field_args(s, 1, h);
                a.cond_in = hin;
                launch_mp_inner_begin(a, bs);
                ei = add_while(bs, hin, s->body_stream2, [&](cudaStream_t bs2) {
                    launch_mp_inner_iteration(a, bs2);
                    return cudaSuccess;
                });
                if (ei == cudaSuccess) launch_mp_refine(a, bs);
                return ei;
            });
        }
        if (e == cudaSuccess) launch_field_update(field_args(s, 0, 0), st);
        launch_nodal(field_args(s, 0, 0), st);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(s, PIC_ECUDA, std::string("step graph capture failed: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(s, PIC_ECUDA, std::string("cudaGraphInstantiate failed: ") + cudaGetErrorString(e));
    }
    *gout = g;
    *xout = x;
    return PIC_OK;
}

int build_graph(pic_sim* s) {
    drop_graph(s);
    int rc = capture(s, (1 << kNumParts) - 1, &s->graph, &s->gexec);
    s->graph_kernels = -1;
    size_t n = 0;
    if (rc == PIC_OK && cudaGraphGetNodes(s->graph, nullptr, &n) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(n);
        long long k = 0;
        if (n && cudaGraphGetNodes(s->graph, nodes.data(), &n) == cudaSuccess) {
            for (cudaGraphNode_t node : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(node, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
            }
            s->graph_kernels = k;
        }
    }
    cudaGetLastError();
    return rc;
}

// Kernels one step launches outside the PCG loop: the step graph's kernel nodes, or
// the same count from the step's structure for direct launches.
long long step_kernels(pic_sim* s, bool graph) {
    if (graph && s->graph_kernels >= 0) return s->graph_kernels;
    // step begin and end; field part: explicit half step, update_E, explicit_B, or
    // zero_x, rhs, update_E, update_B (+ the cooperative solve)
    long long k = (s->prm.flags & PIC_EXPLICIT) ? 5 : 6;
    if (!(s->prm.flags & PIC_EXPLICIT) && s->prm.precision == PIC_MIXED32) k -= 1;  // k_rhs_dw zeroes x itself
    if (s->prm.precision == PIC_MIXED32) {
        k += mixed_step_kernels(s->mixed);
    } else {
        k += (s->nblk_push[0] > 0 ? 1 : 0) + (s->nblk_push[1] > 0 ? 1 : 0);
        k += s->hgrids[0].inject ? 1 : 0;
    }
    if (s->learned) k += 2;  // k_guess, k_guess_residual
    if (s->use_coop) k += 1;
    if (s->any_nodal) k += 1;  // k_nodal
    return k;
}

// Kernels the PCG loop launched for the given loop-counter increments (none with the
// cooperative solve: its iterations run inside one launch).
long long loop_kernels(const pic_sim* s, unsigned long long d_iters, unsigned long long d_refine) {
    if (s->use_coop) return 0;
    return 2 * (long long)d_iters + (s->prm.precision == PIC_MIXED32 ? 3 * (long long)d_refine : 0);
}

// Direct launches (PIC_NO_GRAPH): the PCG loop is driven from the host.
int run_step_direct(pic_sim* s) {
    cudaStream_t st = s->stream;
    enqueue_part(s, kPartPre, st);
    enqueue_part(s, kPartPush, st);
    enqueue_part(s, kPartPost, st);
    const FieldArgs a = field_args(s, 0, 0);
    if (s->prm.flags & PIC_EXPLICIT) {
        launch_explicit_fields(a, st);
        launch_nodal(a, st);
        enqueue_part(s, kPartEnd, st);
        CK(cudaGetLastError());
        return PIC_OK;
    }
    launch_rhs(a, st);
    if (s->learned) {
        if (s->use_coop) {
            launch_learned_guess(s->guess, s->dgrids, s->cg, s->ntot, s->bvec, s->r32, s->x, s->e32, st);
            launch_guess_residual32(a, st);
        } else {
            launch_learned_guess(s->guess, s->dgrids, s->cg, s->ntot, s->bvec, nullptr, s->x, nullptr, st);
            launch_guess_residual(a, st);
        }
    }
    if (s->use_coop) {
        CK(launch_mp_coop(s->coop, a, st));
        launch_field_update(a, st);
        launch_nodal(a, st);
        enqueue_part(s, kPartEnd, st);
        CK(cudaGetLastError());
        return PIC_OK;
    }
    unsigned int nact = 0, nin = 0;
    CK(cudaMemcpyAsync(&nact, &s->st->n_active, sizeof nact, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    while (nact > 0) {
        if (s->prm.precision == PIC_FP64) {
            launch_cg_iteration(a, st);
        } else {
            launch_mp_inner_begin(a, st);
            CK(cudaMemcpyAsync(&nin, &s->st->n_in_active, sizeof nin, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            while (nin > 0) {
                launch_mp_inner_iteration(a, st);
                CK(cudaMemcpyAsync(&nin, &s->st->n_in_active, sizeof nin, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            }
            launch_mp_refine(a, st);
        }
        CK(cudaMemcpyAsync(&nact, &s->st->n_active, sizeof nact, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    launch_field_update(a, st);
    launch_nodal(a, st);
    enqueue_part(s, kPartEnd, st);
    CK(cudaGetLastError());
    return PIC_OK;
}

// Pairs per species the moving injector can add over a whole run (it stops at x = nx).
long long inj_capacity(const GridDev& G) {
    if (!G.inject) return 0;
    const double w = (1.0 + std::sqrt(1.0 - 1.0 / (G.gamma0 * G.gamma0))) * G.cfl;
    const double steps = std::ceil((G.nx - G.inj_x0) / G.cfl) + 1.0;
    return (long long)G.ny * ((long long)std::ceil(G.ppc * w * steps) + 2);
}

// FP64 particle arrays of species sp with room for at least `need` particles, `n`
// of them live (contents kept when growing), and the push segment covering them: with
// the injector the segment covers the whole capacity and its count grows on the device.
int fp64_arrays(pic_sim* s, int sp, long long need, long long n) {
    if (need > s->pcap[sp]) {
        double* na[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        for (int a = 0; a < 5; a++) {
            if (dalloc(&na[a], (size_t)need) != cudaSuccess) {
                cudaGetLastError();
                for (int b = 0; b < 5; b++) dfree(na[b]);
                return fail(s, PIC_ENOMEM, "particle allocation failed");
            }
            if (s->pa[sp][a] && s->np[sp])
                CK(cudaMemcpy(na[a], s->pa[sp][a], s->np[sp] * sizeof(double), cudaMemcpyDeviceToDevice));
            dfree(s->pa[sp][a]);
            s->pa[sp][a] = na[a];
        }
        s->pcap[sp] = need;
    }
    const bool inj = s->hgrids[0].inject != 0;
    SegDev seg{};
    seg.start = 0;
    seg.count = n;
    seg.grid = 0;
    seg.species = sp;
    seg.blk_first = 0;
    seg.nblk = (int)(((inj ? s->pcap[sp] : n) + kPushThreads - 1) / kPushThreads);
    s->nblk_push[sp] = seg.nblk;
    s->np[sp] = n;
    CK(cudaMemcpy(s->dsegs + sp, &seg, sizeof seg, cudaMemcpyHostToDevice));
    dfree(s->dblk_seg[sp]);
    s->dblk_seg[sp] = nullptr;
    if (seg.nblk) {
        std::vector<int> t(seg.nblk, 0);
        CK(dalloc(&s->dblk_seg[sp], seg.nblk));
        CK(cudaMemcpy(s->dblk_seg[sp], t.data(), seg.nblk * sizeof(int), cudaMemcpyHostToDevice));
    }
    return PIC_OK;
}

// Live FP64 particle counts after steps that may have injected.
int fp64_counts(pic_sim* s) {
    if (s->prm.precision != PIC_FP64 || !s->hgrids[0].inject) return PIC_OK;
    SegDev seg[2];
    CK(cudaMemcpy(seg, s->dsegs, sizeof seg, cudaMemcpyDeviceToHost));
    s->np[0] = seg[0].count;
    s->np[1] = seg[1].count;
    return PIC_OK;
}

// Node density of the selected simulation into rho (device, ncell values): the charge
// density (which = PIC_RHO) or one species' number density (PIC_DENSITY_P / _E); when
// mom is given, w * the total momentum of both species is added into mom (device, 3).
int charge_density(pic_sim* s, double* rho, double* mom = nullptr, int which = PIC_RHO) {
    const GridDev& G = s->hgrids[s->sel];
    const double area = G.dx * G.dy;
    double q[2] = {G.qw[0] / area, G.qw[1] / area};
    if (which == PIC_DENSITY_P) q[0] = 1.0 / area, q[1] = 0.0;
    if (which == PIC_DENSITY_E) q[0] = 0.0, q[1] = 1.0 / area;
    CK(cudaMemsetAsync(rho, 0, G.ncell * sizeof(double), s->stream));
    if (s->mixed) return mixed_rho_momentum(s->mixed, s->sel, q, rho, mom, s->stream, s->err);
    for (int sp = 0; sp < 2; sp++) {
        if (!s->np[sp]) continue;
        if (q[sp] != 0.0) launch_rho_fp64(G, s->pa[sp][0], s->pa[sp][1], s->np[sp], q[sp], rho, s->stream);
        if (mom) launch_momentum_fp64(s->pa[sp][2], s->pa[sp][3], s->pa[sp][4], s->np[sp], G.w, mom, s->stream);
    }
    CK(cudaGetLastError());
    return PIC_OK;
}

int check_species(pic_sim* s, int sp) {
    if (sp < 0 || sp > 1) return fail(s, PIC_EINVAL, "species must be 0 (positrons) or 1 (electrons)");
    return PIC_OK;
}

// Device-side conversion of loaded FP64 particles: wrap into the box and scale to grid
// units; count non-finite entries (and, with walls, positions outside [0, Lx)).
__global__ void k_load_fp64(long long n, double* x, double* y, const double* ux, const double* uy,
                            const double* uz, double Lx, double Ly, double idx, double idy, int nx,
                            int ny, int walls, unsigned long long* nbad) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double X = x[k], Y = y[k];
    if (!isfinite(X) || !isfinite(Y) || !isfinite(ux[k]) || !isfinite(uy[k]) || !isfinite(uz[k]) ||
        (walls && !(X >= 0.0 && X < Lx))) {
        atomicAdd(nbad, 1ull);
        x[k] = 0.0;
        y[k] = 0.0;
        return;
    }
    X = X - floor(X / Lx) * Lx;
    Y = Y - floor(Y / Ly) * Ly;
    X *= idx;
    Y *= idy;
    if (X >= nx || X < 0) X = 0.0;
    if (Y >= ny || Y < 0) Y = 0.0;
    x[k] = X;
    y[k] = Y;
}

__global__ void k_unload_fp64(long long n, const double* x, const double* y, double dx, double dy,
                              double* ox, double* oy) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    ox[k] = x[k] * dx;
    oy[k] = y[k] * dy;
}

__global__ void k_fix_to_f64(long long n, const long long* a, double jinv, double* b) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) b[k] = (double)a[k] * jinv;
}

// Map device status counters that changed since the last check to a return code.
int device_errors(pic_sim* s, const DevStatus& hs) {
    int rc = PIC_OK;
    if (hs.sync_timeout != s->seen_sync) {
        rc = fail(s, PIC_ETIMEOUT, "a grid barrier of the cooperative PCG timed out");
    } else if (hs.cg_noconv != s->seen_noconv) {
        rc = fail(s, PIC_ECG_NOCONV, "PCG reached cg_max_iter before cg_rtol");
    } else if (hs.nan_count != s->seen_nan) {
        rc = fail(s, PIC_ENAN, "non-finite particle momentum or position");
    } else if (hs.lost != s->seen_lost) {
        rc = fail(s, PIC_ENOMEM, "particle storage exhausted (overflow list full)");
    } else if (hs.cfl_viol != s->seen_cfl) {
        rc = fail(s, PIC_ECFL, "a particle moved one cell or more in one step");
    }
    s->seen_noconv = hs.cg_noconv;
    s->seen_nan = hs.nan_count;
    s->seen_cfl = hs.cfl_viol;
    s->seen_lost = hs.lost;
    s->seen_sync = hs.sync_timeout;
    return rc;
}

int finish_call(pic_sim* s) {
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return PIC_OK;
}

constexpr int kMaxBatch = 4096;
// flags that hold for a whole handle: every simulation of a batch gives the same
constexpr int kHandleFlags = PIC_NO_GRAPH | PIC_NO_COOP | PIC_EXPLICIT | PIC_CG_INNER;

int init_handle(const pic_params* prm, int n, pic_sim** out) {
    pic_sim* s = nullptr;
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!prm) return fail(nullptr, PIC_EINVAL, "params is NULL");
    for (int k = 0; k < n; k++) {
        if (validate(prm + k, why) != PIC_OK) {
            if (n > 1) why = "simulation " + std::to_string(k) + ": " + why;
            return fail(nullptr, PIC_EINVAL, why);
        }
    }
    s = new (std::nothrow) pic_sim();
    if (!s) return fail(nullptr, PIC_ENOMEM, "host allocation failed");
    s->prm = prm[0];
    s->prms.assign(prm, prm + n);
    s->learned = prm[0].warm_start == PIC_WS_LEARNED;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(nullptr, PIC_ECUDA, "no CUDA device");
    }
    auto bail = [&](int code) {
        g_init_err = s->err;
        pic_free(s);
        return code;
    };
    // simulations side by side in every grid array; field kernels give each simulation a
    // grid-stride range of at most 4 blocks per SM
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device);
    s->ngrids = n;
    s->hgrids.resize(n);
    s->ntot = 0;
    s->nblk = 0;
    s->hblk_grid.clear();
    for (int g = 0; g < n; g++) {
        GridDev& G = s->hgrids[g];
        fill_grid(prm[g], G);
        G.cell_off = s->ntot;
        s->ntot += (long long)G.ncell;
        G.blk_first = s->nblk;
        G.nblk = (int)std::min<long long>((G.ncell + kFieldThreads - 1) / kFieldThreads,
                                          4ll * std::max(nsm, 1));
        s->nblk += G.nblk;
        s->hblk_grid.insert(s->hblk_grid.end(), G.nblk, g);
    }
    const long long n3 = 3 * s->ntot;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    A(cudaStreamCreateWithFlags(&s->body_stream, cudaStreamNonBlocking));
    A(cudaStreamCreateWithFlags(&s->body_stream2, cudaStreamNonBlocking));
    A(cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking));
    s->stream = s->own_stream;
    A(dalloc(&s->F, 6 * s->ntot));
    A(dalloc(&s->x, n3));
    A(dalloc(&s->r, n3));
    A(dalloc(&s->p, n3));
    A(dalloc(&s->q, n3));
    A(dalloc(&s->part, 4 * (size_t)s->nblk));
    A(dalloc(&s->cg, s->ngrids));
    A(dalloc(&s->done, s->ngrids));
    A(dalloc(&s->st, 1));
    A(dalloc(&s->tmp, s->ntot));
    A(dalloc(&s->dgrids, s->ngrids));
    A(dalloc(&s->dblk_grid, s->nblk));
    A(dalloc(&s->dsegs, 2));
    if (prm[0].precision == PIC_FP64) {
        A(dalloc(&s->J64, n3));
    } else {
        A(dalloc(&s->Jfix, n3));
        A(dalloc(&s->bvec, n3));
        A(dalloc(&s->r32, n3));
        A(dalloc(&s->p32, n3));
        A(dalloc(&s->q32, n3));
        A(dalloc(&s->e32, n3));
        A(dalloc(&s->r32b, n3));
        A(dalloc(&s->z32, n3));
        A(dalloc(&s->F32, 6 * s->ntot));
    }
    for (int k = 0; k < n; k++) s->any_nodal = s->any_nodal || (prm[k].flags & PIC_GATHER_NODAL);
    s->quads = true;
    for (int k = 0; k < n; k++) s->quads = s->quads && prm[k].nx % 4 == 0;
    if (s->any_nodal && prm[0].precision == PIC_FP64) A(dalloc(&s->Fn, 6 * s->ntot));
    if (e != cudaSuccess) {
        s->err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return bail(PIC_ENOMEM);
    }
    A(cudaMemset(s->F, 0, 6 * s->ntot * sizeof(double)));
    A(cudaMemset(s->x, 0, n3 * sizeof(double)));
    A(cudaMemset(s->r, 0, n3 * sizeof(double)));
    A(cudaMemset(s->p, 0, n3 * sizeof(double)));
    A(cudaMemset(s->q, 0, n3 * sizeof(double)));
    A(cudaMemset(s->cg, 0, s->ngrids * sizeof(CgState)));
    A(cudaMemset(s->done, 0, s->ngrids * sizeof(unsigned int)));
    A(cudaMemset(s->st, 0, sizeof(DevStatus)));
    if (s->J64) A(cudaMemset(s->J64, 0, n3 * sizeof(double)));
    if (s->Jfix) A(cudaMemset(s->Jfix, 0, n3 * sizeof(long long)));
    if (s->F32) A(cudaMemset(s->F32, 0, 6 * s->ntot * sizeof(float)));
    if (s->Fn) A(cudaMemset(s->Fn, 0, 6 * s->ntot * sizeof(double)));
    if (prm[0].precision == PIC_MIXED32 && !(prm[0].flags & (PIC_NO_COOP | PIC_EXPLICIT))) {
        const int rc = coop_create(&s->coop, s->hgrids.data(), s->ngrids, (prm[0].flags & PIC_CG_INNER) != 0,
                                   s->err);
        if (rc == PIC_ECUDA) return bail(rc);
        s->use_coop = rc == PIC_OK;
    }
    if (prm[0].precision == PIC_MIXED32) {
        int rc = mixed_create(&s->mixed, prm, s->ngrids, s->hgrids.data(), s->dgrids, s->ntot, s->F32,
                              s->Jfix, s->cg, s->st, s->err);
        if (rc != PIC_OK) return bail(rc);
    }
    A(cudaMemcpy(s->dgrids, s->hgrids.data(), s->ngrids * sizeof(GridDev), cudaMemcpyHostToDevice));
    A(cudaMemcpy(s->dblk_grid, s->hblk_grid.data(), s->nblk * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaDeviceSynchronize());
    if (e == cudaSuccess && prm[0].precision == PIC_FP64 && s->hgrids[0].inject) {
        // room for the injector's pairs even in a species that is never loaded
        for (int sp = 0; sp < 2; sp++)
            if (int rc = fp64_arrays(s, sp, inj_capacity(s->hgrids[0]), 0)) return bail(rc);
    }
    if (e != cudaSuccess) {
        s->err = std::string("initialisation failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return bail(PIC_ECUDA);
    }
    *out = s;
    return PIC_OK;
}

// ---- tile autotuning ------------------------------------------------------------------
// splitmix64 (Steele, Lea & Flood 2014) as a stateless hash: uniform double in [0, 1).
__device__ __forceinline__ double hash01(unsigned long long k) {
    k += 0x9E3779B97F4A7C15ull;
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    k ^= k >> 31;
    return (double)(k >> 11) * (1.0 / 9007199254740992.0);
}

// A timing workload shaped like a drifting pair plasma: ppc particles per cell at hashed
// offsets, u_x near sqrt(gamma0^2 - 1), transverse momenta of order 1e-3. Output
// [x(n), y(n), ux(n), uy(n), uz(n)] in physical units.
__global__ void k_synth(long long n, int nx, int ppc, double dx, double dy, double u0,
                        unsigned long long seed, double* out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long cell = k / ppc;
    const int i = (int)(cell % nx), j = (int)(cell / nx);
    const unsigned long long b = seed * 0x100000001B3ull + 8ull * (unsigned long long)k;
    out[k] = (i + hash01(b)) * dx;
    out[n + k] = (j + hash01(b + 1)) * dy;
    out[2 * n + k] = u0 + 2e-3 * (hash01(b + 2) - 0.5) * u0;
    out[3 * n + k] = 2e-3 * (hash01(b + 3) - 0.5);
    out[4 * n + k] = 2e-3 * (hash01(b + 4) - 0.5);
}

// Milliseconds per step of the tile kernels of a batch built from `sub` with synthetic
// particles (warm-up steps first); a negative value if the batch cannot be run.
double time_tiles(const std::vector<pic_params>& sub, int steps) {
    pic_sim* h = nullptr;
    if (init_handle(sub.data(), (int)sub.size(), &h) != PIC_OK) return -1.0;
    double ms = -1.0;
    long long nmax = 0;
    for (const pic_params& q : sub) nmax = std::max(nmax, (long long)q.ppc * q.nx * q.ny);
    double* d = nullptr;
    bool ok = dalloc(&d, 5 * (size_t)nmax) == cudaSuccess;
    for (int k = 0; ok && k < (int)sub.size(); k++) {
        const pic_params& q = sub[k];
        const long long n = (long long)q.ppc * q.nx * q.ny;
        ok = pic_select(h, k) == PIC_OK;
        for (int sp = 0; ok && sp < 2; sp++) {
            k_synth<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
                n, q.nx, q.ppc, q.dx, q.dy, std::sqrt(q.gamma0 * q.gamma0 - 1.0), 1000ull * k + sp, d);
            ok = pic_load_particles(h, sp, d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, n) == PIC_OK;
        }
    }
    if (d) cudaFree(d);
    double out[3] = {0, 0, 0};
    if (ok) ok = pic_step(h, 2) == PIC_OK;
    if (ok) ok = pic_profile(h, steps, out, 3) == PIC_OK;
    if (ok) ms = out[2];
    else g_init_err = h->err;
    pic_free(h);
    cudaGetLastError();
    return ms;
}

}  // namespace

// =====================================================================================
extern "C" {

void pic_params_default(pic_params* p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->nx = 64;
    p->ny = 64;
    p->dx = 1.0;
    p->dy = 1.0;
    p->cfl = 1.0;
    p->theta = 0.5;
    p->shape_order = 1;
    p->gamma0 = 20.0;
    p->ppc = 8;
    p->skin_depth = 10.0;
    p->precision = PIC_FP64;
    p->cg_rtol = 1e-10;
    p->cg_max_iter = 200;
    p->warm_start = PIC_WS_ZERO;
    p->flags = 0;
    p->tile_x = 0;
    p->tile_y = 0;
    p->bin_slack = 0.0;
    p->bc_x = PIC_BC_PERIODIC;
    p->inject_x0 = -1.0;
    p->u_th = 0.0;
    p->seed = 0;
}

int pic_init(const pic_params* prm, pic_sim** out) { return init_handle(prm, 1, out); }

int pic_init_batch(const pic_params* prm, int32_t n, pic_sim** out) {
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxBatch) return fail(nullptr, PIC_EINVAL, "n must lie in [1, 4096]");
    if (!prm) return fail(nullptr, PIC_EINVAL, "params is NULL");
    if (n > 1) {
        for (int k = 0; k < n; k++)
            if (prm[k].precision != PIC_MIXED32)
                return fail(nullptr, PIC_EINVAL, "a batch of more than one simulation requires PIC_MIXED32");
        for (int k = 1; k < n; k++)
            if ((prm[k].flags & kHandleFlags) != (prm[0].flags & kHandleFlags))
                return fail(nullptr, PIC_EINVAL,
                            "PIC_NO_GRAPH, PIC_NO_COOP, PIC_EXPLICIT and PIC_CG_INNER must be the same for "
                            "every simulation");
        for (int k = 1; k < n; k++)
            if ((prm[k].warm_start == PIC_WS_LEARNED) != (prm[0].warm_start == PIC_WS_LEARNED))
                return fail(nullptr, PIC_EINVAL, "PIC_WS_LEARNED must be used by all simulations or none");
    }
    return init_handle(prm, n, out);
}

int pic_batch_size(const pic_sim* s) { return s ? s->ngrids : 0; }

int pic_select(pic_sim* s, int32_t k) {
    if (!s) return PIC_EINVAL;
    if (k < 0 || k >= s->ngrids) return fail(s, PIC_EINVAL, "simulation index out of range");
    s->sel = k;
    return PIC_OK;
}

int pic_autotune_tiles(pic_params* prm, int32_t n, int32_t steps, double* best_ms) {
    if (!prm || n < 1 || n > kMaxBatch) return fail(nullptr, PIC_EINVAL, "need 1 <= n <= 4096 parameter sets");
    if (steps < 1 || steps > 1000) return fail(nullptr, PIC_EINVAL, "steps must lie in [1, 1000]");
    std::string why;
    for (int k = 0; k < n; k++) {
        pic_params q = prm[k];
        q.precision = PIC_MIXED32;
        if (validate(&q, why) != PIC_OK) return fail(nullptr, PIC_EINVAL, "simulation " + std::to_string(k) + ": " + why);
    }
    static const int cand[][2] = {{32, 16}, {16, 16}, {32, 8}, {64, 8}, {64, 16}, {16, 8}, {32, 32}};
    for (int P = 1; P <= 3; P++) {
        std::vector<int> idx;
        for (int k = 0; k < n; k++)
            if (prm[k].shape_order == P) idx.push_back(k);
        if (best_ms) best_ms[P - 1] = 0.0;
        if (idx.empty()) continue;
        double best = -1.0;
        int bx = 0, by = 0;
        std::vector<std::vector<int>> seen;
        for (const auto& c : cand) {
            std::vector<pic_params> sub;
            std::vector<int> eff;
            bool fits = true;
            for (int k : idx) {
                pic_params q = prm[k];
                q.precision = PIC_MIXED32;
                q.flags &= ~PIC_NO_GRAPH;
                if (q.warm_start == PIC_WS_LEARNED) q.warm_start = PIC_WS_ZERO;  // the tiles do not see it
                q.tile_x = c[0];
                q.tile_y = c[1];
                const int tx = std::min(c[0], q.nx), ty = std::min(c[1], q.ny);
                if ((tx + 5) * (ty + 5) > kMaxWinCells) fits = false;
                eff.push_back(tx);
                eff.push_back(ty);
                sub.push_back(q);
            }
            if (!fits || std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
            seen.push_back(eff);
            const double ms = time_tiles(sub, steps);
            if (ms > 0 && (best < 0 || ms < best)) {
                best = ms;
                bx = c[0];
                by = c[1];
            }
        }
        if (best < 0) return fail(nullptr, PIC_ECUDA, "no tile shape could be timed (" + g_init_err + ")");
        for (int k : idx) {
            prm[k].tile_x = bx;
            prm[k].tile_y = by;
        }
        if (best_ms) best_ms[P - 1] = best;
    }
    return PIC_OK;
}

int pic_set_cnn(pic_sim* s, const pic_cnn* net) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (!net) return fail(s, PIC_EINVAL, "network is NULL");
    if (s->prm.precision != PIC_MIXED32) return fail(s, PIC_EINVAL, "the learned warm start needs PIC_MIXED32");
    CK(cudaStreamSynchronize(s->stream));
    drop_graph(s);
    int rc = cnn_make_guess(net, s->hgrids.data(), s->ngrids, &s->guess, s->err);
    if (rc) return rc;
    s->has_cnn = true;
    return PIC_OK;
}

int pic_set_stream(pic_sim* s, void* stream) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    s->stream = stream ? (cudaStream_t)stream : s->own_stream;
    return PIC_OK;
}

int pic_load_particles(pic_sim* s, int32_t sp, const double* x, const double* y, const double* ux,
                       const double* uy, const double* uz, int64_t n) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (int rc = check_species(s, sp)) return rc;
    if (n < 0) return fail(s, PIC_EINVAL, "n must be >= 0");
    if (n > 0 && (!x || !y || !ux || !uy || !uz)) return fail(s, PIC_EINVAL, "NULL particle array");
    if (n > (int64_t)1 << 40) return fail(s, PIC_EINVAL, "n too large");
    drop_graph(s);
    if (s->prm.precision == PIC_MIXED32) {
        int rc = mixed_load(s->mixed, s->sel, sp, x, y, ux, uy, uz, n, s->stream, s->err);
        if (rc == PIC_OK) rc = finish_call(s);
        return rc;
    }
    // FP64: arrays for n particles (plus what the injector can add)
    s->np[sp] = 0;
    if (int rc = fp64_arrays(s, sp, n + inj_capacity(s->hgrids[0]), 0)) return rc;
    const double* src[5] = {x, y, ux, uy, uz};
    for (int a = 0; a < 5; a++)
        if (n) CK(cudaMemcpyAsync(s->pa[sp][a], src[a], n * sizeof(double), cudaMemcpyDefault, s->stream));
    unsigned long long* nbad = (unsigned long long*)s->tmp;
    CK(cudaMemsetAsync(nbad, 0, sizeof(unsigned long long), s->stream));
    const GridDev& G = s->hgrids[0];
    if (n) {
        k_load_fp64<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(
            n, s->pa[sp][0], s->pa[sp][1], s->pa[sp][2], s->pa[sp][3], s->pa[sp][4], G.nx * G.dx,
            G.ny * G.dy, G.idx, G.idy, G.nx, G.ny, G.walls, nbad);
    }
    unsigned long long hbad = 0;
    CK(cudaMemcpyAsync(&hbad, nbad, sizeof hbad, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (hbad) {
        s->np[sp] = 0;
        fp64_arrays(s, sp, 0, 0);
        return fail(s, PIC_EINVAL, "non-finite particle position or momentum, or a position outside the walls");
    }
    return fp64_arrays(s, sp, 0, n);
}

int pic_set_fields(pic_sim* s, int32_t which, const double* data, size_t len) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (which < PIC_EX || which > PIC_BZ) return fail(s, PIC_EINVAL, "which must be PIC_EX..PIC_BZ");
    const GridDev& G = s->hgrids[s->sel];
    if (!data || len < (size_t)G.ncell) return fail(s, PIC_EINVAL, "data must hold nx*ny values");
    CK(cudaMemcpyAsync(s->F + which * s->ntot + G.cell_off, data, G.ncell * sizeof(double),
                       cudaMemcpyDefault, s->stream));
    if (G.walls && (which == PIC_EY || which == PIC_EZ || which == PIC_BX))  // zero on the wall
        CK(cudaMemset2DAsync(s->F + which * s->ntot + G.cell_off, G.nx * sizeof(double), 0, sizeof(double),
                             G.ny, s->stream));
    launch_fields_to_f32(field_args(s, 0, 0), s->stream);
    return finish_call(s);
}

namespace {

// MIXED32 runs a call in chunks of this many steps: particles that found no room in their
// tile's bin wait in the overflow list (pushed from global memory, far slower) until the
// host re-sorts them into larger bins after a chunk.
constexpr int kStepChunk = 32;

int step_chunk(pic_sim* s, int32_t n) {
    // a new chunk starts clean: errors stop the rest of the chunk that raised them, and
    // the call returns
    DevStatus hs{};
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const unsigned long long steps0 = hs.steps_done;
    const unsigned long long li0 = hs.loop_iters[0], lr0 = hs.loop_iters[1];
    hs.stop = 0;
    hs.stop_next = 0;
    CK(cudaMemcpyAsync(s->st, &hs, sizeof hs, cudaMemcpyHostToDevice, s->stream));
    if (s->prm.precision == PIC_MIXED32) {
        int rc = mixed_before_steps(s->mixed, s->stream, s->err);
        if (rc) return rc;
    }
    const bool graph = !(s->prm.flags & PIC_NO_GRAPH);
    check_graph_generation(s);
    if (graph && !s->gexec) {
        if (int rc = build_graph(s)) return rc;
    }
    const long long per_step = step_kernels(s, graph);
    for (int k = 0; k < n; k++) {
        if (graph) {
            CK(cudaGraphLaunch(s->gexec, s->stream));
        } else {
            if (int rc = run_step_direct(s)) return rc;
        }
    }
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    if (int rc = finish_call(s)) return rc;
    s->steps += (long long)(hs.steps_done - steps0);
    s->kernels += n * per_step + loop_kernels(s, hs.loop_iters[0] - li0, hs.loop_iters[1] - lr0);
    if (int rc0 = fp64_counts(s)) return rc0;
    int rc = device_errors(s, hs);
    if (rc == PIC_OK && s->prm.precision == PIC_MIXED32) rc = mixed_after_steps(s->mixed, s->stream, s->err);
    return rc;
}

}  // namespace

int pic_set_wait_limit(pic_sim* s, int32_t spins) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (spins < 0) return fail(s, PIC_EINVAL, "spins must be >= 0");
    DevStatus hs{};
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    hs.spin_limit = (unsigned int)spins;
    CK(cudaMemcpyAsync(s->st, &hs, sizeof hs, cudaMemcpyHostToDevice, s->stream));
    return finish_call(s);
}

int pic_step(pic_sim* s, int32_t n) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (n < 0) return fail(s, PIC_EINVAL, "n must be >= 0");
    if (n == 0) return PIC_OK;
    if (s->learned && !s->has_cnn) return fail(s, PIC_ESTATE, "PIC_WS_LEARNED needs a network (pic_set_cnn)");
    const int chunk = s->prm.precision == PIC_MIXED32 ? kStepChunk : n;
    for (int done = 0; done < n;) {
        const int m = std::min(chunk, n - done);
        if (int rc = step_chunk(s, m)) return rc;
        done += m;
    }
    return PIC_OK;
}

namespace {

// n profiled steps; per-phase times and PCG iterations are added into acc[0..4].
int profile_chunk(pic_sim* s, int32_t n, double* acc) {
    for (int k = 0; k < 6; k++)
        if (!s->ev[k]) CK(cudaEventCreate(&s->ev[k]));
    if (s->prm.precision == PIC_MIXED32) {
        int rc = mixed_before_steps(s->mixed, s->stream, s->err);
        if (rc) return rc;
    }
    check_graph_generation(s);
    for (int k = 0; k < kNumParts; k++)
        if (!s->pexec[k])
            if (int rc = capture(s, 1 << k, &s->pgraph[k], &s->pexec[k])) return rc;
    CgState c0{}, c1{};
    DevStatus hs{};
    CK(cudaMemcpyAsync(&c0, s->cg + s->sel, sizeof c0, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const unsigned long long steps0 = hs.steps_done;
    const unsigned long long li0 = hs.loop_iters[0], lr0 = hs.loop_iters[1];
    hs.stop = 0;
    hs.stop_next = 0;
    CK(cudaMemcpyAsync(s->st, &hs, sizeof hs, cudaMemcpyHostToDevice, s->stream));
    for (int k = 0; k < n; k++) {
        for (int part = 0; part < kNumParts; part++) {
            CK(cudaEventRecord(s->ev[part], s->stream));
            CK(cudaGraphLaunch(s->pexec[part], s->stream));
        }
        CK(cudaEventRecord(s->ev[5], s->stream));
        CK(cudaStreamSynchronize(s->stream));
        float t[5];
        CK(cudaEventElapsedTime(&t[0], s->ev[0], s->ev[5]));  // whole step
        CK(cudaEventElapsedTime(&t[1], s->ev[0], s->ev[3]));  // particle half
        CK(cudaEventElapsedTime(&t[2], s->ev[1], s->ev[2]));  // dominant particle kernel
        CK(cudaEventElapsedTime(&t[3], s->ev[3], s->ev[4]));  // field solve
        for (int a = 0; a < 4; a++) acc[a] += t[a];
    }
    CK(cudaMemcpyAsync(&c1, s->cg + s->sel, sizeof c1, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->steps += (long long)(hs.steps_done - steps0);
    s->kernels += n * step_kernels(s, false) + loop_kernels(s, hs.loop_iters[0] - li0, hs.loop_iters[1] - lr0);
    if (int rc0 = fp64_counts(s)) return rc0;
    acc[4] += (double)(c1.total_iters - c0.total_iters);
    int rc = device_errors(s, hs);
    if (rc == PIC_OK && s->prm.precision == PIC_MIXED32) rc = mixed_after_steps(s->mixed, s->stream, s->err);
    return rc;
}

}  // namespace

int pic_profile(pic_sim* s, int32_t n, double* out, int32_t n_out) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (n < 1 || !out || n_out < 1) return fail(s, PIC_EINVAL, "need n >= 1 and an output array");
    if (s->learned && !s->has_cnn) return fail(s, PIC_ESTATE, "PIC_WS_LEARNED needs a network (pic_set_cnn)");
    double acc[5] = {0, 0, 0, 0, 0};
    const int chunk = s->prm.precision == PIC_MIXED32 ? kStepChunk : n;  // as pic_step
    for (int done = 0; done < n;) {
        const int m = std::min(chunk, n - done);
        if (int rc = profile_chunk(s, m, acc)) return rc;
        done += m;
    }
    for (int a = 0; a < n_out && a < 5; a++) out[a] = acc[a] / n;
    return PIC_OK;
}

namespace {

// Device pointer to grid quantity `which` of the selected simulation (J, rho: converted
// into s->tmp).
int field_source(pic_sim* s, int32_t which, const double** out_src) {
    if (which < PIC_EX || which > PIC_DENSITY_E) return fail(s, PIC_EINVAL, "which must be PIC_EX..PIC_DENSITY_E");
    if (which >= PIC_RHSX && which <= PIC_RHSZ && !s->bvec)
        return fail(s, PIC_ESTATE, "the right-hand side is kept in PIC_MIXED32 only");
    const GridDev& G = s->hgrids[s->sel];
    const long long nc = G.ncell, off = G.cell_off;
    const double* src = nullptr;
    if (which <= PIC_BZ) {
        src = s->F + which * s->ntot + off;
    } else if (which <= PIC_JZ) {
        const int c = which - PIC_JX;
        if (s->J64) {
            src = s->J64 + c * s->ntot + off;
        } else {
            k_fix_to_f64<<<(unsigned)((nc + 255) / 256), 256, 0, s->stream>>>(
                nc, s->Jfix + c * s->ntot + off, G.jinv, s->tmp);
            src = s->tmp;
        }
    } else if (which <= PIC_DBZ) {
        src = s->x + (which - PIC_DBX) * s->ntot + off;
    } else if (which <= PIC_RHSZ) {
        src = s->bvec + (which - PIC_RHSX) * s->ntot + off;
    } else {
        if (int rc = charge_density(s, s->tmp, nullptr, which)) return rc;
        src = s->tmp;
    }
    *out_src = src;
    return PIC_OK;
}

}  // namespace

int pic_fields(pic_sim* s, int32_t which, double* out, size_t len) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    const long long nc = s->hgrids[s->sel].ncell;
    if (!out || len < (size_t)nc) return fail(s, PIC_EINVAL, "out must hold nx*ny values");
    const double* src = nullptr;
    if (int rc = field_source(s, which, &src)) return rc;
    CK(cudaMemcpyAsync(out, src, nc * sizeof(double), cudaMemcpyDefault, s->stream));
    return finish_call(s);
}

int pic_spectrum(pic_sim* s, int32_t which, double* out, size_t len) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    const GridDev& G = s->hgrids[s->sel];
    const long long nc = G.ncell;
    if (!out || len < (size_t)nc) return fail(s, PIC_EINVAL, "out must hold nx*ny values");
    const double* src = nullptr;
    if (int rc = field_source(s, which, &src)) return rc;
    double* dout = nullptr;
    CK(dalloc(&dout, nc));
    int rc = spectrum_2d(src, G.nx, G.ny, dout, s->stream, s->err);
    if (rc == PIC_OK) {
        cudaError_t e = cudaMemcpyAsync(out, dout, nc * sizeof(double), cudaMemcpyDefault, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = fail(s, PIC_ECUDA, std::string("pic_spectrum: ") + cudaGetErrorString(e));
    }
    cudaFree(dout);
    if (rc) return rc;
    return finish_call(s);
}

int pic_resonance_ky(double cfl_x, double cfl_y, double beta, double kx_dx, double* ky_dy) {
    if (!ky_dy || !(cfl_x > 0.0) || !(cfl_y > 0.0) || !(beta > 0.0 && beta < 1.0) || !(kx_dx > 0.0 && kx_dx <= kPi))
        return PIC_EINVAL;
    const double a = 0.5 * beta * cfl_x * kx_dx;  // V k_x dt / 2
    if (a >= 0.5 * kPi) return PIC_EINVAL;
    const double t = std::tan(a), sx = cfl_x * std::sin(0.5 * kx_dx);
    const double d = t * t - sx * sx;
    if (d < 0.0) return PIC_EINVAL;
    const double arg = std::sqrt(d) / cfl_y;
    if (arg > 1.0) return PIC_EINVAL;
    *ky_dy = 2.0 * std::asin(arg);
    return PIC_OK;
}

int pic_moments(pic_sim* s, pic_moments_t* m) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (!m) return fail(s, PIC_EINVAL, "out is NULL");
    CgState c{};
    DevStatus hs{};
    CK(cudaMemcpyAsync(&c, s->cg + s->sel, sizeof c, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    if (int rc = finish_call(s)) return rc;
    memset(m, 0, sizeof *m);
    const GridDev& G = s->hgrids[s->sel];
    m->step = s->steps;
    m->time = s->steps * G.dt;
    m->U_E = c.ue;
    m->U_B = c.ub;
    m->U_K = c.uk;
    m->macro_weight = G.w;
    m->n_particles[0] = pic_particle_count(s, 0);
    m->n_particles[1] = pic_particle_count(s, 1);
    m->cg_iters_last = c.last_iters;
    m->cg_iters_max = c.max_iters;
    m->cg_iters_total = c.total_iters;
    m->cg_rel_resid = c.rel;
    m->cfl_violations = (int64_t)hs.cfl_viol;
    m->overflow_moves = (int64_t)hs.overflow;
    if (s->mixed) m->rebins = mixed_rebins(s->mixed);
    m->cg_refinements = c.total_outer;
    m->loop_iters = (int64_t)hs.loop_iters[0];
    m->loop_refinements = (int64_t)hs.loop_iters[1];
    m->kernel_launches = s->kernels;
    // the largest-iteration counter restarts at every pic_moments call
    const int zero = 0;
    CK(cudaMemcpyAsync(&s->cg[s->sel].max_iters, &zero, sizeof zero, cudaMemcpyHostToDevice, s->stream));
    return finish_call(s);
}

int64_t pic_particle_count(pic_sim* s, int32_t sp) {
    if (!s || sp < 0 || sp > 1) return -1;
    if (s->mixed) return mixed_count(s->mixed, s->sel, sp);
    return s->np[sp];
}

int pic_particles(pic_sim* s, int32_t sp, double* out, int64_t n) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (int rc = check_species(s, sp)) return rc;
    if (n != pic_particle_count(s, sp)) return fail(s, PIC_EINVAL, "n must equal pic_particle_count");
    if (n == 0) return PIC_OK;
    if (!out) return fail(s, PIC_EINVAL, "out is NULL");
    if (s->mixed) {
        int rc = mixed_particles(s->mixed, s->sel, sp, out, n, s->stream, s->err);
        if (rc == PIC_OK) rc = finish_call(s);
        return rc;
    }
    const GridDev& G = s->hgrids[0];
    double* t = nullptr;
    CK(dalloc(&t, 2 * (size_t)n));
    k_unload_fp64<<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(n, s->pa[sp][0], s->pa[sp][1],
                                                                      G.dx, G.dy, t, t + n);
    cudaError_t e = cudaMemcpyAsync(out, t, 2 * n * sizeof(double), cudaMemcpyDefault, s->stream);
    for (int a = 2; a < 5 && e == cudaSuccess; a++)
        e = cudaMemcpyAsync(out + a * n, s->pa[sp][a], n * sizeof(double), cudaMemcpyDefault, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(t);
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, std::string("pic_particles: ") + cudaGetErrorString(e));
    return PIC_OK;
}

int pic_conservation(pic_sim* s, double* out, int32_t n_out) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (!out || n_out < 1) return fail(s, PIC_EINVAL, "out is NULL");
    const GridDev& G = s->hgrids[s->sel];
    double* mom = nullptr;
    CK(dalloc(&mom, 3));
    CK(cudaMemsetAsync(mom, 0, 3 * sizeof(double), s->stream));
    int rc = charge_density(s, s->tmp, mom);
    const long long nc = G.ncell;
    std::vector<double> rho(nc), ex(nc), ey(nc);
    double hm[3] = {0, 0, 0};
    if (rc == PIC_OK) {
        cudaError_t e = cudaMemcpyAsync(rho.data(), s->tmp, nc * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ex.data(), s->F + G.cell_off, nc * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ey.data(), s->F + s->ntot + G.cell_off, nc * sizeof(double), cudaMemcpyDeviceToHost,
                                s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hm, mom, sizeof hm, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) rc = fail(s, PIC_ECUDA, std::string("pic_conservation: ") + cudaGetErrorString(e));
    }
    cudaFree(mom);
    if (rc) return rc;
    // Gauss's law on the nodes: div E - 4 pi rho (off the wall column with walls, where
    // the conductor holds the surface charge)
    double q = 0.0, mx = 0.0, ss = 0.0;
    long long cnt = 0;
    for (int j = 0; j < G.ny; j++)
        for (int i = 0; i < G.nx; i++) {
            const long long k = (long long)j * G.nx + i;
            q += rho[k] * G.dx * G.dy;
            if (G.walls && i == 0) continue;
            const double exw = ex[(long long)j * G.nx + (i == 0 ? G.nx - 1 : i - 1)];
            const double eys = ey[(long long)(j == 0 ? G.ny - 1 : j - 1) * G.nx + i];
            const double r = (ex[k] - exw) * G.idx + (ey[k] - eys) * G.idy - 4.0 * kPi * rho[k];
            mx = std::max(mx, std::fabs(r));
            ss += r * r;
            cnt++;
        }
    const double vals[6] = {hm[0], hm[1], hm[2], q, mx, cnt ? std::sqrt(ss / cnt) : 0.0};
    for (int k = 0; k < n_out && k < 6; k++) out[k] = vals[k];
    return PIC_OK;
}

// ---- checkpoints ----------------------------------------------------------------------
namespace {
constexpr char kSaveMagic[8] = {'P', 'I', 'C', 'S', 'T', 'A', 'T', 'E'};
constexpr int32_t kSaveVersion = 1;

bool same_problem(const pic_params& a, const pic_params& b) {
    return a.nx == b.nx && a.ny == b.ny && a.dx == b.dx && a.dy == b.dy && a.cfl == b.cfl &&
           a.theta == b.theta && a.shape_order == b.shape_order && a.gamma0 == b.gamma0 && a.ppc == b.ppc &&
           a.skin_depth == b.skin_depth && a.precision == b.precision && a.bc_x == b.bc_x &&
           a.inject_x0 == b.inject_x0 && a.u_th == b.u_th && a.seed == b.seed;
}
}  // namespace

int pic_save(pic_sim* s, const char* path) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (!path) return fail(s, PIC_EINVAL, "path is NULL");
    DevStatus hs{};
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(s, PIC_EINVAL, std::string("cannot open ") + path + " for writing");
    const int sel0 = s->sel;
    int rc = PIC_OK;
    bool ok = fwrite(kSaveMagic, 1, 8, f) == 8;
    const int32_t head[3] = {kSaveVersion, s->ngrids, s->prm.precision};
    const int64_t steps[2] = {s->steps, (int64_t)hs.steps_done};
    ok = ok && fwrite(head, sizeof head, 1, f) == 1 && fwrite(steps, sizeof steps, 1, f) == 1;
    for (int g = 0; ok && rc == PIC_OK && g < s->ngrids; g++) {
        s->sel = g;
        const GridDev& G = s->hgrids[g];
        ok = fwrite(&s->prms[g], sizeof(pic_params), 1, f) == 1;
        std::vector<double> buf((size_t)G.ncell);
        for (int c = 0; ok && c < 9; c++) {  // E, B, then the last dB (warm start)
            const double* src = c < 6 ? s->F + c * s->ntot + G.cell_off : s->x + (c - 6) * s->ntot + G.cell_off;
            if (cudaMemcpy(buf.data(), src, G.ncell * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = fail(s, PIC_ECUDA, "pic_save: field copy failed");
                break;
            }
            ok = fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
        }
        for (int sp = 0; ok && rc == PIC_OK && sp < 2; sp++) {
            const int64_t n = pic_particle_count(s, sp);
            std::vector<double> p((size_t)std::max<int64_t>(1, 5 * n));
            if (n) rc = pic_particles(s, sp, p.data(), n);
            ok = ok && fwrite(&n, sizeof n, 1, f) == 1 && (n == 0 || fwrite(p.data(), sizeof(double), 5 * n, f) == (size_t)(5 * n));
        }
    }
    s->sel = sel0;
    if (fclose(f) != 0) ok = false;
    if (rc) return rc;
    if (!ok) return fail(s, PIC_EINVAL, std::string("write to ") + path + " failed");
    return PIC_OK;
}

int pic_restore(pic_sim* s, const char* path) {
    if (!s) return PIC_EINVAL;
    cudaSetDevice(s->device);
    if (!path) return fail(s, PIC_EINVAL, "path is NULL");
    // the whole file is read and checked before anything on the handle changes
    struct Saved {
        std::vector<double> fields;     // 9 x ncell: E, B, dB
        std::vector<double> parts[2];   // 5 x n each
        int64_t n[2];
    };
    std::vector<Saved> saved((size_t)s->ngrids);
    int64_t steps[2];
    {
        FILE* f = fopen(path, "rb");
        if (!f) return fail(s, PIC_EINVAL, std::string("cannot open ") + path);
        std::string why;
        char magic[8];
        int32_t head[3];
        if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kSaveMagic, 8) != 0) why = "not a checkpoint file";
        else if (fread(head, sizeof head, 1, f) != 1 || head[0] != kSaveVersion) why = "unknown checkpoint version";
        else if (head[1] != s->ngrids || head[2] != s->prm.precision) why = "checkpoint of a different handle";
        else if (fread(steps, sizeof steps, 1, f) != 1 || steps[0] < 0 || steps[1] < 0) why = "truncated file";
        for (int g = 0; why.empty() && g < s->ngrids; g++) {
            pic_params p{};
            if (fread(&p, sizeof p, 1, f) != 1) { why = "truncated file"; break; }
            if (!same_problem(p, s->prms[g])) { why = "simulation " + std::to_string(g) + " has other parameters"; break; }
            Saved& v = saved[g];
            const size_t nc = (size_t)s->hgrids[g].ncell;
            v.fields.resize(9 * nc);
            if (fread(v.fields.data(), sizeof(double), 9 * nc, f) != 9 * nc) { why = "truncated file"; break; }
            for (int sp = 0; why.empty() && sp < 2; sp++) {
                if (fread(&v.n[sp], sizeof(int64_t), 1, f) != 1 || v.n[sp] < 0 || v.n[sp] > ((int64_t)1 << 40)) {
                    why = "truncated file";
                    break;
                }
                v.parts[sp].resize((size_t)(5 * v.n[sp]));
                if (fread(v.parts[sp].data(), sizeof(double), v.parts[sp].size(), f) != v.parts[sp].size())
                    why = "truncated file";
            }
        }
        fclose(f);
        if (!why.empty()) return fail(s, PIC_EINVAL, "pic_restore: " + why);
    }
    const int sel0 = s->sel;
    int rc = PIC_OK;
    for (int g = 0; g < s->ngrids && rc == PIC_OK; g++) {
        const GridDev& G = s->hgrids[g];
        for (int c = 0; c < 9; c++) {
            double* dst = c < 6 ? s->F + c * s->ntot + G.cell_off : s->x + (c - 6) * s->ntot + G.cell_off;
            CK(cudaMemcpyAsync(dst, saved[g].fields.data() + c * G.ncell, G.ncell * sizeof(double),
                               cudaMemcpyHostToDevice, s->stream));
        }
        s->sel = g;
        for (int sp = 0; sp < 2 && rc == PIC_OK; sp++) {
            const double* pp = saved[g].parts[sp].data();
            const int64_t n = saved[g].n[sp];
            rc = pic_load_particles(s, sp, pp, pp + n, pp + 2 * n, pp + 3 * n, pp + 4 * n, n);
        }
    }
    s->sel = sel0;
    if (rc) return rc;
    // step counters (the injector's schedule follows them) and the FP32 field copies
    DevStatus hs{};
    CK(cudaMemcpyAsync(&hs, s->st, sizeof hs, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    hs.steps_done = (unsigned long long)steps[1];
    CK(cudaMemcpyAsync(s->st, &hs, sizeof hs, cudaMemcpyHostToDevice, s->stream));
    s->steps = steps[0];
    launch_fields_to_f32(field_args(s, 0, 0), s->stream);
    return finish_call(s);
}

const char* pic_last_error(const pic_sim* s) {
    return s ? s->err.c_str() : g_init_err.c_str();
}

void pic_free(pic_sim* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graph(s);
    if (s->mixed) mixed_destroy(s->mixed);
    cnn_free_guess(&s->guess);
    coop_free(&s->coop);
    void* ptrs[] = {s->dgrids, s->dblk_grid, s->F, s->J64, s->Jfix, s->F32, s->Fn, s->x, s->r, s->p, s->q,
                    s->part, s->cg, s->done, s->st, s->tmp, s->dsegs, s->dblk_seg[0], s->dblk_seg[1],
                    s->bvec, s->r32, s->p32, s->q32, s->e32, s->r32b, s->z32};
    for (void* p : ptrs) dfree(p);
    for (int sp = 0; sp < 2; sp++)
        for (int a = 0; a < 5; a++) dfree(s->pa[sp][a]);
    if (s->body_stream) cudaStreamDestroy(s->body_stream);
    if (s->body_stream2) cudaStreamDestroy(s->body_stream2);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    for (int k = 0; k < 6; k++)
        if (s->ev[k]) cudaEventDestroy(s->ev[k]);
    delete s;
}

}  // extern "C"

// ---- check of the FP32-pair building blocks (include/pic.h) ----------------------------
static __global__ void k_dword_check(const double* x, const long long* d, long long n, float* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = x[i], b = x[(i + 1) % n];
    const pic::DW pa = pic::dw_from(a), pb = pic::dw_from(b), pk = pic::dw_from_i64(d[i]);
    const pic::DW s = pic::dw_add(pa, pb), m = pic::dw_mul(pa, pb);
    float* o = out + 10 * i;
    o[0] = pa.h;
    o[1] = pa.l;
    o[2] = pic::f32_rn(a);
    o[3] = pk.h;
    o[4] = pk.l;
    o[5] = s.h;
    o[6] = s.l;
    o[7] = m.h;
    o[8] = m.l;
    o[9] = (float)(pic::dw_join(pa) - a);
}

int pic_dword_check(const double* x, const int64_t* d, int64_t n, float* out) {
    if (!x || !d || !out || n < 1 || n > (1ll << 24)) return fail(nullptr, PIC_EINVAL, "bad arguments");
    double* dx = nullptr;
    long long* dd = nullptr;
    float* dout = nullptr;
    cudaError_t e = cudaMalloc(&dx, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dd, n * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&dout, 10 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dd, d, n * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_dword_check<<<(unsigned)((n + 255) / 256), 256>>>(dx, dd, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 10 * n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dd);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, std::string("pic_dword_check: ") + cudaGetErrorString(e));
    return PIC_OK;
}
