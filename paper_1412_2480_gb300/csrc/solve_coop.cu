// solve_coop.cu -- the MIXED32 solve of Eq. (7) as one persistent cooperative kernel.
//
// After the right-hand side b and the initial residual r = b - A x0 (FP64), the whole
// mixed-precision PCG runs inside one launch: iterative refinement in FP64 around an
// FP32 inner preconditioned CG on A e = r, as the WHILE-node version in fields.cu does,
// but with grid barriers between the phases of an iteration instead of kernel
// boundaries, so an inner iteration costs two barriers and two passes over L2-resident
// FP32 vectors.
//
// Inner PCG with z = M r (M = p(A), GridDev::pc0..pcy), per iteration:
//   direction pass: p = z + beta p, q = A z + beta q (= A p), partial (p, q)  -> alpha
//   update pass:    r' = r - alpha q, e += alpha p, z = M r', partials (r', r'), (r', z)
//                   -> beta = (r', z) / (r, z)
// The update pass forms M r' at a cell from r and q at its four neighbours (r' there is
// r - alpha q, both unchanged in this pass), so r' goes to the other of two residual
// buffers and no third barrier is needed.
//
// By default the inner solve is instead a Chebyshev iteration, done tile by tile with
// no grid-wide step at all: A's spectrum lies in [c0 - 2 (cx + cy), c0 + 2 (cx + cy)]
// (Gershgorin; the interval is exact for periodic boxes and holds with the wall images,
// which keep A symmetric positive definite), so m steps of the three-term Chebyshev
// recurrence on that interval reduce every error component by 1/T_m(sigma),
// sigma = c0 / (2 (cx + cy)) >= 5/4 here, with no inner products. Step k at a cell needs
// step k-1 at its four neighbours, so a tile of 32 x 64 cells loaded with a halo of 12
// >= m - 1 cells in shared memory computes all m steps by itself (the halo's outer ring
// goes stale one cell per step and never reaches the interior) and adds its interior's
// correction to x. m is chosen per refinement from the reduction it needs (as the CG's
// inner tolerance is), at most 13 (1/T_13(2) = 7e-8 at CFL 1, theta 1/2, near the FP32
// floor). During the solve x is held as FP32 pairs and the residual pass runs in pair
// arithmetic (dword.cuh), so no FP64 instruction is spent inside a refinement; x is
// joined back to FP64 at the end. A refinement costs two grid barriers (tiles,
// residual) instead of two per inner iteration. PIC_CG_INNER, or a simulation's
// cg_rtol below 1e-13, keeps the CG.
//
// Work is cut into fixed chunks of 2048 cells of one simulation; a chunk's partial sums
// are formed in a fixed order and written to its own slot, and every CTA forms each
// simulation's sums from its chunk partials in a fixed order. Results therefore depend
// neither on the number of CTAs nor on the other simulations of a batch: every CTA
// holds the same per-simulation scalars (alpha, beta, tolerances, convergence flags)
// without a further exchange.
#include <algorithm>
#include <string>
#include <vector>

#include "dword.cuh"
#include "engine.h"
#include "pic.h"

namespace pic {

namespace {

constexpr int kCoopThreads = 256;
constexpr int kChunkCells = 2048;
constexpr int kPerThread = kChunkCells / kCoopThreads;
constexpr int kInnerMax = 64;  // inner iterations per refinement, as in the WHILE-node solve
constexpr int kCoopMaxChunks = 4096;  // two partials per chunk staged in shared memory: 64 KB

// Chebyshev inner solve: interior tile (32 x 64 cells), most steps per solve (the
// window's halo is kChebMaxIt - 1 cells on every side, whatever the steps), the window
// (56 x 88 cells: 4 strips of 22 rows, one column per thread, 224 threads), its row
// pitch and height in shared memory with a ring of zero ghost cells, one buffer's size.
constexpr int kChebTileX = 32;
constexpr int kChebTileY = 64;
constexpr int kChebMaxIt = 13;
constexpr int kChebHalo = kChebMaxIt - 1;
constexpr int kChebW = kChebTileX + 2 * kChebHalo;
constexpr int kChebH = kChebTileY + 2 * kChebHalo;
constexpr int kChebStrips = 4;
constexpr int kChebRows = kChebH / kChebStrips;
constexpr int kChebPitch = kChebW + 2;
constexpr int kChebCells = kChebPitch * (kChebH + 2);
constexpr int kChebTileCells = kChebTileX * kChebTileY;  // the interior, staged for the x update
static_assert(kChebRows * kChebStrips == kChebH && kChebW * kChebStrips <= kCoopThreads, "window layout");
constexpr double kChebFloor = 1e-7;
constexpr double kChebRtolMin = 1e-13;  // the FP32-pair residual resolves about 1e-14 of ||b||
constexpr double kChebWorst = 1e-3;

struct CoopArgs {
    const GridDev* grids;
    int ngrids;
    const int2* gchunk;     // per simulation: first chunk, chunk count
    const int* chunk_grid;  // per chunk: simulation
    int nchunks;
    const int* tile_grid;   // Chebyshev tiles: simulation, first cell (x, y)
    const int2* tile_xy;
    int ntiles;
    long long ntot;
    const double* b;
    double* x;
    double* r;
    float* r32[2];          // the inner residual, alternating between update passes
    float* z32;             // M r
    float* p32;
    float* q32;
    float* e32;
    double* part;           // 2 buffers x 2 values x nchunks, alternating between phases
    unsigned int* bar;      // [0] arrivals, [1] generation
    CgState* cg;
    DevStatus* st;
};

struct GState {
    double rr, bb, scale, rr_in0, rr_in, rz, alpha, beta, tol_in, rel, rtol;
    int active, in_active, iters, in_iters, outer, maxit;
    int cheb, m;  // inner solve by the Chebyshev iteration; its steps this refinement
    int dw;       // x is held as FP32 pairs in (p32, q32) until the final join
    float sig;    // c0 / (2 (cx + cy))
    // FP32 and pair forms of the simulation's constants and of the refinement's scale,
    // formed by one thread per simulation: on this part every FP64 operation (a
    // conversion included) costs as much as ~100 FP32 ones, too much to repeat per thread
    float c0f, cxf, cyf, pc0f, pcxf, pcyf, scf, invf, alphaf, betaf;
    double inv;
    DW C0, CX, CY;
};

// Grid-wide barrier of a cooperative launch (all CTAs resident): arrivals on one counter
// (word 0), release by advancing the generation (word 1). Bounded: false if the other
// CTAs did not arrive within `limit` polls; the CTA then leaves the kernel, and so do
// the others at their next barrier (none waits for ever). (A two-level tree of
// counters was slower here.)
constexpr int kBarWords = 2;

__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned int* timeout, unsigned int limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        const unsigned int g0 = *gen;
        int ok = 1;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1u) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned int it = 0;
            while (*gen == g0) {
                if (++it > limit) {
                    atomicExch(timeout, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum of one simulation's chunk partials (staged in shared memory), by one warp, in a
// fixed order.
__device__ __forceinline__ double chunk_sum(const double* sp, int2 gc) {
    double s = 0.0;
    for (int k = threadIdx.x & 31; k < gc.y; k += 32) s += sp[gc.x + k];
    return warp_sum(s);
}

// All chunk partials into shared memory, eight independent loads in flight per thread.
__device__ __forceinline__ void stage_partials(const double* part, int n, double* sp) {
    for (int base = 0; base < n; base += 8 * kCoopThreads) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = base + u * kCoopThreads + threadIdx.x;
            v[u] = k < n ? __ldcg(part + k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = base + u * kCoopThreads + threadIdx.x;
            if (k < n) sp[k] = v[u];
        }
    }
    __syncthreads();
}

enum Phase { kBegin, kDirection, kUpdate, kX, kResidual, kJoin, kResidualDW };

// Per-chunk constants, in registers.
struct ChunkC {
    int nx, ny, ncell, l0, walls, rb;  // rb: residual buffer holding the current r
    int dw;                            // x lives as FP32 pairs (a.p32, a.q32): the Chebyshev path
    long long off, ntot;
    double c0, cx, cy, inv;
    float c0f, cxf, cyf, betaf, alphaf, pc0f, pcxf, pcyf, scf;
    DW C0, CX, CY;
};

// M v for the four cells of a quad: centre quad v, north and south quads, west and east
// scalars (images already applied).
__device__ __forceinline__ float4 precond4(const ChunkC& q, float4 c, float4 n, float4 s, float w, float e) {
    float4 z;
    z.x = fmaf(q.pc0f, c.x, fmaf(q.pcxf, w + c.y, q.pcyf * (n.x + s.x)));
    z.y = fmaf(q.pc0f, c.y, fmaf(q.pcxf, c.x + c.z, q.pcyf * (n.y + s.y)));
    z.z = fmaf(q.pc0f, c.z, fmaf(q.pcxf, c.y + c.w, q.pcyf * (n.z + s.z)));
    z.w = fmaf(q.pc0f, c.w, fmaf(q.pcxf, c.z + e, q.pcyf * (n.w + s.w)));
    return z;
}

// West / east neighbours of a quad at a conducting wall (images: Bx odd and zero on the
// wall node x = nx, By and Bz even), the same rule for every stencil on the B lattices.
__device__ __forceinline__ void wall_images(const ChunkC& q, int i, int c, float4 v, float& w, float& e) {
    if (!q.walls) return;
    if (i == 0) w = c == 0 ? -v.y : v.x;
    if (i + 4 == q.nx) e = c == 0 ? 0.f : v.w;
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void ld4d(const double* p, double v[4]) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
__device__ __forceinline__ void st4d(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// One phase on the cells of a chunk this thread owns: quads of 4 cells along x (cells
// 4 (q0 + qq 256 + tid) .. + 3 of the simulation), read and written as float4 / double2
// vectors; the west and east neighbours of a quad are two scalar loads. nx is a
// multiple of 4, so a quad never crosses a row. FULL: the chunk has all its cells, so
// there is no bounds test. acc1, acc2: FP32 partial sums of the phase (r.r and r.z for
// kBegin and kUpdate, p.q for kDirection); accd: the FP64 residual's r.r.
template <int PH, bool FULL>
__device__ __forceinline__ void chunk_cells(const CoopArgs& a, const ChunkC& q, float& acc1, float& acc2,
                                            double& accd) {
    const long long ntot = q.ntot;
#pragma unroll
    for (int qq = 0; qq < kPerThread / 4; qq++) {
        const int l = q.l0 + 4 * (qq * kCoopThreads + (int)threadIdx.x);
        if (!FULL && l >= q.ncell) continue;
        const int j = l / q.nx, i = l - j * q.nx;
        const long long row = q.off + (long long)j * q.nx;
        const long long k = row + i;
        const long long kwv = row + (i == 0 ? q.nx - 1 : i - 1);
        const long long kev = row + (i + 4 == q.nx ? 0 : i + 4);
        const long long kn = q.off + (long long)(j + 1 == q.ny ? 0 : j + 1) * q.nx + i;
        const long long ks = q.off + (long long)(j == 0 ? q.ny - 1 : j - 1) * q.nx + i;
        if constexpr (PH == kBegin) {
            // the FP64 residual's FP32 copy (buffer 0, written with it) times the scale, a
            // power of two (so this equals rounding r * scale), into buffer 1; e = 0;
            // z = M r from the neighbours' copies, scaled alike
            const float sc = q.scf;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float* R = a.r32[0] + c * ntot;
                const auto sc4 = [sc](float4 v) { return make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc); };
                const float4 fc = sc4(ld4(R + k)), fn = sc4(ld4(R + kn)), fs = sc4(ld4(R + ks));
                float fw = __ldcg(R + kwv) * sc, fe = __ldcg(R + kev) * sc;
                wall_images(q, i, c, fc, fw, fe);
                const float4 z = precond4(q, fc, fn, fs, fw, fe);
                st4(a.r32[1] + c * ntot + k, fc);
                st4(a.z32 + c * ntot + k, z);
                st4(a.e32 + c * ntot + k, make_float4(0.f, 0.f, 0.f, 0.f));
                acc1 = dot4(fc, fc, acc1);
                acc2 = dot4(fc, z, acc2);
            }
        } else if constexpr (PH == kDirection) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float* Z = a.z32 + c * ntot;
                const float4 zc = ld4(Z + k), zn = ld4(Z + kn), zs = ld4(Z + ks);
                float zw = __ldcg(Z + kwv), ze = __ldcg(Z + kev);
                wall_images(q, i, c, zc, zw, ze);
                const float4 po = ld4(a.p32 + c * ntot + k), qo = ld4(a.q32 + c * ntot + k);
                float4 Az;
                Az.x = q.c0f * zc.x - q.cxf * (zw + zc.y) - q.cyf * (zn.x + zs.x);
                Az.y = q.c0f * zc.y - q.cxf * (zc.x + zc.z) - q.cyf * (zn.y + zs.y);
                Az.z = q.c0f * zc.z - q.cxf * (zc.y + zc.w) - q.cyf * (zn.z + zs.z);
                Az.w = q.c0f * zc.w - q.cxf * (zc.z + ze) - q.cyf * (zn.w + zs.w);
                // beta = 0 on the first iteration: p and q of the last solve are not used
                const bool first = q.betaf == 0.f;
                const float b = q.betaf;
                const float4 pn = first ? zc
                                        : make_float4(fmaf(b, po.x, zc.x), fmaf(b, po.y, zc.y),
                                                      fmaf(b, po.z, zc.z), fmaf(b, po.w, zc.w));
                const float4 qn = first ? Az
                                        : make_float4(fmaf(b, qo.x, Az.x), fmaf(b, qo.y, Az.y),
                                                      fmaf(b, qo.z, Az.z), fmaf(b, qo.w, Az.w));
                st4(a.p32 + c * ntot + k, pn);
                st4(a.q32 + c * ntot + k, qn);
                acc1 = dot4(pn, qn, acc1);
            }
        } else if constexpr (PH == kUpdate) {
            const float al = q.alphaf;
            const float* Rc = a.r32[q.rb];
            float* Rn = a.r32[q.rb ^ 1];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const long long o = c * ntot;
                const float4 rc = ld4(Rc + o + k), rn = ld4(Rc + o + kn), rs = ld4(Rc + o + ks);
                const float4 qc = ld4(a.q32 + o + k), qn = ld4(a.q32 + o + kn), qs = ld4(a.q32 + o + ks);
                const float rw = __ldcg(Rc + o + kwv), re = __ldcg(Rc + o + kev);
                const float qw = __ldcg(a.q32 + o + kwv), qe = __ldcg(a.q32 + o + kev);
                const float4 pp = ld4(a.p32 + o + k), e = ld4(a.e32 + o + k);
                const auto upd = [al](float4 r, float4 v) {
                    return make_float4(fmaf(-al, v.x, r.x), fmaf(-al, v.y, r.y), fmaf(-al, v.z, r.z),
                                       fmaf(-al, v.w, r.w));
                };
                const float4 wc = upd(rc, qc), wn = upd(rn, qn), ws = upd(rs, qs);
                float ww = fmaf(-al, qw, rw), we = fmaf(-al, qe, re);
                wall_images(q, i, c, wc, ww, we);
                const float4 z = precond4(q, wc, wn, ws, ww, we);
                st4(Rn + o + k, wc);
                st4(a.z32 + o + k, z);
                st4(a.e32 + o + k, make_float4(fmaf(al, pp.x, e.x), fmaf(al, pp.y, e.y), fmaf(al, pp.z, e.z),
                                               fmaf(al, pp.w, e.w)));
                acc1 = dot4(wc, wc, acc1);
                acc2 = dot4(wc, z, acc2);
            }
        } else if constexpr (PH == kX) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const long long o = c * ntot + k;
                double xv[4];
                ld4d(a.x + o, xv);
                const float4 e = ld4(a.e32 + o);
                xv[0] += (double)e.x * q.inv;
                xv[1] += (double)e.y * q.inv;
                xv[2] += (double)e.z * q.inv;
                xv[3] += (double)e.w * q.inv;
                st4d(a.x + o, xv);
            }
        } else if constexpr (PH == kJoin) {  // x = h + l (FP64), the solve's result
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const long long o = c * ntot + k;
                const float4 h = ld4(a.p32 + o), lo = ld4(a.q32 + o);
                const double xv[4] = {dw_join({h.x, lo.x}), dw_join({h.y, lo.y}), dw_join({h.z, lo.z}),
                                      dw_join({h.w, lo.w})};
                st4d(a.x + o, xv);
            }
        } else if constexpr (PH == kResidualDW) {  // on the pairs: r = b - A x, its FP32 copy, (r, r)
            const DW C0 = q.C0, CX = q.CX, CY = q.CY;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float* XH = a.p32 + c * ntot;
                const float* XL = a.q32 + c * ntot;
                const float4 hc = ld4(XH + k), lc = ld4(XL + k), hn = ld4(XH + kn), ln = ld4(XL + kn);
                const float4 hs = ld4(XH + ks), ls = ld4(XL + ks);
                DW xw{__ldcg(XH + kwv), __ldcg(XL + kwv)}, xe{__ldcg(XH + kev), __ldcg(XL + kev)};
                double bv[4];
                ld4d(a.b + c * ntot + k, bv);
                const DW xc[4] = {{hc.x, lc.x}, {hc.y, lc.y}, {hc.z, lc.z}, {hc.w, lc.w}};
                const DW xn[4] = {{hn.x, ln.x}, {hn.y, ln.y}, {hn.z, ln.z}, {hn.w, ln.w}};
                const DW xs[4] = {{hs.x, ls.x}, {hs.y, ls.y}, {hs.z, ls.z}, {hs.w, ls.w}};
                if (q.walls) {
                    if (i == 0) xw = c == 0 ? dw_neg(xc[1]) : xc[0];
                    if (i + 4 == q.nx) xe = c == 0 ? DW{0.f, 0.f} : xc[3];
                }
                float rf[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const DW w = u == 0 ? xw : xc[u - 1];
                    const DW e = u == 3 ? xe : xc[u + 1];
                    const DW off = dw_add(dw_mul(CX, dw_add(w, e)), dw_mul(CY, dw_add(xn[u], xs[u])));
                    const DW Ax = dw_add(dw_mul(C0, xc[u]), dw_neg(off));
                    const DW r = dw_add(dw_from(bv[u]), dw_neg(Ax));
                    rf[u] = r.h;
                    acc1 = fmaf(r.h, r.h, acc1);
                }
                st4(a.r32[0] + c * ntot + k, make_float4(rf[0], rf[1], rf[2], rf[3]));
            }
        } else {  // kResidual: r = b - A x in FP64
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const double* X = a.x + c * ntot;
                double xc[4], xn[4], xs[4], bv[4], rv[4];
                ld4d(X + k, xc);
                ld4d(X + kn, xn);
                ld4d(X + ks, xs);
                ld4d(a.b + c * ntot + k, bv);
                double xw = __ldcg(X + kwv), xe = __ldcg(X + kev);
                if (q.walls) {
                    if (i == 0) xw = c == 0 ? -xc[1] : xc[0];
                    if (i + 4 == q.nx) xe = c == 0 ? 0.0 : xc[3];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const double w = u == 0 ? xw : xc[u - 1];
                    const double e = u == 3 ? xe : xc[u + 1];
                    rv[u] = bv[u] - (q.c0 * xc[u] - q.cx * (w + e) - q.cy * (xn[u] + xs[u]));
                    accd += rv[u] * rv[u];
                }
                st4d(a.r + c * ntot + k, rv);
                // its FP32 copy for the next inner solve's first pass
                st4(a.r32[0] + c * ntot + k, make_float4((float)rv[0], (float)rv[1], (float)rv[2], (float)rv[3]));
            }
        }
    }
}

// The direction pass on a full chunk, component by component with the loads of both
// quads issued before any arithmetic: the stores of one component cannot be proved
// apart from the loads of the next, so a quad-by-quad order would serialise six L2
// round trips per phase.
constexpr int kQuads = kPerThread / 4;

__device__ __forceinline__ void direction_full(const CoopArgs& a, const ChunkC& q, float& acc1) {
    int k[kQuads], kn[kQuads], ks[kQuads], kw[kQuads], ke[kQuads], ii[kQuads];
#pragma unroll
    for (int qq = 0; qq < kQuads; qq++) {
        const int l = q.l0 + 4 * (qq * kCoopThreads + (int)threadIdx.x);
        const int j = l / q.nx, i = l - j * q.nx;
        const int row = j * q.nx;  // cell offsets within the simulation
        ii[qq] = i;
        k[qq] = row + i;
        kw[qq] = row + (i == 0 ? q.nx - 1 : i - 1);
        ke[qq] = row + (i + 4 == q.nx ? 0 : i + 4);
        kn[qq] = (j + 1 == q.ny ? 0 : j + 1) * q.nx + i;
        ks[qq] = (j == 0 ? q.ny - 1 : j - 1) * q.nx + i;
    }
    const bool first = q.betaf == 0.f;  // beta = 0: p and q of the last solve are not used
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float* Z = a.z32 + c * q.ntot + q.off;
        float* Pp = a.p32 + c * q.ntot + q.off;
        float* Qp = a.q32 + c * q.ntot + q.off;
        float4 zc[kQuads], zn[kQuads], zs[kQuads], po[kQuads], qo[kQuads];
        float zw[kQuads], ze[kQuads];
#pragma unroll
        for (int qq = 0; qq < kQuads; qq++) {
            zc[qq] = ld4(Z + k[qq]);
            zn[qq] = ld4(Z + kn[qq]);
            zs[qq] = ld4(Z + ks[qq]);
            zw[qq] = __ldcg(Z + kw[qq]);
            ze[qq] = __ldcg(Z + ke[qq]);
            po[qq] = ld4(Pp + k[qq]);
            qo[qq] = ld4(Qp + k[qq]);
        }
#pragma unroll
        for (int qq = 0; qq < kQuads; qq++) {
            wall_images(q, ii[qq], c, zc[qq], zw[qq], ze[qq]);
            const float4 r0 = zc[qq], r1 = zn[qq], r2 = zs[qq];
            float4 Az;
            Az.x = q.c0f * r0.x - q.cxf * (zw[qq] + r0.y) - q.cyf * (r1.x + r2.x);
            Az.y = q.c0f * r0.y - q.cxf * (r0.x + r0.z) - q.cyf * (r1.y + r2.y);
            Az.z = q.c0f * r0.z - q.cxf * (r0.y + r0.w) - q.cyf * (r1.z + r2.z);
            Az.w = q.c0f * r0.w - q.cxf * (r0.z + ze[qq]) - q.cyf * (r1.w + r2.w);
            const float b = q.betaf;
            const float4 pn = first ? r0
                                    : make_float4(fmaf(b, po[qq].x, r0.x), fmaf(b, po[qq].y, r0.y),
                                                  fmaf(b, po[qq].z, r0.z), fmaf(b, po[qq].w, r0.w));
            const float4 qn = first ? Az
                                    : make_float4(fmaf(b, qo[qq].x, Az.x), fmaf(b, qo[qq].y, Az.y),
                                                  fmaf(b, qo[qq].z, Az.z), fmaf(b, qo[qq].w, Az.w));
            st4(Pp + k[qq], pn);
            st4(Qp + k[qq], qn);
            acc1 = dot4(pn, qn, acc1);
        }
    }
}

// The pair residual on a full chunk, component by component with the loads of both
// quads issued before any arithmetic (as direction_full, for the same reason).
__device__ __forceinline__ void residual_dw_full(const CoopArgs& a, const ChunkC& q, float& acc1) {
    int k[kQuads], kn[kQuads], ks[kQuads], kw[kQuads], ke[kQuads], ii[kQuads];
#pragma unroll
    for (int qq = 0; qq < kQuads; qq++) {
        const int l = q.l0 + 4 * (qq * kCoopThreads + (int)threadIdx.x);
        const int j = l / q.nx, i = l - j * q.nx;
        const int row = j * q.nx;
        ii[qq] = i;
        k[qq] = row + i;
        kw[qq] = row + (i == 0 ? q.nx - 1 : i - 1);
        ke[qq] = row + (i + 4 == q.nx ? 0 : i + 4);
        kn[qq] = (j + 1 == q.ny ? 0 : j + 1) * q.nx + i;
        ks[qq] = (j == 0 ? q.ny - 1 : j - 1) * q.nx + i;
    }
    const DW C0 = q.C0, CX = q.CX, CY = q.CY;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const long long o = c * q.ntot + q.off;
        const float* XH = a.p32 + o;
        const float* XL = a.q32 + o;
        float4 hc[kQuads], lc[kQuads], hn[kQuads], ln[kQuads], hs[kQuads], ls[kQuads];
        float hw[kQuads], lw[kQuads], he[kQuads], le[kQuads];
        double bv[kQuads][4];
#pragma unroll
        for (int qq = 0; qq < kQuads; qq++) {
            hc[qq] = ld4(XH + k[qq]);
            lc[qq] = ld4(XL + k[qq]);
            hn[qq] = ld4(XH + kn[qq]);
            ln[qq] = ld4(XL + kn[qq]);
            hs[qq] = ld4(XH + ks[qq]);
            ls[qq] = ld4(XL + ks[qq]);
            hw[qq] = __ldcg(XH + kw[qq]);
            lw[qq] = __ldcg(XL + kw[qq]);
            he[qq] = __ldcg(XH + ke[qq]);
            le[qq] = __ldcg(XL + ke[qq]);
            ld4d(a.b + o + k[qq], bv[qq]);
        }
#pragma unroll
        for (int qq = 0; qq < kQuads; qq++) {
            const DW xc[4] = {{hc[qq].x, lc[qq].x}, {hc[qq].y, lc[qq].y}, {hc[qq].z, lc[qq].z}, {hc[qq].w, lc[qq].w}};
            const DW xn[4] = {{hn[qq].x, ln[qq].x}, {hn[qq].y, ln[qq].y}, {hn[qq].z, ln[qq].z}, {hn[qq].w, ln[qq].w}};
            const DW xs[4] = {{hs[qq].x, ls[qq].x}, {hs[qq].y, ls[qq].y}, {hs[qq].z, ls[qq].z}, {hs[qq].w, ls[qq].w}};
            DW xw{hw[qq], lw[qq]}, xe{he[qq], le[qq]};
            if (q.walls) {
                if (ii[qq] == 0) xw = c == 0 ? dw_neg(xc[1]) : xc[0];
                if (ii[qq] + 4 == q.nx) xe = c == 0 ? DW{0.f, 0.f} : xc[3];
            }
            float rf[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const DW w = u == 0 ? xw : xc[u - 1];
                const DW e = u == 3 ? xe : xc[u + 1];
                const DW off = dw_add(dw_mul(CX, dw_add(w, e)), dw_mul(CY, dw_add(xn[u], xs[u])));
                const DW Ax = dw_add(dw_mul(C0, xc[u]), dw_neg(off));
                const DW r = dw_add(dw_from(bv[qq][u]), dw_neg(Ax));
                rf[u] = r.h;
                acc1 = fmaf(r.h, r.h, acc1);
            }
            st4(a.r32[0] + o + k[qq], make_float4(rf[0], rf[1], rf[2], rf[3]));
        }
    }
}

template <int PH>
__device__ __forceinline__ void chunk_phase(const CoopArgs& a, const ChunkC& q, float& acc1, float& acc2,
                                            double& accd) {
    const bool full = q.l0 + kChunkCells <= q.ncell;
    if constexpr (PH == kDirection) {
        if (full) return direction_full(a, q, acc1);
    }
    if constexpr (PH == kResidualDW) {
        if (full) return residual_dw_full(a, q, acc1);
    }
    if (full) chunk_cells<PH, true>(a, q, acc1, acc2, accd);
    else chunk_cells<PH, false>(a, q, acc1, acc2, accd);
}

// The Chebyshev inner solve of A e = r sc (r = the FP32 copy of the residual, sc its
// power-of-two scale) on one component of one tile, then x += e / sc on the tile's
// interior. With theta_c = c0, delta = 2 (cx + cy), sigma = theta_c / delta (the
// three-term recurrence of the Chebyshev iteration, e.g. Saad, Iterative Methods for
// Sparse Linear Systems, Sec. 12.3):
//   e_1 = d_0 = t_0 / theta_c, rho_0 = 1 / sigma, t_0 = r sc;
//   k = 1 .. m-1:  t_k = r sc - A e_k, rho_k = 1 / (2 sigma - rho_{k-1}),
//                  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) t_k,  e_{k+1} = e_k + d_k.
// The window holds the tile and kChebHalo >= m - 1 cells around it (wrapped
// periodically; at a wall the columns beyond it are dead and the wall's images are
// applied exactly). Thread tid < 224 owns window column tid % 56 and the 22-row strip
// tid / 56: r sc, d and e of its cells stay in registers; e also goes to shared memory
// each step (two buffers, one barrier per step) for the neighbouring columns and the
// strips above and below. The ring of ghost cells around the window stays zero.

// 16-byte asynchronous global -> shared copies (cp.async, sm_80 and later): the tile's
// x is fetched while its Chebyshev steps run.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One step on a thread's strip: reads the old e of its neighbours from src, writes the
// new e to dst (distinct buffers).
// WALL: this column is a wall column (wl or wr set); the other columns take the form
// without the image selects.
template <bool WALL>
__device__ __forceinline__ void cheb_step(const float* __restrict__ src, float* __restrict__ dst, int base,
                                          float (&e)[kChebRows], float (&d)[kChebRows],
                                          const float (&rs)[kChebRows], float c0f, float cxf, float cyf,
                                          float ca, float cb, bool wl, bool wr, bool odd) {
    float up = src[base - kChebPitch];
    float wn = src[base - 1], en = src[base + 1];  // the next row's west and east neighbours
    const float last = src[base + kChebRows * kChebPitch];  // the row below the strip
#pragma unroll
    for (int k = 0; k < kChebRows; k++) {
        const int l = base + k * kChebPitch;
        const float ec = e[k];
        const float dn = k + 1 < kChebRows ? e[k + 1 < kChebRows ? k + 1 : k] : last;
        float wv = wn, ev = en;
        if (k + 1 < kChebRows) {  // loads one row ahead of the arithmetic
            wn = src[l + kChebPitch - 1];
            en = src[l + kChebPitch + 1];
        }
        if (WALL) {
            if (wl) wv = odd ? -ev : ec;  // conductor images: Bx odd and zero on the wall node
            if (wr) ev = odd ? 0.f : ec;  // x = nx, By and Bz even
        }
        const float Ae = fmaf(c0f, ec, -fmaf(cxf, wv + ev, cyf * (up + dn)));
        d[k] = fmaf(ca, d[k], cb * (rs[k] - Ae));
        up = ec;
        e[k] = ec + d[k];
        dst[l] = e[k];
    }
}

__device__ __forceinline__ void cheb_tile(const CoopArgs& a, const GState& s, int g, int t, int c, float* ew) {
    const GridDev* Gp = a.grids + g;
    const int nx = __ldg(&Gp->nx), ny = __ldg(&Gp->ny), walls = __ldg(&Gp->walls);
    const long long off = __ldg(&Gp->cell_off);
    const float c0f = s.c0f, cxf = s.cxf, cyf = s.cyf;
    const int2 t0 = __ldg(a.tile_xy + t);
    const int X0 = t0.x, Y0 = t0.y;
    const int X1 = min(X0 + kChebTileX, nx), Y1 = min(Y0 + kChebTileY, ny);
    const int m = s.m;
    const int tid = threadIdx.x;
    const bool act = tid < kChebW * kChebStrips;
    const int col = tid % kChebW, strip = tid / kChebW;
    const int r0 = strip * kChebRows;
    const int base = (r0 + 1) * kChebPitch + col + 1;
    const int gx = X0 - kChebHalo + col;                       // unwrapped column
    const bool live = act && (!walls || (gx >= 0 && gx < nx));  // dead: beyond a wall
    const bool wl = walls && gx == 0, wr = walls && gx == nx - 1;
    int gxw = gx;
    while (gxw < 0) gxw += nx;
    while (gxw >= nx) gxw -= nx;
    int gy = Y0 - kChebHalo + r0;  // first row of the strip, wrapped
    while (gy < 0) gy += ny;
    while (gy >= ny) gy -= ny;
    const float sc = s.scf;
    const float sig = s.sig, delta = c0f / sig, ith = 1.f / c0f;
    const float* Rg = a.r32[0] + c * a.ntot + off + gxw;
    float rs[kChebRows], d[kChebRows], e[kChebRows];
    float* ea = ew;
    float* eb = ew + kChebCells;
    // the interior's x, staged asynchronously during the steps: pairs (h rows, then l
    // rows) or, in the solve's first refinement, FP64 values; rows of kChebTileX, 16-byte
    // chunks (nx, the offsets and X0 are multiples of 4 cells, so chunks stay aligned)
    float* xst = ew + 2 * kChebCells;
    const int nrow = Y1 - Y0, ncol = X1 - X0;
    const long long ob = c * a.ntot + off + (long long)Y0 * nx + X0;
    if (s.dw) {
        for (int q = tid; q < 2 * kChebTileY * (kChebTileX / 4); q += kCoopThreads) {
            const int arr = q / (kChebTileY * (kChebTileX / 4)), rem = q - arr * (kChebTileY * (kChebTileX / 4));
            const int y = rem / (kChebTileX / 4), x4 = 4 * (rem - y * (kChebTileX / 4));
            if (y < nrow && x4 < ncol)
                cp_async16(xst + arr * kChebTileCells + y * kChebTileX + x4,
                           (arr ? a.q32 : a.p32) + ob + (long long)y * nx + x4);
        }
    } else {
        double* xd = reinterpret_cast<double*>(xst);
        for (int q = tid; q < kChebTileY * (kChebTileX / 2); q += kCoopThreads) {
            const int y = q / (kChebTileX / 2), x2 = 2 * (q - y * (kChebTileX / 2));
            if (y < nrow && x2 < ncol) cp_async16(xd + y * kChebTileX + x2, a.x + ob + (long long)y * nx + x2);
        }
    }
    cp_async_commit();
#pragma unroll
    for (int k = 0; k < kChebRows; k++) {
        rs[k] = live ? __ldcg(Rg + (long long)gy * nx) * sc : 0.f;
        d[k] = rs[k] * ith;
        e[k] = d[k];
        if (act) ea[base + k * kChebPitch] = e[k];
        if (++gy == ny) gy = 0;
    }
    __syncthreads();
    float rho = 1.f / sig;
    for (int it = 1; it < m; it++) {
        const float rn = 1.f / (2.f * sig - rho);
        const float ca = rn * rho, cb = 2.f * rn / delta;
        rho = rn;
        if (act) {
            if (wl || wr) cheb_step<true>(ea, eb, base, e, d, rs, c0f, cxf, cyf, ca, cb, wl, wr, c == 0);
            else cheb_step<false>(ea, eb, base, e, d, rs, c0f, cxf, cyf, ca, cb, false, false, false);
        }
        __syncthreads();
        float* tmp = ea;
        ea = eb;
        eb = tmp;
    }
    // interior: x += e / sc in FP32 pairs (1 / sc is a power of two, exact in FP32); the
    // first refinement of the solve takes x from its FP64 array. e is read back from the
    // window so that warp w updates rows w, w + 8, ... with one lane per column: whole
    // 128-byte rows per access, all eight loads of a lane in flight at once.
    cp_async_wait_all();
    __syncthreads();  // every thread's staged chunks visible
    {
        constexpr int kWarps = kCoopThreads / 32, kPer = kChebTileY / kWarps;
        const int lane = tid & 31, wp = tid >> 5;
        const int gxl = X0 + lane;
        if (gxl < X1) {
            const float invf = s.invf;
            const long long o0 = c * a.ntot + off + gxl;
            const bool pairs = s.dw != 0;
            DW v[kPer];
#pragma unroll
            for (int j = 0; j < kPer; j++) {
                const int yl = wp + kWarps * j, q = yl * kChebTileX + lane;
                v[j] = pairs ? DW{xst[q], xst[kChebTileCells + q]}
                             : dw_from(reinterpret_cast<const double*>(xst)[q]);
            }
#pragma unroll
            for (int j = 0; j < kPer; j++) {
                const int y = Y0 + wp + kWarps * j;
                if (y < Y1) {
                    const float ev = ea[(y - Y0 + kChebHalo + 1) * kChebPitch + lane + kChebHalo + 1];
                    const DW w = dw_add_f(v[j], __fmul_rn(ev, invf));
                    const long long o = o0 + (long long)y * nx;
                    a.p32[o] = w.h;
                    a.q32[o] = w.l;
                }
            }
        }
    }
    __syncthreads();  // the window is reused by the next item
}

// CG inner solve: 4 CTAs per SM (64 registers), 608 resident CTAs, so a 2048 x 512
// grid (512 chunks) gives every CTA at most one chunk per phase. With Chebyshev tiles
// (CHEB): 2 CTAs per SM, so that a thread holds its column strip in registers.
template <bool CHEB>
__global__ void __launch_bounds__(kCoopThreads, CHEB ? 2 : 4) k_mp_coop(const CoopArgs a) {
    __shared__ GState gs[kCoopMaxGrids];
    __shared__ double red[32];
    extern __shared__ __align__(16) double sp[];  // 2 x nchunks staged partial sums
    DevStatus* st = a.st;
    if (st->stop) return;  // the same for every CTA: stop changes only between launches
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned int nb = gridDim.x;
    const unsigned int lim = st->spin_limit ? st->spin_limit : (1u << 22);  // the same in every CTA
    for (int g = tid; g < a.ngrids; g += blockDim.x) {
        const CgState& c = a.cg[g];
        GState s{};
        s.rr = c.rr;
        s.bb = c.bb;
        s.rel = c.rel;
        s.active = c.active;
        s.iters = 0;
        s.outer = 0;
        s.rtol = a.grids[g].rtol;
        s.maxit = a.grids[g].maxit;
        const double c0 = a.grids[g].c0, dl = 2.0 * (a.grids[g].cx + a.grids[g].cy);
        const double sig = dl > 0.0 ? c0 / dl : 0.0;
        // Chebyshev when 13 steps reduce the error by kChebWorst at least (T_13(sigma) =
        // cosh(13 acosh sigma) >= 1 / kChebWorst) and the tiles cover the simulation
        s.cheb = CHEB && sig > 1.0 && kChebMaxIt * acosh(sig) >= acosh(1.0 / kChebWorst) && s.rtol >= kChebRtolMin;
        s.dw = 0;
        s.sig = (float)sig;
        s.m = 0;
        const GridDev& G = a.grids[g];
        s.c0f = (float)G.c0;
        s.cxf = (float)G.cx;
        s.cyf = (float)G.cy;
        s.pc0f = (float)G.pc0;
        s.pcxf = (float)G.pcx;
        s.pcyf = (float)G.pcy;
        s.C0 = dw_from(G.c0);
        s.CX = dw_from(G.cx);
        s.CY = dw_from(G.cy);
        gs[g] = s;
    }
    __syncthreads();
    // window of the Chebyshev tiles after the staged partial sums: two e buffers whose
    // ghost rings stay zero (the steps write window cells only)
    float* ew = reinterpret_cast<float*>(sp + 2 * a.nchunks);
    if constexpr (CHEB)
        for (int k = tid; k < 2 * kChebCells; k += blockDim.x) ew[k] = 0.f;
    int buf = 0;
    int rb = 0;  // residual buffer holding the current inner r (the same in every CTA)
    bool ok = true;
    const auto two = [](Phase ph) { return ph == kBegin || ph == kUpdate; };  // phases with two sums

    // Whether simulation state s takes part in phase ph (the inner CG phases only for
    // simulations without the Chebyshev solve).
    const auto takes = [](Phase ph, const GState& s) {
        if (ph == kDirection || ph == kUpdate) return s.active && s.in_active;
        if (ph == kBegin || ph == kX) return s.active && !s.cheb;
        if (ph == kJoin) return s.dw != 0;
        return s.active != 0;
    };
    // One pass over this CTA's chunks of the simulations taking part in `ph`, with
    // per-chunk partial sums into buffer `buf` where the phase reduces.
    auto pass = [&](Phase ph) {
        double* part = a.part + (size_t)buf * 2 * a.nchunks;
        for (int ch = blockIdx.x; ch < a.nchunks; ch += nb) {
            const int g = __ldg(a.chunk_grid + ch);
            const GState& s = gs[g];
            if (!takes(ph, s)) continue;  // uniform over the CTA
            // per-chunk constants in registers (FP64 -> FP32 conversions run on the slow
            // FP64 pipe: once per chunk, not per cell)
            const GridDev* Gp = a.grids + g;
            ChunkC q;
            q.nx = __ldg(&Gp->nx);
            q.ny = __ldg(&Gp->ny);
            q.ncell = __ldg(&Gp->ncell);
            q.walls = __ldg(&Gp->walls);
            q.off = __ldg(&Gp->cell_off);
            q.ntot = a.ntot;
            q.rb = rb;
            q.c0 = __ldg(&Gp->c0);
            q.cx = __ldg(&Gp->cx);
            q.cy = __ldg(&Gp->cy);
            q.c0f = s.c0f;
            q.cxf = s.cxf;
            q.cyf = s.cyf;
            q.pc0f = s.pc0f;
            q.pcxf = s.pcxf;
            q.pcyf = s.pcyf;
            q.C0 = s.C0;
            q.CX = s.CX;
            q.CY = s.CY;
            q.betaf = s.betaf;
            q.alphaf = s.alphaf;
            q.scf = s.scf;
            q.inv = s.inv;
            q.dw = s.dw;
            q.l0 = (ch - __ldg(&a.gchunk[g].x)) * kChunkCells;
            float acc1 = 0.f, acc2 = 0.f;
            double accd = 0.0;
            switch (ph) {
            case kBegin: chunk_phase<kBegin>(a, q, acc1, acc2, accd); break;
            case kDirection: chunk_phase<kDirection>(a, q, acc1, acc2, accd); break;
            case kUpdate: chunk_phase<kUpdate>(a, q, acc1, acc2, accd); break;
            case kX: chunk_phase<kX>(a, q, acc1, acc2, accd); break;
            case kJoin:
                if constexpr (CHEB) chunk_phase<kJoin>(a, q, acc1, acc2, accd);
                break;
            default:
                if constexpr (CHEB)
                    if (q.dw) {
                        chunk_phase<kResidualDW>(a, q, acc1, acc2, accd);
                        break;
                    }
                chunk_phase<kResidual>(a, q, acc1, acc2, accd);
                break;
            }
            if (ph != kX && ph != kJoin) {
                const double t1 = block_sum(ph == kResidual && !q.dw ? accd : (double)acc1, red);
                if (tid == 0) part[ch] = t1;
                __syncthreads();  // red is reused next
                if (two(ph)) {
                    const double t2 = block_sum((double)acc2, red);
                    if (tid == 0) part[a.nchunks + ch] = t2;
                    __syncthreads();
                }
            }
        }
    };
    // After a barrier: every CTA forms the sums of the phase for all simulations taking
    // part, then updates their scalars identically.
    auto reduce = [&](Phase ph) {
        const double* part = a.part + (size_t)buf * 2 * a.nchunks;
        stage_partials(part, two(ph) ? 2 * a.nchunks : a.nchunks, sp);
        for (int g = warp; g < a.ngrids; g += kCoopThreads / 32) {
            GState& s = gs[g];
            if (!takes(ph, s)) continue;
            const double t = chunk_sum(sp, a.gchunk[g]);
            const double t2 = two(ph) ? chunk_sum(sp + a.nchunks, a.gchunk[g]) : 0.0;
            if (lane != 0) continue;
            if (ph == kBegin) {
                s.rr_in0 = t;
                s.rr_in = t;
                s.rz = t2;
                s.beta = 0.0;
                s.betaf = 0.f;
                s.in_iters = 0;
                s.tol_in = fmax(2e-6, 0.5 * s.rtol * sqrt(s.bb / fmax(s.rr, 1e-300)));
                s.in_active = (t > 0.0 && t2 > 0.0) ? 1 : 0;
            } else if (ph == kDirection) {
                s.alpha = s.rz / t;
                s.alphaf = (float)s.alpha;
            } else if (ph == kUpdate) {
                s.beta = t2 / s.rz;
                s.betaf = (float)s.beta;
                s.rz = t2;
                s.rr_in = t;
                s.in_iters += 1;
                s.iters += 1;
                if (sqrt(t / s.rr_in0) <= s.tol_in || s.in_iters >= kInnerMax || s.iters >= s.maxit ||
                    !(t2 > 0.0))
                    s.in_active = 0;
            } else if (ph == kResidual) {
                s.rr = t;
                s.rel = sqrt(t / s.bb);
                s.outer += 1;
                if (s.rel <= s.rtol) {
                    s.active = 0;
                } else if (s.iters >= s.maxit || s.outer >= s.maxit) {
                    s.active = 0;
                    if (blockIdx.x == 0) {
                        atomicAdd(&st->cg_noconv, 1u);
                        st->stop_next = 1u;
                    }
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    };
    auto any = [&](bool inner) {
        int n = 0;
        for (int g = 0; g < a.ngrids; g++) n += inner ? (gs[g].active && gs[g].in_active) : gs[g].active;
        return n > 0;
    };
    auto any_mode = [&](int cheb) {
        int n = 0;
        for (int g = 0; g < a.ngrids; g++) n += gs[g].active && gs[g].cheb == cheb;
        return n > 0;
    };

    while (ok && any(false)) {
        for (int g = tid; g < a.ngrids; g += blockDim.x)
            if (gs[g].active) {
                GState& s = gs[g];
                // r32 of about unit RMS: the power of two in [s/2, s), s = sqrt(3 ncell / (r, r))
                int ex;
                frexp(sqrt(3.0 * a.grids[g].ncell / s.rr), &ex);
                s.scale = ldexp(1.0, ex - 1);
                s.inv = ldexp(1.0, 1 - ex);
                s.scf = (float)s.scale;
                s.invf = (float)s.inv;
                s.in_active = 0;
                if (s.cheb) {
                    // the reduction this refinement needs (the CG's inner tolerance), in
                    // Chebyshev steps: 1 / T_m(sigma) <= tgt
                    const double tgt = fmax(kChebFloor, 0.5 * s.rtol * sqrt(s.bb / fmax(s.rr, 1e-300)));
                    const int m = (int)ceil(acosh(1.0 / tgt) / acosh((double)s.sig));
                    s.m = max(1, min(kChebMaxIt, m));
                }
            }
        __syncthreads();
        if (CHEB && any_mode(1)) {
            const int nitems = 3 * a.ntiles;
            for (int it = blockIdx.x; it < nitems; it += nb) {
                const int t = it / 3, c = it - 3 * (it / 3);
                const int g = __ldg(a.tile_grid + t);
                if (!(gs[g].active && gs[g].cheb)) continue;  // uniform over the CTA
                if constexpr (CHEB) cheb_tile(a, gs[g], g, t, c, ew);
            }
            for (int g = tid; g < a.ngrids; g += blockDim.x)
                if (gs[g].active && gs[g].cheb) {
                    gs[g].iters += gs[g].m;
                    gs[g].dw = 1;  // the tiles wrote x as pairs
                }
            if (blockIdx.x == 0 && tid == 0) {
                int mx = 0;
                for (int g = 0; g < a.ngrids; g++)
                    if (gs[g].active && gs[g].cheb) mx = max(mx, gs[g].m);
                st->loop_iters[0] += (unsigned long long)mx;
            }
            __syncthreads();
        }
        if (!any_mode(0)) {
            ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
            if (!ok) break;
            pass(kResidual);
            ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
            if (!ok) break;
            reduce(kResidual);
            if (blockIdx.x == 0 && tid == 0) st->loop_iters[1] += 1ull;
            continue;
        }
        pass(kBegin);
        rb = 1;  // the first pass wrote the scaled residual into buffer 1
        ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
        if (!ok) break;
        reduce(kBegin);
        while (any(true)) {
            pass(kDirection);
            ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
            if (!ok) break;
            reduce(kDirection);
            pass(kUpdate);
            rb ^= 1;  // the update pass wrote r' into the other buffer
            ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
            if (!ok) break;
            reduce(kUpdate);
            if (blockIdx.x == 0 && tid == 0) st->loop_iters[0] += 1ull;
        }
        if (!ok) break;
        pass(kX);
        ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
        if (!ok) break;
        pass(kResidual);
        ok = grid_barrier(a.bar, nb, &st->sync_timeout, lim);
        if (!ok) break;
        reduce(kResidual);
        if (blockIdx.x == 0 && tid == 0) st->loop_iters[1] += 1ull;
    }
    if (!ok) {
        if (tid == 0) st->stop_next = 1u;
        return;
    }
    if (CHEB) pass(kJoin);  // no barrier after: nothing in this launch reads x again
    if (blockIdx.x == 0) {
        for (int g = tid; g < a.ngrids; g += blockDim.x) {
            CgState& c = a.cg[g];
            const GState& s = gs[g];
            c.rr = s.rr;
            c.rel = s.rel;
            c.active = 0;
            c.iters = s.iters;
            c.outer = s.outer;
            c.total_outer += s.outer;
        }
    }
}

}  // namespace

size_t coop_smem(const CoopSolve& cs) {
    return 2 * (size_t)cs.nchunks * sizeof(double) +
           (cs.cheb ? (2 * (size_t)kChebCells + 2 * (size_t)kChebTileCells) * sizeof(float) : 0);
}

// Whether simulation g can take the Chebyshev inner solve (as the kernel decides).
bool cheb_ok(const GridDev& G) {
    const double dl = 2.0 * (G.cx + G.cy);
    const double sig = dl > 0.0 ? G.c0 / dl : 0.0;
    return sig > 1.0 && kChebMaxIt * std::acosh(sig) >= std::acosh(1.0 / kChebWorst);
}

int coop_create(CoopSolve* cs, const GridDev* hg, int ngrids, bool cg_inner, std::string& err) {
    coop_free(cs);
    if (ngrids > kCoopMaxGrids) return PIC_EINVAL;  // the caller keeps the WHILE-node solve
    for (int g = 0; g < ngrids; g++)
        if (hg[g].nx % 4) return PIC_EINVAL;  // quads of 4 cells along x
    std::vector<int2> gc(ngrids);
    std::vector<int> cg;
    std::vector<int> tg;
    std::vector<int2> txy;
    for (int g = 0; g < ngrids; g++) {
        const int n = (hg[g].ncell + kChunkCells - 1) / kChunkCells;
        gc[g] = make_int2((int)cg.size(), n);
        cg.insert(cg.end(), n, g);
        for (int y = 0; y < hg[g].ny; y += kChebTileY)
            for (int x = 0; x < hg[g].nx; x += kChebTileX) {
                tg.push_back(g);
                txy.push_back(make_int2(x, y));
            }
    }
    int dev = 0, nsm = 0, occ = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if ((int)cg.size() > kCoopMaxChunks) return PIC_EINVAL;
    cs->nchunks = (int)cg.size();
    cs->cg_inner = cg_inner ? 1 : 0;
    cs->cheb = 0;
    for (int g = 0; g < ngrids && !cg_inner; g++) cs->cheb |= cheb_ok(hg[g]) ? 1 : 0;
    const size_t smem = coop_smem(*cs);
    const auto kern = cs->cheb ? k_mp_coop<true> : k_mp_coop<false>;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCoopThreads, smem);
    if (e == cudaSuccess && (!coop || occ < 1)) {
        *cs = CoopSolve{};
        return PIC_EINVAL;
    }
    if (e == cudaSuccess) e = cudaMalloc(&cs->gchunk, ngrids * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&cs->chunk_grid, cg.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&cs->tile_grid, tg.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&cs->tile_xy, txy.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&cs->part, 4 * cg.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&cs->bar, kBarWords * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpy(cs->gchunk, gc.data(), ngrids * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cs->chunk_grid, cg.data(), cg.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cs->tile_grid, tg.data(), tg.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(cs->tile_xy, txy.data(), txy.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(cs->bar, 0, kBarWords * sizeof(unsigned int));
    if (e != cudaSuccess) {
        err = std::string("cooperative solve set-up failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        coop_free(cs);
        return PIC_ECUDA;
    }
    cs->ngrids = ngrids;
    cs->ntiles = (int)tg.size();
    // enough CTAs for the chunks (and the Chebyshev tiles' three components), no more
    // than are resident at once
    const int items = cs->cheb ? std::max(cs->nchunks, 3 * cs->ntiles) : cs->nchunks;
    cs->nblocks = std::max(1, std::min(items, occ * nsm));
    return PIC_OK;
}

void coop_free(CoopSolve* cs) {
    void* ps[] = {cs->gchunk, cs->chunk_grid, cs->tile_grid, cs->tile_xy, cs->part, cs->bar};
    for (void* p : ps)
        if (p) cudaFree(p);
    *cs = CoopSolve{};
}

cudaError_t launch_mp_coop(const CoopSolve& cs, const FieldArgs& f, cudaStream_t s) {
    CoopArgs a{};
    a.grids = f.grids;
    a.ngrids = f.ngrids;
    a.gchunk = cs.gchunk;
    a.chunk_grid = cs.chunk_grid;
    a.nchunks = cs.nchunks;
    a.tile_grid = cs.tile_grid;
    a.tile_xy = cs.tile_xy;
    a.ntiles = cs.ntiles;
    a.ntot = f.ntot;
    a.b = f.b;
    a.x = f.x;
    a.r = f.r;
    a.r32[0] = f.r32;
    a.r32[1] = f.r32b;
    a.z32 = f.z32;
    a.p32 = f.p32;
    a.q32 = f.q32;
    a.e32 = f.e32;
    a.part = cs.part;
    a.bar = cs.bar;
    a.cg = f.cg;
    a.st = f.st;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)cs.nblocks);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = coop_smem(cs);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // barrier counters from zero on every launch (a launch that gave up on a barrier
    // leaves arrivals behind)
    cudaError_t e = cudaMemsetAsync(cs.bar, 0, kBarWords * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    return cs.cheb ? cudaLaunchKernelEx(&cfg, k_mp_coop<true>, a) : cudaLaunchKernelEx(&cfg, k_mp_coop<false>, a);
}

}  // namespace pic
