// fields.cu -- the implicit field solve of the particle cycle, FP64 throughout:
//   right-hand side of Eq. (7), PCG iterations on [1 - (theta c dt)^2 Lap] dB = b, and
//   the E, B update from Eqs. (5)-(6).
//
// One thread per cell handles the three components of every vector. Reductions use
// per-block partials and a "last block finishes" step per simulation (fixed summation
// order, so results do not depend on block scheduling); the last simulation to finish
// sets the WHILE condition of the captured PCG loop, so the loop runs exactly as many
// iterations as the slowest simulation needs, with no host round trip.
//
// Staggering (Sec. 2, Fig. 1; index k = j*nx + i): Ez at (i,j); Ex, By at (i+1/2,j);
// Ey, Bx at (i,j+1/2); Bz at (i+1/2,j+1/2). J shares the E lattices.
#include "dword.cuh"
#include "engine.h"

namespace pic {

namespace {

struct Cell {
    int g, i, j;
    long long k;   // global cell index (cell_off + j*nx + i)
    long long ke, kw, kn, ks;  // neighbours (i+1), (i-1), (j+1), (j-1), wrapped
    bool ew, ww;   // with walls: the east / west neighbour lies beyond a wall
    bool valid;
};

// Cell l (0 <= l < ncell) of simulation g.
__device__ __forceinline__ Cell cell_at(const GridDev& G, int g, int l) {
    Cell c;
    c.g = g;
    c.valid = true;
    c.j = l / G.nx;
    c.i = l - c.j * G.nx;
    const long long row = G.cell_off + (long long)c.j * G.nx;
    c.k = row + c.i;
    c.ke = row + (c.i + 1 == G.nx ? 0 : c.i + 1);
    c.kw = row + (c.i == 0 ? G.nx - 1 : c.i - 1);
    const int jn = c.j + 1 == G.ny ? 0 : c.j + 1;
    const int js = c.j == 0 ? G.ny - 1 : c.j - 1;
    c.kn = G.cell_off + (long long)jn * G.nx + c.i;
    c.ks = G.cell_off + (long long)js * G.nx + c.i;
    c.ew = G.walls && c.i + 1 == G.nx;
    c.ww = G.walls && c.i == 0;
    return c;
}

// x-neighbours with conducting walls (images of a perfect conductor): a quantity on an
// integer-x lattice (Ey, Ez, Bx, and the currents Jy, Jz as the field solve sees them) is
// odd under reflection at a wall and vanishes on the wall nodes; one on a half-integer
// lattice (Ex, By, Bz, Jx) is even. Without walls these are the periodic neighbours.
template <typename T>
__device__ __forceinline__ T east_odd(const T* V, const Cell& c) { return c.ew ? T(0) : V[c.ke]; }
template <typename T>
__device__ __forceinline__ T west_odd(const T* V, const Cell& c) { return c.ww ? -V[c.k + 1] : V[c.kw]; }
template <typename T>
__device__ __forceinline__ T east_even(const T* V, const Cell& c) { return c.ew ? V[c.k] : V[c.ke]; }
template <typename T>
__device__ __forceinline__ T west_even(const T* V, const Cell& c) { return c.ww ? V[c.k] : V[c.kw]; }
// Sum of the two x-neighbours of component a of a B-lattice vector (a = 0: Bx, odd).
template <typename T>
__device__ __forceinline__ T nbx(const T* V, const Cell& c, int a) {
    return a == 0 ? east_odd(V, c) + west_odd(V, c) : east_even(V, c) + west_even(V, c);
}

// Grid-stride loop over the cells of simulation g. A simulation gets a bounded number
// of blocks (a few per SM), so the per-simulation completion counter of the reductions
// sees few same-address atomics per kernel.
#define FOR_CELLS(G, g, c)                                                                  \
    for (int l_ = (blockIdx.x - (G).blk_first) * blockDim.x + threadIdx.x; l_ < (G).ncell;  \
         l_ += (G).nblk * blockDim.x)                                                       \
        if (const Cell c = cell_at((G), (g), l_); true)

// Current value at k: FP64 as is; the MIXED32 current is 64-bit fixed point.
template <typename T>
__device__ __forceinline__ double ld(const T* p, long long k, double jinv) {
    if constexpr (sizeof(T) == 8 && T(1) / T(2) == T(0)) return (double)p[k] * jinv;
    else return (double)p[k];
}

// Difference p[k1] - p[k2] of the current, times s: fixed-point values are subtracted
// exactly as integers and converted once (int64 -> FP64 conversions and FP64 products
// are slow on this part), with the fixed-point unit folded into s by the caller.
template <typename T>
__device__ __forceinline__ double dld(const T* p, long long k1, long long k2, double s) {
    if constexpr (sizeof(T) == 8 && T(1) / T(2) == T(0)) return (double)(p[k1] - p[k2]) * s;
    else return (p[k1] - p[k2]) * s;
}

// Sum `nv` values per thread over the block, store them as this block's partials, and
// return true in every thread of the block that completes its simulation last. The
// finishing block then holds the simulation-wide sums in `tot`.
template <int NV>
__device__ bool reduce_and_finish(const GridDev& G, int g, double v[NV], double* part,
                                  int nblk_total, unsigned int* done, double tot[NV]) {
    __shared__ double scratch[32];
    __shared__ bool last;
#pragma unroll
    for (int a = 0; a < NV; a++) {
        const double s = block_sum(v[a], scratch);
        if (threadIdx.x == 0) part[a * nblk_total + blockIdx.x] = s;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&done[g], 1u);
        last = (t == (unsigned)G.nblk - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int a = 0; a < NV; a++) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < G.nblk; b += blockDim.x)
            acc += __ldcg(&part[a * nblk_total + G.blk_first + b]);
        tot[a] = block_sum(acc, scratch);
    }
    if (threadIdx.x == 0) done[g] = 0u;
    return true;
}

// Called by the finishing block of each simulation after it updated cg[g]: the last
// simulation to finish counts the simulations still iterating (the outer PCG, or the
// inner FP32 loop when INNER) and sets the loop's WHILE condition.
template <bool INNER = false>
__device__ void finish_all_grids(int ngrids, int n_participating, CgState* cg, DevStatus* st,
                                 cudaGraphConditionalHandle cond, int use_cond, int count_slot = -1) {
    if (threadIdx.x != 0) return;
    __threadfence();
    const unsigned t = atomicAdd(&st->grids_done, 1u);
    if (t != (unsigned)n_participating - 1u) return;
    __threadfence();
    unsigned n = 0;
    for (int g = 0; g < ngrids; g++)
        n += (unsigned)(INNER ? __ldcg(&cg[g].in_active) : __ldcg(&cg[g].active));
    if (INNER) st->n_in_active = n;
    else st->n_active = n;
    if (count_slot >= 0) st->loop_iters[count_slot] += 1ull;  // loop iterations the handle ran
    st->grids_done = 0u;
    if (use_cond) cudaGraphSetConditional(cond, n > 0u ? 1u : 0u);
}

// ---- Eq. (7) right-hand side --------------------------------------------------------
// b = theta (c dt)^2 (Lap B^n + (4 pi / c) curl J^{n+1/2}) - c dt curl E^n  (c = 1)
// Initial residual r = b - A x0 (x0 = previous dB with warm start, else 0), p = r.
template <typename JT>
__global__ void __launch_bounds__(kFieldThreads)
k_rhs(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
      int nblk_total, long long ntot, const double* __restrict__ F, const JT* __restrict__ J,
      double* __restrict__ x, double* __restrict__ r, CgState* cg, double* part,
      unsigned int* done, DevStatus* st, cudaGraphConditionalHandle cond, int use_cond,
      double* __restrict__ bout, float* __restrict__ r32) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // b.b, r.r, |E|^2, |B|^2
    // Constants folded so that each term is one multiply-add on this part's slow FP64 pipe:
    //   b = ax (nbx(B) - 2 B) + ay (B_n + B_s - 2 B) + kj (curl J) - dt (curl E)
    // with ax = theta dt^2 / dx^2, ay = theta dt^2 / dy^2 (the Laplacian's differences are
    // formed first, so a uniform field gives exactly zero), and the current's differences
    // (exact integer differences of the fixed-point words) scaled by kj = 4 pi theta dt^2
    // times the fixed-point unit over dx or dy.
    const double th_dt2 = G.theta * G.dt * G.dt;
    const double ax = th_dt2 * G.idx * G.idx, ay = th_dt2 * G.idy * G.idy;
    // (the fixed-point unit jinv is 1 for an FP64 current)
    const double ji = (sizeof(JT) == 8 && JT(1) / JT(2) == JT(0)) ? G.jinv : 1.0;
    const double kjx = 4.0 * kPi * th_dt2 * ji * G.idx, kjy = 4.0 * kPi * th_dt2 * ji * G.idy;
    const double dtx = G.dt * G.idx, dty = G.dt * G.idy;
    if (!st->stop) FOR_CELLS(G, g, c) {
        const double* Ex = F;
        const double* Ey = F + ntot;
        const double* Ez = F + 2 * ntot;
        const JT* Jx = J;
        const JT* Jy = J + ntot;
        const JT* Jz = J + 2 * ntot;
        // dt curl E and theta dt^2 4 pi curl J on the B lattices
        const double ez = Ez[c.k];
        const double eEx = dty * (Ez[c.kn] - ez);
        const double eEy = -dtx * (east_odd(Ez, c) - ez);
        const double eEz = fma(dtx, east_odd(Ey, c) - Ey[c.k], -dty * (Ex[c.kn] - Ex[c.k]));
        double jJx, jJy, jJz;
        if (!G.walls) {
            jJx = dld(Jz, c.kn, c.k, kjy);
            jJy = -dld(Jz, c.ke, c.k, kjx);
            jJz = dld(Jy, c.ke, c.k, kjx) - dld(Jx, c.kn, c.k, kjy);
        } else {
            // the conductor carries the current of its wall nodes: Jy = Jz = 0 there
            const bool w0 = c.i == 0;
            const double jzc = w0 ? 0.0 : ld(Jz, c.k, 1.0), jzn = w0 ? 0.0 : ld(Jz, c.kn, 1.0);
            const double jze = c.ew ? 0.0 : ld(Jz, c.ke, 1.0);
            const double jyc = w0 ? 0.0 : ld(Jy, c.k, 1.0), jye = c.ew ? 0.0 : ld(Jy, c.ke, 1.0);
            jJx = (jzn - jzc) * kjy;
            jJy = -(jze - jzc) * kjx;
            jJz = (jye - jyc) * kjx - (ld(Jx, c.kn, 1.0) - ld(Jx, c.k, 1.0)) * kjy;
        }
        const double eE[3] = {eEx, eEy, eEz};
        const double jJ[3] = {jJx, jJy, jJz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double* B = F + (3 + a) * ntot;
            const double bc = B[c.k];
            const double b2 = bc + bc;
            const double b = fma(ax, nbx(B, c, a) - b2, fma(ay, (B[c.kn] + B[c.ks]) - b2, jJ[a] - eE[a]));
            double res = b;
            const long long o = a * ntot;
            if (G.warm == 1) {  // previous step's dB as the initial guess
                const double* X = x + o;
                const double Ax = G.c0 * X[c.k] - G.cx * nbx(X, c, a) - G.cy * (X[c.kn] + X[c.ks]);
                res = b - Ax;
                v[1] = fma(res, res, v[1]);
            }
            r[o + c.k] = res;
            if (r32) r32[o + c.k] = (float)res;  // FP32 copy for the cooperative solve
            if (bout) bout[o + c.k] = b;
            v[0] = fma(b, b, v[0]);
            v[3] = fma(bc, bc, v[3]);
        }
        v[2] = fma(Ex[c.k], Ex[c.k], fma(Ey[c.k], Ey[c.k], fma(ez, ez, v[2])));
    }
    double tot[4];
    if (!reduce_and_finish<4>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        const double e = G.dx * G.dy / (8.0 * kPi);
        s.ue = tot[2] * e;
        s.ub = tot[3] * e;
        s.bb = tot[0];
        s.rr = G.warm == 1 ? tot[1] : tot[0];  // r = b unless the previous dB is the guess
        s.beta = 0.0;
        s.iters = 0;
        s.outer = 0;
        s.rel = tot[0] > 0.0 ? sqrt(s.rr / tot[0]) : 0.0;
        s.active = (!st->stop && tot[0] > 0.0 && s.rel > G.rtol) ? 1 : 0;
    }
    finish_all_grids(ngrids, ngrids, cg, st, cond, use_cond);
}

// ---- the same right-hand side for the MIXED32 solve, in FP32-pair arithmetic ---------
// Same formula, cells and outputs as k_rhs<long long>, but every sum and product runs on
// FP32 pairs (dword.cuh: 47 significant bits) instead of the FP64 pipe: the FP64 values
// read are split by bit manipulation, the current's exact integer differences are
// converted once each, and b and r are joined back to FP64 with one add. The sums of
// squares (||b||, ||r||, the energies U_E, U_B) are formed from the pairs' leading
// words in FP32 per thread and in FP64 over the block. Where the warm start is off it
// also zeroes x at its cells (it reads no x then), in place of a k_zero_x launch.
__device__ __forceinline__ DW dwp(const float (&v)[2]) { return {v[0], v[1]}; }
__device__ __forceinline__ DW dw_i64(long long d) { return dw_from_i64(d); }

// reduce_and_finish for FP32-pair values: the block's sums are formed in pair arithmetic
// (a block_sum in FP64 would cost ten FP64 additions per thread and value on this part)
// and stored as FP64 partials; the finishing block then proceeds as reduce_and_finish.
template <int NV>
__device__ bool reduce_and_finish_dw(const GridDev& G, int g, DW v[NV], double* part, int nblk_total,
                                     unsigned int* done, double tot[NV]) {
    __shared__ DW wsum[NV][32];
    __shared__ double scratch[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int a = 0; a < NV; a++) {
        const DW w = warp_sum_dw(v[a]);
        if (lane == 0) wsum[a][wid] = w;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int a = 0; a < NV; a++) {
            const DW w = warp_sum_dw(lane < nw ? wsum[a][lane] : DW{0.f, 0.f});
            if (lane == 0) part[a * nblk_total + blockIdx.x] = dw_join(w);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&done[g], 1u);
        last = (t == (unsigned)G.nblk - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int a = 0; a < NV; a++) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < G.nblk; b += blockDim.x)
            acc += __ldcg(&part[a * nblk_total + G.blk_first + b]);
        tot[a] = block_sum(acc, scratch);
    }
    if (threadIdx.x == 0) done[g] = 0u;
    return true;
}
// x-neighbours of a B-lattice component as pairs, with the conductor's images
__device__ __forceinline__ DW dw_nbx(const double* V, const Cell& c, int a) {
    DW e, w;
    if (a == 0) {  // odd
        e = c.ew ? DW{0.f, 0.f} : dw_from(V[c.ke]);
        w = c.ww ? dw_neg(dw_from(V[c.k + 1])) : dw_from(V[c.kw]);
    } else {
        e = dw_from(c.ew ? V[c.k] : V[c.ke]);
        w = dw_from(c.ww ? V[c.k] : V[c.kw]);
    }
    return dw_add(e, w);
}

__global__ void __launch_bounds__(kFieldThreads)
k_rhs_dw(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids, int nblk_total,
         long long ntot, const double* __restrict__ F, const long long* __restrict__ J, double* __restrict__ x,
         double* __restrict__ r, CgState* cg, double* part, unsigned int* done, DevStatus* st,
         cudaGraphConditionalHandle cond, int use_cond, double* __restrict__ bout, float* __restrict__ r32) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    float v[4] = {0.f, 0.f, 0.f, 0.f};  // b.b, r.r, |E|^2, |B|^2
    const DW AX = dwp(G.dw_ax), AY = dwp(G.dw_ay), KJX = dwp(G.dw_kjx), KJY = dwp(G.dw_kjy);
    const DW DTX = dwp(G.dw_dtx), DTY = dwp(G.dw_dty), C0 = dwp(G.dw_c0), CX = dwp(G.dw_cx), CY = dwp(G.dw_cy);
    if (!st->stop) FOR_CELLS(G, g, c) {
        const double* Ex = F;
        const double* Ey = F + ntot;
        const double* Ez = F + 2 * ntot;
        const long long* Jx = J;
        const long long* Jy = J + ntot;
        const long long* Jz = J + 2 * ntot;
        const DW ez = dw_from(Ez[c.k]), ey = dw_from(Ey[c.k]), ex = dw_from(Ex[c.k]);
        // dt curl E on the B lattices
        const DW eEx = dw_mul(DTY, dw_sub(dw_from(Ez[c.kn]), ez));
        const DW eEy = dw_neg(dw_mul(DTX, dw_sub(c.ew ? DW{0.f, 0.f} : dw_from(Ez[c.ke]), ez)));
        const DW eEz = dw_sub(dw_mul(DTX, dw_sub(c.ew ? DW{0.f, 0.f} : dw_from(Ey[c.ke]), ey)),
                              dw_mul(DTY, dw_sub(dw_from(Ex[c.kn]), ex)));
        // theta dt^2 4 pi curl J (the fixed-point unit folded into KJX, KJY)
        DW jJx, jJy, jJz;
        if (!G.walls) {
            jJx = dw_mul(KJY, dw_i64(Jz[c.kn] - Jz[c.k]));
            jJy = dw_neg(dw_mul(KJX, dw_i64(Jz[c.ke] - Jz[c.k])));
            jJz = dw_sub(dw_mul(KJX, dw_i64(Jy[c.ke] - Jy[c.k])), dw_mul(KJY, dw_i64(Jx[c.kn] - Jx[c.k])));
        } else {
            // the conductor carries the current of its wall nodes: Jy = Jz = 0 there
            const bool w0 = c.i == 0;
            const long long jzc = w0 ? 0 : Jz[c.k], jzn = w0 ? 0 : Jz[c.kn], jze = c.ew ? 0 : Jz[c.ke];
            const long long jyc = w0 ? 0 : Jy[c.k], jye = c.ew ? 0 : Jy[c.ke];
            jJx = dw_mul(KJY, dw_i64(jzn - jzc));
            jJy = dw_neg(dw_mul(KJX, dw_i64(jze - jzc)));
            jJz = dw_sub(dw_mul(KJX, dw_i64(jye - jyc)), dw_mul(KJY, dw_i64(Jx[c.kn] - Jx[c.k])));
        }
        const DW eE[3] = {eEx, eEy, eEz};
        const DW jJ[3] = {jJx, jJy, jJz};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double* B = F + (3 + a) * ntot;
            const DW bc = dw_from(B[c.k]);
            const DW b2 = dw_twice(bc);
            const DW lap = dw_add(dw_mul(AX, dw_sub(dw_nbx(B, c, a), b2)),
                                  dw_mul(AY, dw_sub(dw_add(dw_from(B[c.kn]), dw_from(B[c.ks])), b2)));
            const DW b = dw_add(lap, dw_sub(jJ[a], eE[a]));
            DW res = b;
            const long long o = a * ntot;
            if (G.warm == 1) {  // previous step's dB as the initial guess
                const double* X = x + o;
                const DW Ax = dw_sub(dw_mul(C0, dw_from(X[c.k])),
                                     dw_add(dw_mul(CX, dw_nbx(X, c, a)),
                                            dw_mul(CY, dw_add(dw_from(X[c.kn]), dw_from(X[c.ks])))));
                res = dw_sub(b, Ax);
                v[1] = fmaf(res.h, res.h, v[1]);
            }
            if (r) r[o + c.k] = dw_join(res);  // (the cooperative solve reads only the FP32 copy)
            if (r32) r32[o + c.k] = res.h;
            if (bout) bout[o + c.k] = dw_join(b);
            if (G.warm != 1) x[o + c.k] = 0.0;  // x0 = 0 (nothing here reads x then)
            v[0] = fmaf(b.h, b.h, v[0]);
            v[3] = fmaf(bc.h, bc.h, v[3]);
        }
        v[2] = fmaf(ex.h, ex.h, fmaf(ey.h, ey.h, fmaf(ez.h, ez.h, v[2])));
    }
    DW vd[4] = {{v[0], 0.f}, {v[1], 0.f}, {v[2], 0.f}, {v[3], 0.f}};
    double tot[4];
    if (!reduce_and_finish_dw<4>(G, g, vd, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        const double e = G.dx * G.dy / (8.0 * kPi);
        s.ue = tot[2] * e;
        s.ub = tot[3] * e;
        s.bb = tot[0];
        s.rr = G.warm == 1 ? tot[1] : tot[0];  // r = b unless the previous dB is the guess
        s.beta = 0.0;
        s.iters = 0;
        s.outer = 0;
        s.rel = tot[0] > 0.0 ? sqrt(s.rr / tot[0]) : 0.0;
        s.active = (!st->stop && tot[0] > 0.0 && s.rel > G.rtol) ? 1 : 0;
    }
    finish_all_grids(ngrids, ngrids, cg, st, cond, use_cond);
}

// Zero the solution where the warm start is off (x0 = 0), for the FP64 path. Separate
// from k_rhs because k_rhs reads x at neighbours when warm starting.
__global__ void __launch_bounds__(kFieldThreads)
k_zero_x(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
         double* __restrict__ x) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    if (G.warm == 1) return;
    FOR_CELLS(G, g, c) {
        x[c.k] = 0.0;
        x[ntot + c.k] = 0.0;
        x[2 * ntot + c.k] = 0.0;
    }
}

// ---- PCG iteration, part 1 ------------------------------------------------------
// With the Jacobi preconditioner of a constant-coefficient operator (diagonal c0), the
// preconditioned iterates equal plain CG's, so z = r is used. The A-product of the new
// direction p = r + beta p_old is formed as A r + beta (A p_old): A is linear, so this
// equals A p while touching only r at neighbours.
__global__ void __launch_bounds__(kFieldThreads)
k_cg_direction(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
               int nblk_total, long long ntot, const double* __restrict__ r,
               double* __restrict__ p, double* __restrict__ q, CgState* cg, double* part,
               unsigned int* done) {
    const int g = blk_grid[blockIdx.x];
    if (!cg[g].active) return;
    const GridDev& G = grids[g];
    const double beta = cg[g].beta;
    double v[1] = {0.0};
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const double* R = r + o;
            const double rc = R[c.k];
            const double Ar = G.c0 * rc - G.cx * nbx(R, c, a) - G.cy * (R[c.kn] + R[c.ks]);
            double pn, qn;
            if (beta == 0.0) {
                pn = rc;
                qn = Ar;
            } else {
                pn = rc + beta * p[o + c.k];
                qn = Ar + beta * q[o + c.k];
            }
            p[o + c.k] = pn;
            q[o + c.k] = qn;
            v[0] += pn * qn;
        }
    }
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) cg[g].alpha = cg[g].rr / tot[0];
}

// ---- PCG iteration, part 2 ------------------------------------------------------
// x += alpha p; r -= alpha A p; convergence test ||r|| <= rtol ||b||.
__global__ void __launch_bounds__(kFieldThreads)
k_cg_update(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
            int nblk_total, long long ntot, double* __restrict__ x, double* __restrict__ r,
            const double* __restrict__ p, const double* __restrict__ q, CgState* cg,
            double* part, unsigned int* done, DevStatus* st, cudaGraphConditionalHandle cond,
            int use_cond) {
    const int g = blk_grid[blockIdx.x];
    const unsigned n_part = st->n_active;  // simulations iterating in this launch
    if (!cg[g].active) return;
    const GridDev& G = grids[g];
    const double alpha = cg[g].alpha;
    double v[1] = {0.0};
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot + c.k;
            x[o] += alpha * p[o];
            const double rn = r[o] - alpha * q[o];
            r[o] = rn;
            v[0] += rn * rn;
        }
    }
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.beta = tot[0] / s.rr;
        s.rr = tot[0];
        s.iters += 1;
        s.rel = sqrt(tot[0] / s.bb);
        if (s.rel <= G.rtol) {
            s.active = 0;
        } else if (s.iters >= G.maxit) {
            s.active = 0;
            atomicAdd(&st->cg_noconv, 1u);
            st->stop_next = 1u;
        }
    }
    finish_all_grids(ngrids, (int)n_part, cg, st, cond, use_cond, 0);
}

// ---- Field update, Eqs. (5)-(6) --------------------------------------------------
// E^{n+1} = E^n + c dt curl(B^n + theta dB) - 4 pi dt J^{n+1/2}; the curl of a
// B-lattice vector lands on the E lattices.
template <typename JT>
__global__ void __launch_bounds__(kFieldThreads)
k_update_E(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
           double* __restrict__ F, const JT* __restrict__ J, const double* __restrict__ x,
           const CgState* __restrict__ cg, const DevStatus* st) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const double th = cg[g].bb > 0.0 ? G.theta : 0.0;  // dB = 0 when b = 0
    const double* Bx = F + 3 * ntot;
    const double* By = F + 4 * ntot;
    const double* Bz = F + 5 * ntot;
    const double* Xx = x;
    const double* Xy = x + ntot;
    const double* Xz = x + 2 * ntot;
    auto hx = [&](long long k) { return Bx[k] + th * Xx[k]; };
    auto hy = [&](long long k) { return By[k] + th * Xy[k]; };
    auto hz = [&](long long k) { return Bz[k] + th * Xz[k]; };
    // (constants folded: each term is one multiply-add on this part's slow FP64 pipe)
    const double fj = 4.0 * kPi * G.dt * ((sizeof(JT) == 8 && JT(1) / JT(2) == JT(0)) ? G.jinv : 1.0);
    const double dtx = G.dt * G.idx, dty = G.dt * G.idy;
    FOR_CELLS(G, g, c) {
        const double hzc = hz(c.k);
        const long long kw = c.ww ? c.k : c.kw;  // Bz, By even at a wall
        F[c.k] += fma(dty, hzc - hz(c.ks), -fj * (double)J[c.k]);
        if (c.ww) {  // the conductor keeps Ey = Ez = 0 on the wall
            F[ntot + c.k] = 0.0;
            F[2 * ntot + c.k] = 0.0;
        } else {
            F[ntot + c.k] += fma(-dtx, hzc - hz(kw), -fj * (double)J[ntot + c.k]);
            F[2 * ntot + c.k] += fma(dtx, hy(c.k) - hy(kw), fma(-dty, hx(c.k) - hx(c.ks), -fj * (double)J[2 * ntot + c.k]));
        }
    }
}

// The MIXED32 E update in FP32-pair arithmetic: the same formula and cells as
// k_update_E<long long>, joined back to FP64 with one add per component.
__global__ void __launch_bounds__(kFieldThreads)
k_update_E_dw(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
              double* __restrict__ F, const long long* __restrict__ J, const double* __restrict__ x,
              const CgState* __restrict__ cg, const DevStatus* st) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const DW TH = cg[g].bb > 0.0 ? dwp(G.dw_th) : DW{0.f, 0.f};  // dB = 0 when b = 0
    const DW FJ = dwp(G.dw_fj), DTX = dwp(G.dw_dtx), DTY = dwp(G.dw_dty);
    const double* Bx = F + 3 * ntot;
    const double* By = F + 4 * ntot;
    const double* Bz = F + 5 * ntot;
    const double* Xx = x;
    const double* Xy = x + ntot;
    const double* Xz = x + 2 * ntot;
    auto h = [&](const double* B, const double* X, long long k) { return dw_add(dw_from(B[k]), dw_mul(TH, dw_from(X[k]))); };
    FOR_CELLS(G, g, c) {
        const DW hzc = h(Bz, Xz, c.k);
        const long long kw = c.ww ? c.k : c.kw;  // Bz, By even at a wall
        const DW dEx = dw_sub(dw_mul(DTY, dw_sub(hzc, h(Bz, Xz, c.ks))), dw_mul(FJ, dw_i64(J[c.k])));
        F[c.k] = dw_join(dw_add(dw_from(F[c.k]), dEx));
        if (c.ww) {  // the conductor keeps Ey = Ez = 0 on the wall
            F[ntot + c.k] = 0.0;
            F[2 * ntot + c.k] = 0.0;
        } else {
            const DW dEy = dw_neg(dw_add(dw_mul(DTX, dw_sub(hzc, h(Bz, Xz, kw))), dw_mul(FJ, dw_i64(J[ntot + c.k]))));
            const DW dEz = dw_sub(dw_sub(dw_mul(DTX, dw_sub(h(By, Xy, c.k), h(By, Xy, kw))),
                                         dw_mul(DTY, dw_sub(h(Bx, Xx, c.k), h(Bx, Xx, c.ks)))),
                                  dw_mul(FJ, dw_i64(J[2 * ntot + c.k])));
            F[ntot + c.k] = dw_join(dw_add(dw_from(F[ntot + c.k]), dEy));
            F[2 * ntot + c.k] = dw_join(dw_add(dw_from(F[2 * ntot + c.k]), dEz));
        }
    }
}

// Vector access to four consecutive FP64 values (16-byte aligned: cell offsets and nx are
// multiples of 4 where the quad kernels run).
__device__ __forceinline__ void ld4d(const double* p, double v[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
__device__ __forceinline__ void st4d(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// Grid-stride loop over the quads (4 cells along x) of simulation g, for nx a multiple
// of 4: quad q covers cells 4q .. 4q + 3 of the simulation, in one row.
#define FOR_QUADS(G, l)                                                                        \
    for (int q_ = (blockIdx.x - (G).blk_first) * blockDim.x + threadIdx.x; q_ < ((G).ncell >> 2); \
         q_ += (G).nblk * blockDim.x)                                                          \
        if (const int l = 4 * q_; true)

// k_update_E_dw on quads of cells, for nx a multiple of 4: the same pair arithmetic per
// cell (so the same bits), with B, dB, E and J moved as vectors and more loads in flight
// per thread. The quad's west neighbour is one scalar load.
__global__ void __launch_bounds__(kFieldThreads)
k_update_E_dw4(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
               double* __restrict__ F, const long long* __restrict__ J, const double* __restrict__ x,
               const CgState* __restrict__ cg, const DevStatus* st) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const DW TH = cg[g].bb > 0.0 ? dwp(G.dw_th) : DW{0.f, 0.f};  // dB = 0 when b = 0
    const DW FJ = dwp(G.dw_fj), DTX = dwp(G.dw_dtx), DTY = dwp(G.dw_dty);
    const double* B = F + 3 * ntot;
    // B + theta dB of component c at the quad starting at k, and at one cell
    const auto h4 = [&](int c, long long k, DW h[4]) {
        double bv[4], xv[4];
        ld4d(B + c * ntot + k, bv);
        ld4d(x + c * ntot + k, xv);
#pragma unroll
        for (int u = 0; u < 4; u++) h[u] = dw_add(dw_from(bv[u]), dw_mul(TH, dw_from(xv[u])));
    };
    const auto h1 = [&](int c, long long k) {
        return dw_add(dw_from(B[c * ntot + k]), dw_mul(TH, dw_from(x[c * ntot + k])));
    };
    const auto j4 = [&](int c, long long k, DW j[4]) {
        const longlong2 v0 = reinterpret_cast<const longlong2*>(J + c * ntot + k)[0];
        const longlong2 v1 = reinterpret_cast<const longlong2*>(J + c * ntot + k)[1];
        j[0] = dw_mul(FJ, dw_i64(v0.x));
        j[1] = dw_mul(FJ, dw_i64(v0.y));
        j[2] = dw_mul(FJ, dw_i64(v1.x));
        j[3] = dw_mul(FJ, dw_i64(v1.y));
    };
    FOR_QUADS(G, l) {
        const int jr = l / G.nx, i = l - jr * G.nx;
        const long long row = G.cell_off + (long long)jr * G.nx;
        const long long k = row + i;
        const bool ww = G.walls && i == 0;
        const long long kw = ww ? k : row + (i == 0 ? G.nx - 1 : i - 1);  // Bz, By even at a wall
        const long long ks = G.cell_off + (long long)(jr == 0 ? G.ny - 1 : jr - 1) * G.nx + i;
        DW hz[4], t[4], jj[4];
        double e[4];
        h4(2, k, hz);
        h4(2, ks, t);
        j4(0, k, jj);
        ld4d(F + k, e);  // Ex
#pragma unroll
        for (int u = 0; u < 4; u++) e[u] = dw_join(dw_add(dw_from(e[u]), dw_sub(dw_mul(DTY, dw_sub(hz[u], t[u])), jj[u])));
        st4d(F + k, e);
        {
            const DW hzw = h1(2, kw);
            j4(1, k, jj);
            ld4d(F + ntot + k, e);  // Ey
#pragma unroll
            for (int u = 0; u < 4; u++)
                e[u] = dw_join(dw_add(dw_from(e[u]), dw_neg(dw_add(dw_mul(DTX, dw_sub(hz[u], u == 0 ? hzw : hz[u - 1])), jj[u]))));
            if (ww) e[0] = 0.0;  // the conductor keeps Ey = Ez = 0 on the wall
            st4d(F + ntot + k, e);
        }
        {
            DW hy[4];
            const DW hyw = h1(1, kw);
            h4(1, k, hy);
            h4(0, k, hz);  // Bx + theta dBx at the quad
            h4(0, ks, t);  // and south of it
            j4(2, k, jj);
            ld4d(F + 2 * ntot + k, e);  // Ez
#pragma unroll
            for (int u = 0; u < 4; u++)
                e[u] = dw_join(dw_add(dw_from(e[u]), dw_sub(dw_sub(dw_mul(DTX, dw_sub(hy[u], u == 0 ? hyw : hy[u - 1])),
                                                                 dw_mul(DTY, dw_sub(hz[u], t[u]))),
                                                          jj[u])));
            if (ww) e[0] = 0.0;
            st4d(F + 2 * ntot + k, e);
        }
    }
}

// k_update_B on quads of cells (nx a multiple of 4): B += dB and the FP32 copies.
__global__ void __launch_bounds__(kFieldThreads)
k_update_B4(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
            double* __restrict__ F, const double* __restrict__ x, const CgState* __restrict__ cg,
            const DevStatus* st, float* __restrict__ F32) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const bool have = cg[g].bb > 0.0;
    FOR_QUADS(G, l) {
        const long long k = G.cell_off + l;
        double bv[3][4], xv[3][4], ev[3][4];
#pragma unroll
        for (int a = 0; a < 3; a++) {  // every load first
            ld4d(F + (3 + a) * ntot + k, bv[a]);
            if (have) {
                ld4d(x + a * ntot + k, xv[a]);
            } else {
#pragma unroll
                for (int u = 0; u < 4; u++) xv[a][u] = 0.0;
            }
            if (F32) ld4d(F + a * ntot + k, ev[a]);
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
#pragma unroll
            for (int u = 0; u < 4; u++) bv[a][u] += xv[a][u];
            st4d(F + (3 + a) * ntot + k, bv[a]);
            if (F32) {  // (float) by bit manipulation off the FP64 pipe
                reinterpret_cast<float4*>(F32 + (3 + a) * ntot + k)[0] =
                    make_float4(f32_rn(bv[a][0]), f32_rn(bv[a][1]), f32_rn(bv[a][2]), f32_rn(bv[a][3]));
                reinterpret_cast<float4*>(F32 + a * ntot + k)[0] =
                    make_float4(f32_rn(ev[a][0]), f32_rn(ev[a][1]), f32_rn(ev[a][2]), f32_rn(ev[a][3]));
            }
        }
    }
}

// Explicit FDTD (Eqs. 3-4; PIC_EXPLICIT), with B kept at integer time levels for the
// gather: x = B^{n+1/2} - B^n = -(c dt/2) curl E^n here, together with the energies of
// level n; then k_update_E with theta = 1 applies E^{n+1} = E^n + c dt curl B^{n+1/2}
// - 4 pi dt J; then k_explicit_B forms B^{n+1} = B^{n+1/2} - (c dt/2) curl E^{n+1}.
__global__ void __launch_bounds__(kFieldThreads)
k_explicit_half(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int nblk_total,
                long long ntot, const double* __restrict__ F, double* __restrict__ x, CgState* cg,
                double* part, unsigned int* done, const DevStatus* st) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    double v[2] = {0.0, 0.0};  // |E|^2, |B|^2
    if (!st->stop) FOR_CELLS(G, g, c) {
        const double* Ex = F;
        const double* Ey = F + ntot;
        const double* Ez = F + 2 * ntot;
        const double ez = Ez[c.k];
        const double h = -0.5 * G.dt;
        x[c.k] = h * (Ez[c.kn] - ez) * G.idy;
        x[ntot + c.k] = -h * (east_odd(Ez, c) - ez) * G.idx;
        x[2 * ntot + c.k] = h * ((east_odd(Ey, c) - Ey[c.k]) * G.idx - (Ex[c.kn] - Ex[c.k]) * G.idy);
        v[0] += Ex[c.k] * Ex[c.k] + Ey[c.k] * Ey[c.k] + ez * ez;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double b = F[(3 + a) * ntot + c.k];
            v[1] += b * b;
        }
    }
    double tot[2];
    if (!reduce_and_finish<2>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        const double e = G.dx * G.dy / (8.0 * kPi);
        s.ue = tot[0] * e;
        s.ub = tot[1] * e;
        s.bb = 1.0;  // k_update_E applies x (with theta = 1)
        s.rr = 0.0;
        s.rel = 0.0;
        s.iters = 0;
        s.outer = 0;
        s.active = 0;
    }
}

__global__ void __launch_bounds__(kFieldThreads)
k_explicit_B(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
             double* __restrict__ F, const double* __restrict__ x, const DevStatus* st,
             float* __restrict__ F32) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const double* Ex = F;
    const double* Ey = F + ntot;
    const double* Ez = F + 2 * ntot;
    const double h = -0.5 * G.dt;
    FOR_CELLS(G, g, c) {
        const double ez = Ez[c.k];
        const double dB[3] = {h * (Ez[c.kn] - ez) * G.idy, -h * (east_odd(Ez, c) - ez) * G.idx,
                              h * ((east_odd(Ey, c) - Ey[c.k]) * G.idx - (Ex[c.kn] - Ex[c.k]) * G.idy)};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = (3 + a) * ntot + c.k;
            const double b = F[o] + x[a * ntot + c.k] + dB[a];
            F[o] = b;
            if (F32) F32[o] = (float)b;
        }
        if (F32) {
            F32[c.k] = (float)Ex[c.k];
            F32[ntot + c.k] = (float)Ey[c.k];
            F32[2 * ntot + c.k] = (float)ez;
        }
    }
}

// B^{n+1} = B^n + dB, then the FP32 copies used by the MIXED32 gather.
__global__ void __launch_bounds__(kFieldThreads)
k_update_B(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
           double* __restrict__ F, const double* __restrict__ x, const CgState* __restrict__ cg,
           const DevStatus* st, float* __restrict__ F32) {
    if (st->stop) return;
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const bool have = cg[g].bb > 0.0;
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = (3 + a) * ntot + c.k;
            const double b = F[o] + (have ? x[a * ntot + c.k] : 0.0);
            F[o] = b;
            if (F32) F32[o] = f32_rn(b);  // (float)b, by bit manipulation off the FP64 pipe
        }
        if (F32) {
#pragma unroll
            for (int a = 0; a < 3; a++) F32[a * ntot + c.k] = f32_rn(F[a * ntot + c.k]);
        }
    }
}

// The alternative gather reading (PIC_GATHER_NODAL): E and B averaged from their
// staggered lattices to the nodes -- Ex, By over their two x-neighbours, Ey, Bx over
// their two y-neighbours, Bz over the four surrounding cells; Ez already sits on the
// nodes -- for the particle kernels, which then gather every component with the node
// weights of the charge deposit. Periodic boundaries only.
__global__ void __launch_bounds__(kFieldThreads)
k_nodal(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
        const double* __restrict__ F, double* __restrict__ Fn, float* __restrict__ F32) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    if (!G.nodal) return;
    FOR_CELLS(G, g, c) {
        const long long ksw = c.ks + (c.kw - c.k);  // south-west neighbour
        double v[6];
        v[0] = 0.5 * (F[c.kw] + F[c.k]);
        v[1] = 0.5 * (F[ntot + c.ks] + F[ntot + c.k]);
        v[2] = F[2 * ntot + c.k];
        v[3] = 0.5 * (F[3 * ntot + c.ks] + F[3 * ntot + c.k]);
        v[4] = 0.5 * (F[4 * ntot + c.kw] + F[4 * ntot + c.k]);
        v[5] = 0.25 * ((F[5 * ntot + ksw] + F[5 * ntot + c.ks]) + (F[5 * ntot + c.kw] + F[5 * ntot + c.k]));
#pragma unroll
        for (int a = 0; a < 6; a++) {
            if (Fn) Fn[a * ntot + c.k] = v[a];
            if (F32) F32[a * ntot + c.k] = (float)v[a];
        }
    }
}

__global__ void __launch_bounds__(kFieldThreads)
k_to_f32(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
         const double* __restrict__ F, float* __restrict__ F32) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 6; a++) F32[a * ntot + c.k] = (float)F[a * ntot + c.k];
    }
}

// Start of a step: an error raised during the previous step stops this one; clear the
// per-step kinetic-energy accumulators.
__global__ void k_step_begin(int ngrids, CgState* cg, DevStatus* st) {
    if (threadIdx.x == 0) {
        if (st->stop_next) st->stop = 1u;
        if (!st->stop) st->steps_done += 1ull;
    }
    for (int g = threadIdx.x; g < ngrids; g += blockDim.x) cg[g].uk = 0.0;
}

// End of a step: PCG statistics.
__global__ void k_step_end(int ngrids, CgState* cg, const DevStatus* st) {
    if (st->stop) return;
    for (int g = threadIdx.x; g < ngrids; g += blockDim.x) {
        CgState& s = cg[g];
        s.last_iters = s.iters;
        s.max_iters = s.iters > s.max_iters ? s.iters : s.max_iters;
        s.total_iters += s.iters;
    }
}

// ---- Mixed-precision PCG (MIXED32) ----------------------------------------------
// Iterative refinement around an FP32 inner CG: with the FP64 residual r = b - A x, the
// inner loop solves A e = r in FP32 vectors (dot products accumulated in FP64) to a
// relative tolerance tol_in, then x += e and r = b - A x are formed in FP64. The outer
// test is the same ||r||_2 <= rtol ||b||_2 on the FP64 residual, so the solution meets
// the tolerance of the plain FP64 PCG while most vector traffic and arithmetic is FP32.
constexpr int kMaxInnerIters = 64;

// Inner preconditioned CG (MIXED32): z = M r with M = pc0 I + pcx (E + W) + pcy (N + S)
// (GridDev), the same 5-point shape and wall images as A.
template <typename T>
__device__ __forceinline__ T precond_at(const GridDev& G, const T* V, const Cell& c, int a) {
    return T(G.pc0) * V[c.k] + T(G.pcx) * nbx(V, c, a) + T(G.pcy) * (V[c.kn] + V[c.ks]);
}

// r32 = r / rms(r) (buffer 0), e = 0, z = M r32; (r, r) and (r, z).
__global__ void __launch_bounds__(kFieldThreads)
k_mp_begin(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
           int nblk_total, long long ntot, const double* __restrict__ r, float* __restrict__ r32,
           float* __restrict__ z32, float* __restrict__ e32, CgState* cg, double* part, unsigned int* done,
           DevStatus* st, cudaGraphConditionalHandle cond_in, int use_cond) {
    const int g = blk_grid[blockIdx.x];
    const unsigned n_part = st->n_active;
    if (!cg[g].active) return;
    const GridDev& G = grids[g];
    const double scale = sqrt(3.0 * G.ncell / cg[g].rr);  // r32 of unit RMS
    float acc = 0.f, acc2 = 0.f;
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot + c.k;
            const float f = (float)(r[o] * scale);
            const float z = (float)(precond_at(G, r + a * ntot, c, a) * scale);
            r32[o] = f;
            z32[o] = z;
            e32[o] = 0.f;
            acc = fmaf(f, f, acc);
            acc2 = fmaf(f, z, acc2);
        }
    }
    double v[2] = {(double)acc, (double)acc2};
    double tot[2];
    if (!reduce_and_finish<2>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.rr_in0 = tot[0];
        s.rr_in = tot[0];
        s.rz_in = tot[1];
        s.beta_in = 0.0;
        s.in_iters = 0;
        s.in_scale = scale;
        // ask the inner loop for what the outer test still needs, within FP32's reach
        s.tol_in = fmax(2e-6, 0.5 * G.rtol * sqrt(s.bb / fmax(s.rr, 1e-300)));
        s.in_active = (tot[0] > 0.0 && tot[1] > 0.0) ? 1 : 0;
    }
    finish_all_grids<true>(ngrids, (int)n_part, cg, st, cond_in, use_cond);
}

// p = z + beta p, q = A z + beta q (= A p); alpha = (r, z) / (p, q).
__global__ void __launch_bounds__(kFieldThreads)
k_mp_direction(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
               int nblk_total, long long ntot, const float* __restrict__ z32, float* __restrict__ p32,
               float* __restrict__ q32, CgState* cg, double* part, unsigned int* done) {
    const int g = blk_grid[blockIdx.x];
    if (!cg[g].in_active) return;
    const GridDev& G = grids[g];
    const float beta = (float)cg[g].beta_in;
    const float c0 = (float)G.c0, cx = (float)G.cx, cy = (float)G.cy;
    float acc = 0.f;  // a thread's few products in FP32, summed across threads in FP64
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const float* Z = z32 + o;
            const float zc = Z[c.k];
            const float Az = c0 * zc - cx * nbx(Z, c, a) - cy * (Z[c.kn] + Z[c.ks]);
            float pn, qn;
            if (beta == 0.f) {
                pn = zc;
                qn = Az;
            } else {
                pn = fmaf(beta, p32[o + c.k], zc);
                qn = fmaf(beta, q32[o + c.k], Az);
            }
            p32[o + c.k] = pn;
            q32[o + c.k] = qn;
            acc = fmaf(pn, qn, acc);
        }
    }
    double v[1] = {(double)acc};
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) cg[g].alpha_in = cg[g].rz_in / tot[0];
}

// r' = r - alpha q into the other residual buffer, e += alpha p, z = M r' (formed from r
// and q at the neighbours, which this kernel does not change); beta = (r', z) / (r, z).
__global__ void __launch_bounds__(kFieldThreads)
k_mp_update(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
            int nblk_total, long long ntot, float* __restrict__ e32, float* __restrict__ r32a,
            float* __restrict__ r32b, float* __restrict__ z32, const float* __restrict__ p32,
            const float* __restrict__ q32, CgState* cg, double* part, unsigned int* done, DevStatus* st,
            cudaGraphConditionalHandle cond_in, int use_cond) {
    const int g = blk_grid[blockIdx.x];
    const unsigned n_part = st->n_in_active;
    if (!cg[g].in_active) return;
    const GridDev& G = grids[g];
    const float alpha = (float)cg[g].alpha_in;
    const float pc0 = (float)G.pc0, pcx = (float)G.pcx, pcy = (float)G.pcy;
    const bool odd = cg[g].in_iters & 1;  // buffer b holds r after an odd number of updates
    const float* Rc = odd ? r32b : r32a;
    float* Rn = odd ? r32a : r32b;
    float acc = 0.f, acc2 = 0.f;
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const float* R = Rc + o;
            const float* Q = q32 + o;
            const auto w = [&](long long k) { return fmaf(-alpha, Q[k], R[k]); };
            const float wc = w(c.k);
            float wx;  // sum of the two x-neighbours, images at the walls as in nbx
            if (a == 0) wx = (c.ew ? 0.f : w(c.ke)) + (c.ww ? -w(c.k + 1) : w(c.kw));
            else wx = (c.ew ? wc : w(c.ke)) + (c.ww ? wc : w(c.kw));
            const float z = fmaf(pc0, wc, fmaf(pcx, wx, pcy * (w(c.kn) + w(c.ks))));
            Rn[o + c.k] = wc;
            z32[o + c.k] = z;
            e32[o + c.k] = fmaf(alpha, p32[o + c.k], e32[o + c.k]);
            acc = fmaf(wc, wc, acc);
            acc2 = fmaf(wc, z, acc2);
        }
    }
    double v[2] = {(double)acc, (double)acc2};
    double tot[2];
    if (!reduce_and_finish<2>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.beta_in = tot[1] / s.rz_in;
        s.rz_in = tot[1];
        s.rr_in = tot[0];
        s.in_iters += 1;
        s.iters += 1;
        if (sqrt(tot[0] / s.rr_in0) <= s.tol_in || s.in_iters >= kMaxInnerIters || s.iters >= G.maxit ||
            !(tot[1] > 0.0))
            s.in_active = 0;
    }
    finish_all_grids<true>(ngrids, (int)n_part, cg, st, cond_in, use_cond, 0);
}

// x += e (FP64).
__global__ void __launch_bounds__(kFieldThreads)
k_mp_x(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, long long ntot,
       double* __restrict__ x, const float* __restrict__ e32, const CgState* __restrict__ cg) {
    const int g = blk_grid[blockIdx.x];
    if (!cg[g].active) return;
    const GridDev& G = grids[g];
    const double inv = 1.0 / cg[g].in_scale;
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) x[a * ntot + c.k] += (double)e32[a * ntot + c.k] * inv;
    }
}

// r = b - A x (FP64) and the outer convergence test.
__global__ void __launch_bounds__(kFieldThreads)
k_mp_r(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
       int nblk_total, long long ntot, const double* __restrict__ b, const double* __restrict__ x,
       double* __restrict__ r, CgState* cg, double* part, unsigned int* done, DevStatus* st,
       cudaGraphConditionalHandle cond, int use_cond) {
    const int g = blk_grid[blockIdx.x];
    const unsigned n_part = st->n_active;
    if (!cg[g].active) return;
    const GridDev& G = grids[g];
    double v[1] = {0.0};
    FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const double* X = x + o;
            const double Ax = G.c0 * X[c.k] - G.cx * nbx(X, c, a) - G.cy * (X[c.kn] + X[c.ks]);
            const double rn = b[o + c.k] - Ax;
            r[o + c.k] = rn;
            v[0] += rn * rn;
        }
    }
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.rr = tot[0];
        s.rel = sqrt(tot[0] / s.bb);
        s.outer += 1;
        s.total_outer += 1;
        if (s.rel <= G.rtol) {
            s.active = 0;
        } else if (s.iters >= G.maxit || s.outer >= G.maxit) {
            s.active = 0;
            atomicAdd(&st->cg_noconv, 1u);
            st->stop_next = 1u;
        }
    }
    finish_all_grids(ngrids, (int)n_part, cg, st, cond, use_cond, 1);
}

// After a learned initial guess x0 (every simulation): r = b - A x0 (FP64) and the
// starting state of the PCG loop, as k_rhs sets it for the plain guesses.
__global__ void __launch_bounds__(kFieldThreads)
k_guess_residual(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
                 int nblk_total, long long ntot, const double* __restrict__ b, const double* __restrict__ x,
                 double* __restrict__ r, CgState* cg, double* part, unsigned int* done, DevStatus* st,
                 cudaGraphConditionalHandle cond, int use_cond, float* __restrict__ r32) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    double v[1] = {0.0};
    if (!st->stop) FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const double* X = x + o;
            const double Ax = G.c0 * X[c.k] - G.cx * nbx(X, c, a) - G.cy * (X[c.kn] + X[c.ks]);
            const double rn = b[o + c.k] - Ax;
            r[o + c.k] = rn;
            if (r32) r32[o + c.k] = (float)rn;  // FP32 copy for the cooperative solve
            v[0] += rn * rn;
        }
    }
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.rr = tot[0];
        s.rel = s.bb > 0.0 ? sqrt(tot[0] / s.bb) : 0.0;
        s.active = (!st->stop && s.bb > 0.0 && s.rel > G.rtol) ? 1 : 0;
    }
    finish_all_grids(ngrids, ngrids, cg, st, cond, use_cond);
}

// The same for the cooperative solve, in FP32: r32 (the FP32 copy of b that k_rhs left)
// minus A x0 from the guess's FP32 copy. This residual only starts the first inner FP32
// solve; the refinement after it forms the FP64 residual of the updated solution.
__global__ void __launch_bounds__(kFieldThreads)
k_guess_residual32(const GridDev* __restrict__ grids, const int* __restrict__ blk_grid, int ngrids,
                   int nblk_total, long long ntot, const float* __restrict__ x32, float* __restrict__ r32,
                   CgState* cg, double* part, unsigned int* done, DevStatus* st, cudaGraphConditionalHandle cond,
                   int use_cond) {
    const int g = blk_grid[blockIdx.x];
    const GridDev& G = grids[g];
    const float c0 = (float)G.c0, cx = (float)G.cx, cy = (float)G.cy;
    float acc = 0.f;
    if (!st->stop) FOR_CELLS(G, g, c) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const long long o = a * ntot;
            const float* X = x32 + o;
            const float Ax = c0 * X[c.k] - cx * nbx(X, c, a) - cy * (X[c.kn] + X[c.ks]);
            const float rn = r32[o + c.k] - Ax;
            r32[o + c.k] = rn;
            acc = fmaf(rn, rn, acc);
        }
    }
    double v[1] = {(double)acc};
    double tot[1];
    if (!reduce_and_finish<1>(G, g, v, part, nblk_total, done, tot)) return;
    if (threadIdx.x == 0) {
        CgState& s = cg[g];
        s.rr = tot[0];
        s.rel = s.bb > 0.0 ? sqrt(tot[0] / s.bb) : 0.0;
        s.active = (!st->stop && s.bb > 0.0 && s.rel > G.rtol) ? 1 : 0;
    }
    finish_all_grids(ngrids, ngrids, cg, st, cond, use_cond);
}

}  // namespace

void launch_guess_residual32(const FieldArgs& a, cudaStream_t s) {
    k_guess_residual32<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot, a.e32,
                                                        a.r32, a.cg, a.part, a.done, a.st, a.cond, a.use_cond);
}

void launch_guess_residual(const FieldArgs& a, cudaStream_t s) {
    k_guess_residual<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot, a.b, a.x,
                                                      a.r, a.cg, a.part, a.done, a.st, a.cond, a.use_cond, a.r32);
}

void launch_step_begin(const FieldArgs& a, cudaStream_t s) {
    k_step_begin<<<1, 128, 0, s>>>(a.ngrids, a.cg, a.st);
}

void launch_step_end(const FieldArgs& a, cudaStream_t s) {
    k_step_end<<<1, 128, 0, s>>>(a.ngrids, a.cg, a.st);
}

void launch_rhs(const FieldArgs& a, cudaStream_t s) {
    if (!a.Jfix) k_zero_x<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.x);  // (k_rhs_dw zeroes x itself)
    if (a.Jfix)
        k_rhs_dw<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot, a.F, a.Jfix, a.x,
                                                  a.coop ? nullptr : a.r, a.cg, a.part, a.done, a.st, a.cond,
                                                  a.use_cond, a.b, a.r32);
    else
        k_rhs<double><<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk,
                                                       a.ntot, a.F, a.J64, a.x, a.r, a.cg,
                                                       a.part, a.done, a.st, a.cond, a.use_cond,
                                                       a.b, a.r32);
}

void launch_mp_inner_begin(const FieldArgs& a, cudaStream_t s) {
    k_mp_begin<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot, a.r,
                                                a.r32, a.z32, a.e32, a.cg, a.part, a.done, a.st, a.cond_in,
                                                a.use_cond);
}

void launch_mp_inner_iteration(const FieldArgs& a, cudaStream_t s) {
    k_mp_direction<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot,
                                                    a.z32, a.p32, a.q32, a.cg, a.part, a.done);
    k_mp_update<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot,
                                                 a.e32, a.r32, a.r32b, a.z32, a.p32, a.q32, a.cg, a.part,
                                                 a.done, a.st, a.cond_in, a.use_cond);
}

void launch_mp_refine(const FieldArgs& a, cudaStream_t s) {
    k_mp_x<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.x, a.e32, a.cg);
    k_mp_r<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot, a.b,
                                            a.x, a.r, a.cg, a.part, a.done, a.st, a.cond,
                                            a.use_cond);
}

void launch_explicit_fields(const FieldArgs& a, cudaStream_t s) {
    k_explicit_half<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.nblk, a.ntot, a.F, a.x, a.cg,
                                                     a.part, a.done, a.st);
    if (a.Jfix)
        k_update_E<long long><<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.Jfix, a.x,
                                                               a.cg, a.st);
    else
        k_update_E<double><<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.J64, a.x,
                                                            a.cg, a.st);
    k_explicit_B<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.x, a.st, a.F32);
}

void launch_cg_iteration(const FieldArgs& a, cudaStream_t s) {
    k_cg_direction<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk,
                                                    a.ntot, a.r, a.p, a.q, a.cg, a.part, a.done);
    k_cg_update<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ngrids, a.nblk, a.ntot,
                                                 a.x, a.r, a.p, a.q, a.cg, a.part, a.done, a.st,
                                                 a.cond, a.use_cond);
}

void launch_field_update(const FieldArgs& a, cudaStream_t s) {
    if (a.Jfix && a.quads)
        k_update_E_dw4<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.Jfix, a.x, a.cg,
                                                        a.st);
    else if (a.Jfix)
        k_update_E_dw<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.Jfix, a.x, a.cg,
                                                       a.st);
    else
        k_update_E<double><<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F,
                                                            a.J64, a.x, a.cg, a.st);
    if (a.Jfix && a.quads)
        k_update_B4<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.x, a.cg, a.st,
                                                     a.F32);
    else
        k_update_B<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.x, a.cg,
                                                    a.st, a.F32);
}

void launch_nodal(const FieldArgs& a, cudaStream_t s) {
    if (a.any_nodal) k_nodal<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.Fn, a.F32);
}

void launch_fields_to_f32(const FieldArgs& a, cudaStream_t s) {
    if (a.F32) k_to_f32<<<a.nblk, kFieldThreads, 0, s>>>(a.grids, a.blk_grid, a.ntot, a.F, a.F32);
    launch_nodal(a, s);
}

}  // namespace pic
