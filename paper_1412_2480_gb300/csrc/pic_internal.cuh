// pic_internal.cuh -- device-side data structures and helpers of the GB300 PIC library.
//
// Everything a kernel needs to know about one simulation lives in GridDev; several
// simulations can share one launch (the batched parameter scan), so every kernel maps
// its block to a simulation through a small table instead of assuming one grid.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pic {

constexpr double kPi = 3.14159265358979323846;
constexpr int kFieldThreads = 256;  // threads per block of the grid (field) kernels
constexpr int kPushThreads = 256;   // threads per block of the FP64 particle kernel
// Largest tile window (cells) of the MIXED32 kernel: 48 bytes of shared memory per cell
// (six FP32 field words and six fixed-point current words) within the 227 KB of a CTA.
constexpr int kMaxWinCells = 4800;

// One simulation, as the kernels see it. Grid arrays of all simulations are
// concatenated; cell_off is this simulation's first cell.
struct GridDev {
    int nx, ny, order, ncell;
    double dx, dy, dt, theta;
    double idx, idy;      // 1/dx, 1/dy
    double a;             // (theta dt)^2, the coefficient of Eq. (7)
    double c0, cx, cy;    // A v = c0 v - cx (v_e + v_w) - cy (v_n + v_s)
    // Preconditioner of the MIXED32 inner CG, z = M r with M = pc0 I + pcx (E + W) +
    // pcy (N + S) = p(A): the degree-1 polynomial that minimises max |1 - lambda p(lambda)|
    // over A's spectrum [1, c0 + 2 cx + 2 cy] (Chebyshev; the same 5-point shape and wall
    // images as A)
    double pc0, pcx, pcy;
    long long cell_off;
    int blk_first, nblk;  // this simulation's blocks in field-kernel launches
    double qw[2], qm[2];  // charge per macro-particle and charge-to-mass sign per species
    double w;             // macro weight (mass per macro-particle)
    double rtol;
    int maxit, warm;      // warm: 0 zero guess, 1 previous dB, 2 learned guess
    int deposit;          // 0 in test-particle mode
    int walls;            // conducting, reflecting walls at x = 0 and x = nx dx (else periodic)
    int nodal;            // gather reading: fields averaged to the nodes first (PIC_GATHER_NODAL)
    // moving injector (walls only; include/pic.h)
    int inject, ppc;
    double inj_x0, cfl, gamma0, u_th;
    unsigned long long inj_seed;
    // MIXED32 tiling
    int tx, ty, ntx, nty; // tile size and tile counts
    int tile_first, ntiles;
    int wx, wy;           // tile window size: (tx + 5) x (ty + 5), origin (X0-2, Y0-2)
    int cpt, cpt_pad;     // cells per tile (tx ty) and that rounded up to a multiple of 32
    int rcap;             // layers of a bin: particles per cell it can hold
    long long cap;        // layered capacity rcap * cpt_pad per (tile, species) bin
    long long capo;       // capacity of each of the 8 outboxes of a bin
    long long bin_off;    // first particle slot of this simulation's bins
    // MIXED32 current: 64-bit fixed point, J = (double)Jfix * jinv
    double jscale, jinv;
    // MIXED32 push constants, formed once on the host from the FP64 parameters (the FP64
    // pipe is slow on this part, and every thread of a tile would otherwise form them):
    // per species h = (q/m) dt/2, fx = q dx/(dt dx dy), fy = q dy/(dt dx dy),
    // fz = q/(dx dy); dt/dx, dt/dy; js40 = jscale 2^-40 (a tile's window scale is js40 2^k)
    float pk_h[2], pk_fx[2], pk_fy[2], pk_fz[2];
    float pk_dtx, pk_dty, js40;
    // MIXED32 field constants as FP32 pairs (h, l), formed once on the host: the
    // right-hand side's theta dt^2/dx^2, theta dt^2/dy^2, 4 pi theta dt^2 jinv/dx and /dy,
    // dt/dx, dt/dy; A's c0, cx, cy; the E update's 4 pi dt jinv and theta
    float dw_ax[2], dw_ay[2], dw_kjx[2], dw_kjy[2], dw_dtx[2], dw_dty[2];
    float dw_c0[2], dw_cx[2], dw_cy[2], dw_fj[2], dw_th[2];
};

// Per-simulation state of the PCG solve of Eq. (7).
struct CgState {
    double bb, rr, pq, alpha, beta, rel;
    double ue, ub, uk;    // energies of the step being computed (time level n)
    int active, iters, last_iters, max_iters;
    long long total_iters;
    // mixed-precision refinement (MIXED32): FP32 inner CG on A e = r
    double rr_in, rr_in0, alpha_in, beta_in, tol_in;
    double rz_in;     // (r, z) of the preconditioned inner CG
    double in_scale;  // r32 = r * in_scale (unit RMS), e = e32 / in_scale
    int in_active, in_iters, outer, pad;
    long long total_outer;  // FP64 refinements (outer iterations) of all steps
};

// Device status words shared by all kernels of a handle.
struct DevStatus {
    unsigned long long cfl_viol;     // moves of >= 1 cell
    unsigned long long nan_count;    // non-finite momenta or positions
    unsigned long long overflow;     // MIXED32: particles sent through the overflow path
    unsigned int cg_noconv;          // PCG hit maxit
    unsigned int stop;               // nonzero: this and later steps of the call are skipped
    unsigned int stop_next;          // set during a step; becomes `stop` at the next step
    unsigned long long steps_done;   // steps completed (the failing step included)
    unsigned int grids_done;         // counter of the last-grid-finished pattern
    unsigned int n_active;           // simulations whose PCG is still iterating
    unsigned int n_in_active;        // simulations whose inner FP32 CG is still iterating
    unsigned long long lost;         // MIXED32: particles dropped because the overflow list was full
    unsigned int parity;             // MIXED32: which of the two bin buffers is current
    unsigned long long ovf_count[2]; // MIXED32: particles in each overflow list
    unsigned long long loop_iters[2]; // PCG loop iterations run: [0] CG (inner) iterations,
                                      // [1] FP64 refinements (MIXED32 outer iterations)
    unsigned int sync_timeout;        // a grid barrier of the cooperative solve ran out
    unsigned int spin_limit;          // polls of a grid-barrier wait before it gives up (0: 2^22)
};

// One contiguous range of FP64 particles of one species in one simulation.
struct SegDev {
    long long start, count;
    int grid, species, blk_first, nblk;
};

// ---------------------------------------------------------------------------------
// Rounded arithmetic of the particle update. The compiler decides per kernel whether a
// product followed by a sum becomes one fused multiply-add, so the same expression can
// round differently in two kernels. A particle is pushed by the tile kernel (shared-
// memory window or global memory) or, when its bin was full, by the overflow kernel; for
// a run to be bit-for-bit reproducible whichever particles overflow, every rounding of
// the push, the shapes and the deposit is written out: xmul/xadd/xsub never fuse, xfma
// is one fused operation.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------------
// Particle shapes: centred B-splines of order P. Given a coordinate split into an
// integer cell i and a fraction f in [0,1) on a lattice whose node k sits at k, return
// the first node `base` and the P+1 weights of nodes base .. base+P.
// ---------------------------------------------------------------------------------
template <int P, typename R>
__device__ __forceinline__ void shape_nodes(int i, R f, int& base, R w[P + 1]) {
    if constexpr (P == 1) {
        base = i;
        w[0] = xsub(R(1), f);
        w[1] = f;
    } else if constexpr (P == 2) {
        // nearest node c = i (f < 1/2) or i+1; d = x - c in [-1/2, 1/2)
        R d;
        if (f < R(0.5)) {
            base = i - 1;
            d = f;
        } else {
            base = i;
            d = xsub(f, R(1));
        }
        const R hm = xsub(R(0.5), d), hp = xadd(R(0.5), d);
        w[0] = xmul(xmul(R(0.5), hm), hm);
        w[1] = xfma(-d, d, R(0.75));
        w[2] = xmul(xmul(R(0.5), hp), hp);
    } else {
        base = i - 1;
        const R g = xsub(R(1), f);
        const R f2 = xmul(f, f), f3 = xmul(f2, f);
        w[0] = xmul(xmul(xmul(g, g), g), R(1.0 / 6.0));
        w[1] = xmul(xfma(R(3), f3, xfma(R(-6), f2, R(4))), R(1.0 / 6.0));
        w[2] = xmul(xfma(R(3), xsub(xadd(f, f2), f3), R(1)), R(1.0 / 6.0));
        w[3] = xmul(f3, R(1.0 / 6.0));
    }
}

// Same, on the lattice shifted by +1/2 (nodes at k + 1/2, stored at index k).
template <int P, typename R>
__device__ __forceinline__ void shape_nodes_half(int i, R f, int& base, R w[P + 1]) {
    R s = xsub(f, R(0.5));
    int c = i;
    if (s < R(0)) {
        s = xadd(s, R(1));
        c -= 1;
        if (s >= R(1)) {  // s was a tiny negative number and s + 1 rounded up to 1
            s = R(0);
            c += 1;
        }
    }
    shape_nodes<P, R>(c, s, base, w);
}

// Column of node i of an x-lattice with conducting walls at x = 0 and x = nx (method of
// images): sign 0 where the node is a wall node of an odd quantity or the unstored wall
// node x = nx, -1 for the image of an odd quantity, +1 otherwise. half: the lattice sits
// at half-integer x (node i at i + 1/2). Fields read with the conductor's parity (odd
// on integer-x lattices); particle deposits fold with the mirror image's (Jx odd, Jy,
// Jz and rho even).
__host__ __device__ __forceinline__ int wall_col(int i, int nx, bool half, bool odd, int& sign) {
    sign = 1;
    if (half) {
        if (i < 0) i = -i - 1;
        else if (i >= nx) i = 2 * nx - i - 1;
        else return i;
    } else {
        if (i < 0) i = -i;
        else if (i > nx) i = 2 * nx - i;
        else if (i > 0 && i < nx) return i;
        if (i == nx || (odd && i == 0)) {
            sign = 0;
            return 0;
        }
    }
    if (odd) sign = -1;
    return i < 0 ? 0 : (i >= nx ? nx - 1 : i);  // (padding nodes of a tile window only)
}

// Specular reflection at the walls of a particle whose move ended in cell `cell` (-1 or
// nx: beyond a wall) at offset `off` in [0, 1): returns the cell in [0, nx), updates the
// offset to the mirrored position and reverses ux.
template <typename R>
__device__ __forceinline__ int reflect_x(int cell, int nx, R& off, R& ux) {
    if (cell >= 0 && cell < nx) return cell;
    ux = -ux;
    R o = xsub(R(1), off);  // the position mirrored about the wall, within the wall cell
    if (cell < 0) {
        if (o >= R(1)) {  // exactly one cell beyond x = 0: lands on node 1
            off = R(0);
            return 1;
        }
        off = o;
        return 0;
    }
    off = o >= R(1) ? R(1) - R(1) / R(16777216) : o;  // exactly on x = nx: stay just inside
    return nx - 1;
}

// Periodic wrap of a lattice index that is at most a few cells out of range.
__device__ __forceinline__ int wrapi(int k, int n) {
    k = (k < 0) ? k + n : k;
    return (k >= n) ? k - n : k;
}

// ---------------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; the result is valid in every thread. `scratch` holds >= 32 T.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T r = (lane < nw) ? scratch[lane] : T(0);
    r = warp_sum(r);
    return r;
}

}  // namespace pic
