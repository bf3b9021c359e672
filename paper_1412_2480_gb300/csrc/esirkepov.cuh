// esirkepov.cuh -- the particle kernels' shared device arithmetic: momentum-conserving
// gather weights, the relativistic Boris push and the density-decomposition deposit.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// 1/sqrt(x) and 1/x inside the push. FP32: the hardware approximations (MUFU; a few ulp,
// far below the FP32 parity tolerance, and one fixed instruction, so every kernel that
// pushes a particle still gives the same bits) instead of the correctly rounded sequences,
// which cost ten or more instructions each. FP64: the correctly rounded operations.
__device__ __forceinline__ float rsqrt_push(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_push(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rcp_push(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_push(double x) { return 1.0 / x; }

// Relativistic Buneman-Boris push (standard scheme; the paper specifies none), c = 1:
// half electric kick, rotation by t = h B / gamma(u-), s = 2t / (1 + t^2), half kick.
// h = (q/m) dt / 2.
// Every rounding is explicit (xmul, xfma, ...; pic_internal.cuh), so each kernel that
// runs it gives the same bits.
template <typename R>
__device__ __forceinline__ void boris(R h, const R E[3], const R B[3], R u[3]) {
    R um0 = xfma(h, E[0], u[0]), um1 = xfma(h, E[1], u[1]), um2 = xfma(h, E[2], u[2]);
    const R ig = rsqrt_push(xfma(um2, um2, xfma(um1, um1, xfma(um0, um0, R(1)))));
    const R t0 = xmul(xmul(h, B[0]), ig), t1 = xmul(xmul(h, B[1]), ig), t2 = xmul(xmul(h, B[2]), ig);
    const R f = xmul(R(2), rcp_push(xfma(t2, t2, xfma(t1, t1, xfma(t0, t0, R(1))))));
    const R s0 = xmul(f, t0), s1 = xmul(f, t1), s2 = xmul(f, t2);
    const R p0 = xadd(um0, xfma(um1, t2, -xmul(um2, t1)));
    const R p1 = xadd(um1, xfma(um2, t0, -xmul(um0, t2)));
    const R p2 = xadd(um2, xfma(um0, t1, -xmul(um1, t0)));
    um0 = xadd(um0, xfma(p1, s2, -xmul(p2, s1)));
    um1 = xadd(um1, xfma(p2, s0, -xmul(p0, s2)));
    um2 = xadd(um2, xfma(p0, s1, -xmul(p1, s0)));
    u[0] = xfma(h, E[0], um0);
    u[1] = xfma(h, E[1], um1);
    u[2] = xfma(h, E[2], um2);
}

// Weight of node k (0..P+1, a compile-time constant once unrolled) of a (P+2)-wide
// window, for a particle whose P+1 weights start `sh` nodes into the window. For every
// move below one cell the shape bases before and after differ by at most one node, so
// sh is 0 or 1 and each window node is a single select.
template <int P, typename R>
__device__ __forceinline__ R window_weight(const R w[P + 1], bool sh, int k) {
    const R at0 = k <= P ? w[k <= P ? k : 0] : R(0);     // sh = 0
    const R at1 = k >= 1 ? w[k >= 1 ? k - 1 : 0] : R(0);  // sh = 1
    return sh ? at1 : at0;
}

// Density-decomposition (Esirkepov) current of one particle moving from cell/fraction
// (i0+f0x, j0+f0y) to (i1+f1x, j1+f1y), less than one cell in each direction. On the
// common (P+2)^2 window of node weights S0 (old) and S1 (new), DS = S1 - S0:
//   Wx = DSx (S0y + DSy/2),  Wy = DSy (S0x + DSx/2),
//   Wz = S0x S0y + (DSx S0y + S0x DSy)/2 + DSx DSy/3,
//   Jx(i+1/2) = Jx(i-1/2) - fx Wx, Jy(j+1/2) = Jy(j-1/2) - fy Wy, Jz += fz Wz,
// with fx = q dx/(dt dx dy), fy = q dy/(dt dx dy), fz = q vz/(dx dy). The Jx running sum
// over the last window column is zero (charge conservation), so only P+1 columns of Jx
// (and P+1 rows of Jy) are written. `add(comp, ix, iy, value)` receives window-origin
// node indices (unwrapped).
//
// When the old and new shapes start on the same row (the move does not shift the y
// base), the window's last row has S0y = S1y = 0: every Wx and Wz there is zero, and the
// Jy running sum is complete one row earlier (its row-P value is zero up to rounding and
// is not written). A warp whose particles all keep their y base (transverse moves far
// below a cell, as in a relativistic beam) then writes the P+1 rows only: 30% fewer
// shared-memory updates. In the full window each such lane skips its last-row updates
// (exact zeros) and the same Jy value, so a particle's currents do not depend on the path
// its warp takes, and results stay independent of how particles are grouped into warps.
// (Skipping the exact-zero last column of a lane that keeps its x base measured slower:
// the extra predicates cost more than the updates they save.)
template <int P, int WY, typename R, typename Add>
__device__ __forceinline__ void esirkepov_window(int ox, int oy, const R S0x[P + 2], const R DSx[P + 2],
                                                 const R S0y[P + 2], const R DSy[P + 2], R fx, R fy, R fz,
                                                 bool ysame, Add add) {
    // row b of the window is an exact zero for this lane
    const auto row0 = [&](int b) { return WY == P + 2 && b == P + 1 && ysame; };
#pragma unroll
    for (int b = 0; b < WY; b++) {
        const R ry = xmul(fx, xfma(R(0.5), DSy[b], S0y[b]));
        R run = R(0);
#pragma unroll
        for (int a = 0; a <= P; a++) {
            run = xfma(-DSx[a], ry, run);
            if (!row0(b)) add(0, ox + a, oy + b, run);
        }
    }
#pragma unroll
    for (int a = 0; a < P + 2; a++) {
        const R rx = xmul(fy, xfma(R(0.5), DSx[a], S0x[a]));
        R run = R(0);
#pragma unroll
        for (int b = 0; b < WY - 1; b++) {
            run = xfma(-DSy[b], rx, run);
            if (b < P || !ysame) add(1, ox + a, oy + b, run);
        }
    }
#pragma unroll
    for (int b = 0; b < WY; b++) {
        const R cy0 = xmul(fz, xfma(R(0.5), DSy[b], S0y[b]));
        const R cy1 = xmul(fz, xfma(R(1.0 / 3.0), DSy[b], xmul(R(0.5), S0y[b])));
#pragma unroll
        for (int a = 0; a < P + 2; a++)
            if (!row0(b)) add(2, ox + a, oy + b, xfma(S0x[a], cy0, xmul(DSx[a], cy1)));
    }
}

template <int P, typename R, typename Add>
__device__ __forceinline__ void esirkepov(int i0, R f0x, int j0, R f0y, int i1, R f1x, int j1,
                                          R f1y, R fx, R fy, R fz, Add add) {
    int b0x, b1x, b0y, b1y;
    R s0x[P + 1], s1x[P + 1], s0y[P + 1], s1y[P + 1];
    shape_nodes<P, R>(i0, f0x, b0x, s0x);
    shape_nodes<P, R>(i1, f1x, b1x, s1x);
    shape_nodes<P, R>(j0, f0y, b0y, s0y);
    shape_nodes<P, R>(j1, f1y, b1y, s1y);
    const int ox = min(b0x, b1x), oy = min(b0y, b1y);
    const bool h0x = b0x != ox, h1x = b1x != ox, h0y = b0y != oy, h1y = b1y != oy;
    R S0x[P + 2], DSx[P + 2], S0y[P + 2], DSy[P + 2];
#pragma unroll
    for (int k = 0; k < P + 2; k++) {
        S0x[k] = window_weight<P, R>(s0x, h0x, k);
        DSx[k] = xsub(window_weight<P, R>(s1x, h1x, k), S0x[k]);
        S0y[k] = window_weight<P, R>(s0y, h0y, k);
        DSy[k] = xsub(window_weight<P, R>(s1y, h1y, k), S0y[k]);
    }
    const bool ysame = b0y == b1y;
    if (__all_sync(__activemask(), ysame))  // (only lanes with ysame take the short path)
        esirkepov_window<P, P + 1>(ox, oy, S0x, DSx, S0y, DSy, fx, fy, fz, true, add);
    else
        esirkepov_window<P, P + 2>(ox, oy, S0x, DSx, S0y, DSy, fx, fy, fz, ysame, add);
}

// Node charge density of one macro-particle of charge density q (charge / (dx dy)) at
// cell/fraction (i + fx, j + fy): rho(node) += q W_p(x - node) W_p(y - node) on the
// integer lattice. With walls the part beyond a wall folds back as the mirror image's
// (even); the unstored wall node x = nx is dropped.
template <int P>
__device__ __forceinline__ void deposit_rho(const GridDev& G, int i, double fx, int j, double fy, double q,
                                            double* rho) {
    int bx, by;
    double wx[P + 1], wy[P + 1];
    shape_nodes<P, double>(i, fx, bx, wx);
    shape_nodes<P, double>(j, fy, by, wy);
#pragma unroll
    for (int b = 0; b <= P; b++) {
        double* row = rho + (long long)wrapi(by + b, G.ny) * G.nx;
#pragma unroll
        for (int a = 0; a <= P; a++) {
            int s = 1, col = wrapi(bx + a, G.nx);
            if (G.walls) col = wall_col(bx + a, G.nx, false, false, s);
            if (s) atomicAdd(row + col, s * q * wx[a] * wy[b]);
        }
    }
}

}  // namespace pic
