// particles_fp64.cu -- the plain FP64 particle half of the step: one thread per particle
// gathers E^n, B^n straight from the FP64 grid arrays, pushes, moves, and deposits
// J^{n+1/2} with FP64 global atomics. No sorting, no shared-memory tiles: this is the
// reference GPU form that the MIXED32 tiled path is measured against.
//
// Positions are kept in grid units (x/dx, y/dy) in [0, nx) x [0, ny).
#include "engine.h"
#include "esirkepov.cuh"
#include "inject.cuh"

namespace pic {
namespace {

// Momentum-conserving gather (Sec. 1, Sec. 3): each component is interpolated with the
// order-P shape on its own staggered lattice, the same weights that assign charge.
template <int P>
__device__ __forceinline__ double gather(const double* __restrict__ A, int nx, const int col[P + 1],
                                         const double wx[P + 1], const int row[P + 1],
                                         const double wy[P + 1]) {
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b <= P; b++) {
        const double* R = A + row[b];
        double ra = 0.0;
#pragma unroll
        for (int a = 0; a <= P; a++) ra += wx[a] * __ldg(R + col[a]);
        acc += wy[b] * ra;
    }
    return acc;
}

template <int P>
__global__ void __launch_bounds__(kPushThreads)
k_push_fp64(const GridDev* __restrict__ grids, const SegDev* __restrict__ segs,
            const int* __restrict__ blk_seg, long long ntot, const double* __restrict__ F,
            double* __restrict__ J, double* __restrict__ xs, double* __restrict__ ys,
            double* __restrict__ uxs, double* __restrict__ uys, double* __restrict__ uzs,
            CgState* cg, DevStatus* st) {
    if (st->stop) return;
    const SegDev S = segs[blk_seg[blockIdx.x]];
    const GridDev& G = grids[S.grid];
    const long long local = (long long)(blockIdx.x - S.blk_first) * blockDim.x + threadIdx.x;
    double ek = 0.0;
    if (local < S.count) {
        const long long k = S.start + local;
        const int nx = G.nx, ny = G.ny;
        const double X = xs[k], Y = ys[k];
        const int i = (int)floor(X), j = (int)floor(Y);
        const double fxp = X - i, fyp = Y - j;
        int bx0, bxh, by0, byh;
        double wx0[P + 1], wxh[P + 1], wy0[P + 1], wyh[P + 1];
        shape_nodes<P, double>(i, fxp, bx0, wx0);
        shape_nodes_half<P, double>(i, fxp, bxh, wxh);
        shape_nodes<P, double>(j, fyp, by0, wy0);
        shape_nodes_half<P, double>(j, fyp, byh, wyh);
        int c0[P + 1], ch[P + 1], r0[P + 1], rh[P + 1];
        double wx0s[P + 1];  // integer-x weights with the conductor's image signs (Ey, Ez, Bx)
#pragma unroll
        for (int a = 0; a <= P; a++) {
            c0[a] = wrapi(bx0 + a, nx);
            ch[a] = wrapi(bxh + a, nx);
            r0[a] = wrapi(by0 + a, ny) * nx;
            rh[a] = wrapi(byh + a, ny) * nx;
            wx0s[a] = wx0[a];
            if (G.walls) {
                int s;
                c0[a] = wall_col(bx0 + a, nx, false, true, s);
                wx0s[a] = wx0[a] * s;
                ch[a] = wall_col(bxh + a, nx, true, false, s);
            }
        }
        const double* base = F + G.cell_off;
        double E[3], B[3];
        if (G.nodal) {  // F holds node averages: the deposit's weights for every component
#pragma unroll
            for (int a = 0; a < 3; a++) {
                E[a] = gather<P>(base + a * ntot, nx, c0, wx0, r0, wy0);
                B[a] = gather<P>(base + (3 + a) * ntot, nx, c0, wx0, r0, wy0);
            }
        } else {
            // Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2)
            E[0] = gather<P>(base, nx, ch, wxh, r0, wy0);
            E[1] = gather<P>(base + ntot, nx, c0, wx0s, rh, wyh);
            E[2] = gather<P>(base + 2 * ntot, nx, c0, wx0s, r0, wy0);
            B[0] = gather<P>(base + 3 * ntot, nx, c0, wx0s, rh, wyh);
            B[1] = gather<P>(base + 4 * ntot, nx, ch, wxh, r0, wy0);
            B[2] = gather<P>(base + 5 * ntot, nx, ch, wxh, rh, wyh);
        }
        double u[3] = {uxs[k], uys[k], uzs[k]};
        const double g_old = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double qm = G.qm[S.species];
        boris<double>(0.5 * qm * G.dt, E, B, u);
        const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double dX = G.dt * u[0] / gam * G.idx;
        const double dY = G.dt * u[1] / gam * G.idy;
        if (!(fabs(dX) < 1.0 && fabs(dY) < 1.0)) {
            if (!isfinite(dX + dY)) atomicAdd(&st->nan_count, 1ull);
            else atomicAdd(&st->cfl_viol, 1ull);
            st->stop_next = 1u;
        } else {
            double X1 = X + dX, Y1 = Y + dY;
            if (G.deposit) {
                const int i1 = (int)floor(X1), j1 = (int)floor(Y1);
                const double area = G.dx * G.dy;
                const double q = G.qw[S.species];
                double* Jb = J + G.cell_off;
                esirkepov<P, double>(i, fxp, j, fyp, i1, X1 - i1, j1, Y1 - j1,
                                     q * G.dx / (G.dt * area), q * G.dy / (G.dt * area),
                                     q * (u[2] / gam) / area,
                                     [&](int comp, int ix, int iy, double v) {
                                         int cx = wrapi(ix, nx), s = 1;
                                         // with walls a reflected particle continues as its
                                         // mirror image: Jx folds odd, Jy and Jz even
                                         if (G.walls) cx = wall_col(ix, nx, comp == 0, comp == 0, s);
                                         if (s != 0)
                                             atomicAdd(Jb + comp * ntot + (long long)wrapi(iy, ny) * nx + cx,
                                                       s * v);
                                     });
            }
            if (G.walls) {  // specular reflection at the walls
                if (X1 < 0.0) {
                    X1 = -X1;
                    u[0] = -u[0];
                } else if (X1 >= nx) {
                    X1 = 2.0 * nx - X1;
                    u[0] = -u[0];
                }
            } else {  // periodic wrap (Sec. 3)
                if (X1 < 0.0) X1 += nx;
                if (X1 >= nx) X1 -= nx;
                if (X1 >= nx) X1 = 0.0;
            }
            if (Y1 < 0.0) Y1 += ny;
            if (Y1 >= ny) Y1 -= ny;
            if (Y1 >= ny) Y1 = 0.0;
            xs[k] = X1;
            ys[k] = Y1;
        }
        uxs[k] = u[0];
        uys[k] = u[1];
        uzs[k] = u[2];
        ek = G.w * (0.5 * (g_old + gam) - 1.0);
    }
    __shared__ double scratch[32];
    const double s = block_sum(ek, scratch);
    if (threadIdx.x == 0 && s != 0.0) atomicAdd(&cg[S.grid].uk, s);
}

// The injector's pairs of this step appended to the species arrays (one thread per
// row and pair); their slots come from the segment counts, so the order is arbitrary.
__global__ void k_inject_fp64(const Fp64InjectArgs a) {
    const DevStatus* st = a.st;
    if (st->stop) return;
    const GridDev& G = a.grids[0];
    const long long n = (long long)st->steps_done - 1;
    const long long per_row = inj_count(G, n);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = (int)(t / a.kmax);
    const long long k = t - (long long)j * a.kmax;
    if (j >= G.ny || k >= per_row) return;
    double x, y;
    inj_position(G, n, j, k, x, y);
    for (int s = 0; s < 2; s++) {
        double u[3];
        inj_momentum(G, n, j, k, s, u);
        const unsigned long long idx =
            atomicAdd(reinterpret_cast<unsigned long long*>(&a.segs[s].count), 1ull);
        if ((long long)idx >= a.cap[s]) {
            atomicAdd(&a.st->lost, 1ull);  // arrays full: the step fails with PIC_ENOMEM
            a.st->stop_next = 1u;
            continue;
        }
        a.x[s][idx] = x;
        a.y[s][idx] = y;
        a.ux[s][idx] = u[0];
        a.uy[s][idx] = u[1];
        a.uz[s][idx] = u[2];
    }
}

template <int P>
__global__ void k_rho_fp64(GridDev G, const double* __restrict__ x, const double* __restrict__ y, long long n,
                           double q, double* rho) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)floor(x[k]), j = (int)floor(y[k]);
    deposit_rho<P>(G, i, x[k] - i, j, y[k] - j, q, rho);
}

__global__ void k_momentum_fp64(const double* __restrict__ ux, const double* __restrict__ uy,
                                const double* __restrict__ uz, long long n, double w, double* out) {
    __shared__ double red[32];
    double s[3] = {0.0, 0.0, 0.0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        s[0] += ux[k];
        s[1] += uy[k];
        s[2] += uz[k];
    }
    for (int c = 0; c < 3; c++) {
        const double t = block_sum(s[c], red);
        if (threadIdx.x == 0) atomicAdd(out + c, w * t);
        __syncthreads();
    }
}

}  // namespace

void launch_rho_fp64(const GridDev& G, const double* x, const double* y, long long n, double q, double* rho,
                     cudaStream_t s) {
    if (n <= 0) return;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (G.order) {
    case 1: k_rho_fp64<1><<<nb, 256, 0, s>>>(G, x, y, n, q, rho); break;
    case 2: k_rho_fp64<2><<<nb, 256, 0, s>>>(G, x, y, n, q, rho); break;
    default: k_rho_fp64<3><<<nb, 256, 0, s>>>(G, x, y, n, q, rho); break;
    }
}

void launch_momentum_fp64(const double* ux, const double* uy, const double* uz, long long n, double w, double* out,
                          cudaStream_t s) {
    if (n <= 0) return;
    k_momentum_fp64<<<304, 256, 0, s>>>(ux, uy, uz, n, w, out);
}

void launch_inject_fp64(const Fp64InjectArgs& a, cudaStream_t s) {
    const long long threads = (long long)a.ny * a.kmax;
    k_inject_fp64<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
}

void launch_push_fp64(const Fp64PushArgs& a, int order, cudaStream_t s) {
    if (a.nblk == 0) return;
#define PIC_PUSH_ARGS                                                                      \
    a.grids, a.segs, a.blk_seg, a.ntot, a.F, a.J, a.x, a.y, a.ux, a.uy, a.uz, a.cg, a.st
    switch (order) {
    case 1: k_push_fp64<1><<<a.nblk, kPushThreads, 0, s>>>(PIC_PUSH_ARGS); break;
    case 2: k_push_fp64<2><<<a.nblk, kPushThreads, 0, s>>>(PIC_PUSH_ARGS); break;
    default: k_push_fp64<3><<<a.nblk, kPushThreads, 0, s>>>(PIC_PUSH_ARGS); break;
    }
#undef PIC_PUSH_ARGS
}

}  // namespace pic
