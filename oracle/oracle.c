/*
 * oracle.c -- plain, slow, FP64 CPU reference of the per-step particle cycle of the
 * 2D implicit-FDTD PIC method of Ikeya & Matsumoto (PASJ 2015, arXiv:1412.2480).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library; the CUDA product never does.
 * Nothing here is blocked, fused or reordered beyond what the paper's equations
 * state: every loop follows the definition it cites. Single-threaded, so results are
 * deterministic.
 *
 * Layout and units: see oracle.h.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* Staggered offsets (in cells) of the field components Ex, Ey, Ez, Bx, By, Bz on the
 * 2D Yee grid (Sec. 2, Fig. 1; standard arrangement since the figure is empty). */
static const double OFF_X[6] = {0.5, 0.0, 0.0, 0.0, 0.5, 0.5};
static const double OFF_Y[6] = {0.0, 0.5, 0.0, 0.5, 0.0, 0.5};

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t at(const or_grid* g, int i, int j) {
    return (int64_t)wrap(j, g->ny) * g->nx + wrap(i, g->nx);
}

/* Stored index of node (i, j) of a lattice that sits at integer x (half = 0) or at
 * half-integer x (half = 1; node i at x = i + 1/2), for a quantity that is odd (odd = 1)
 * or even under reflection at the walls x = 0 and x = nx, with the image sign in *sign;
 * -1 where the value is zero by symmetry (an odd quantity on a wall node) or is not
 * stored (the wall node x = nx). Periodic in x without walls. */
static int64_t node(const or_grid* g, int half, int odd, int i, int j, double* sign) {
    *sign = 1.0;
    if (!g->walls) return at(g, i, j);
    const int nx = g->nx;
    if (half) {
        if (i < 0) i = -i - 1;
        else if (i >= nx) i = 2 * nx - i - 1;
        else return (int64_t)wrap(j, g->ny) * nx + i;
    } else {
        if (i < 0) i = -i;
        else if (i > nx) i = 2 * nx - i;
        else if (i > 0 && i < nx) return (int64_t)wrap(j, g->ny) * nx + i;
        if (i == nx || (odd && i == 0)) return -1;
    }
    if (odd) *sign = -1.0;
    return (int64_t)wrap(j, g->ny) * nx + i;
}

/* Value of a field-like quantity at node (i, j), images of a perfect conductor
 * included: odd on integer-x lattices (Ey, Ez, Bx, and Jy, Jz as the solver sees them:
 * the conductor carries the wall nodes' current), even on half-integer ones. */
static double val(const or_grid* g, const double* v, int half, int i, int j) {
    double s;
    const int64_t k = node(g, half, !half, i, j, &s);
    return k < 0 ? 0.0 : s * v[k];
}

/* Add a particle's contribution to node (i, j), folded onto the stored node. A particle
 * reflected at a wall continues as its mirror image (same charge, ux reversed): rho,
 * Jy, Jz fold even and Jx odd (odd = 1). */
static void add_at(const or_grid* g, double* v, int half, int odd, int i, int j, double c) {
    double s;
    const int64_t k = node(g, half, odd, i, j, &s);
    if (k >= 0) v[k] += s * c;
}

/* Centred B-spline shapes W_p (Sec. 3: first- and second-order shape functions; the
 * third order extends the same family). W_p is the (p+1)-fold convolution of the
 * unit box, written out piecewise. */
double or_shape(int32_t p, double d) {
    double a = fabs(d);
    switch (p) {
    case 1:
        return a < 1.0 ? 1.0 - a : 0.0;
    case 2:
        if (a < 0.5) return 0.75 - a * a;
        if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    case 3:
        if (a < 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
        if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    default:
        return NAN;
    }
}

/* Momentum-conserving interpolation (Sec. 1 and Sec. 3, citing Birdsall & Langdon):
 * the force on a particle is interpolated with the same shape W_p that assigns its
 * charge. Each component is gathered on its own staggered lattice:
 *   F(x,y) = sum_{i,j} W_p(x/dx - i - ox) W_p(y/dy - j - oy) F_{ij}.
 * The sum runs over a window wider than any support (|d| < 2); zero weights drop out. */
/* The alternative reading (nodal = 1): every component is first averaged from its
 * staggered lattice to the node (i, j) -- over the two neighbours along each staggered
 * direction: Ex, By along x; Ey, Bx along y; Bz over the four surrounding cells; Ez is a
 * node quantity -- and then gathered with the node weights of the charge deposit. */
static double node_average(const or_grid* g, const double* V, int c, int i, int j) {
    switch (c) {
    case 0: case 4: return 0.5 * (val(g, V, 1, i - 1, j) + val(g, V, 1, i, j));
    case 1: case 3: return 0.5 * (val(g, V, 0, i, j - 1) + val(g, V, 0, i, j));
    case 2: return val(g, V, 0, i, j);
    default:
        return 0.25 * (val(g, V, 1, i - 1, j - 1) + val(g, V, 1, i, j - 1) + val(g, V, 1, i - 1, j) +
                       val(g, V, 1, i, j));
    }
}

static void gather_one(const or_grid* g, const double* F, double x, double y, double f[6]) {
    const int64_t N = (int64_t)g->nx * g->ny;
    const double xg = x / g->dx, yg = y / g->dy;
    if (g->nodal) {
        const int i0 = (int)floor(xg) - 2, j0 = (int)floor(yg) - 2;
        for (int c = 0; c < 6; c++) {
            double acc = 0.0;
            for (int j = j0; j <= j0 + 5; j++) {
                const double wy = or_shape(g->order, yg - j);
                if (wy == 0.0) continue;
                for (int i = i0; i <= i0 + 5; i++) {
                    const double wx = or_shape(g->order, xg - i);
                    if (wx == 0.0) continue;
                    acc += wx * wy * node_average(g, F + c * N, c, i, j);
                }
            }
            f[c] = acc;
        }
        return;
    }
    for (int c = 0; c < 6; c++) {
        const double sx = xg - OFF_X[c], sy = yg - OFF_Y[c];
        const int i0 = (int)floor(sx) - 2, j0 = (int)floor(sy) - 2;
        double acc = 0.0;
        for (int j = j0; j <= j0 + 5; j++) {
            const double wy = or_shape(g->order, sy - j);
            if (wy == 0.0) continue;
            for (int i = i0; i <= i0 + 5; i++) {
                const double wx = or_shape(g->order, sx - i);
                if (wx == 0.0) continue;
                acc += wx * wy * val(g, F + c * N, OFF_X[c] != 0.0, i, j);
            }
        }
        f[c] = acc;
    }
}

void or_gather(const or_grid* g, const double* F, int64_t n, const double* x,
               const double* y, double* out) {
    for (int64_t k = 0; k < n; k++) {
        double f[6];
        gather_one(g, F, x[k], y[k], f);
        for (int c = 0; c < 6; c++) out[c * n + k] = f[c];
    }
}

/* Relativistic Buneman-Boris push (the paper gives no pusher; this is the standard
 * one). du/dt = (q/m)(E + v x B / c) with u = gamma v, c = 1, E and B at time n:
 *   u-  = u^{n-1/2} + (q dt / 2m) E
 *   t   = (q dt / 2m) B / gamma(u-),   s = 2 t / (1 + |t|^2)
 *   u'  = u- + u- x t,                 u+ = u- + u' x s
 *   u^{n+1/2} = u+ + (q dt / 2m) E. */
static void boris_one(double qm, double dt, const double E[3], const double B[3], double u[3]) {
    const double h = 0.5 * qm * dt;
    double um[3], t[3], s[3], up[3], upl[3];
    for (int a = 0; a < 3; a++) um[a] = u[a] + h * E[a];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; a++) t[a] = h * B[a] / gm;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; a++) s[a] = 2.0 * t[a] / (1.0 + t2);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    upl[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    upl[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    upl[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int a = 0; a < 3; a++) u[a] = upl[a] + h * E[a];
}

void or_boris(double qm, double dt, int64_t n, const double* E, const double* B, double* u) {
    for (int64_t k = 0; k < n; k++) boris_one(qm, dt, E + 3 * k, B + 3 * k, u + 3 * k);
}

/* Density-decomposition current deposit (Sec. 1 and Sec. 3, citing Esirkepov 2001).
 * With node weights S0 = W_p(x0 - i) and S1 = W_p(x1 - i) on a common window and
 * DS = S1 - S0 (x and y alike), the 2D decomposition of the change of the particle's
 * node charge is
 *   Wx = DSx (S0y + DSy/2)
 *   Wy = DSy (S0x + DSx/2)
 *   Wz = S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3
 * and the currents follow from the discrete continuity equation:
 *   Jx(i+1/2, j) = Jx(i-1/2, j) - q (dx/dt) Wx(i,j) / (dx dy)   (from the window's low edge)
 *   Jy(i, j+1/2) = Jy(i, j-1/2) - q (dy/dt) Wy(i,j) / (dx dy)
 *   Jz(i, j)    += q vz Wz(i,j) / (dx dy).
 * For |x1-x0| < dx the nonzero nodes lie in [floor(min x) - 1, floor(min x) + 3] (order
 * <= 3); the 7-node window starting at floor(min x) - 2 covers them with zeros on both
 * ends, so the running sums start and end at zero. */
void or_deposit_move(const or_grid* g, double qw, double x0, double y0, double x1,
                     double y1, double vz, double* J) {
    enum { W = 7 };
    const int64_t N = (int64_t)g->nx * g->ny;
    double* Jx = J;
    double* Jy = J + N;
    double* Jz = J + 2 * N;
    const double x0g = x0 / g->dx, x1g = x1 / g->dx, y0g = y0 / g->dy, y1g = y1 / g->dy;
    const int i0 = (int)floor(fmin(x0g, x1g)) - 2;
    const int j0 = (int)floor(fmin(y0g, y1g)) - 2;
    double S0x[W], DSx[W], S0y[W], DSy[W];
    for (int a = 0; a < W; a++) {
        S0x[a] = or_shape(g->order, x0g - (i0 + a));
        DSx[a] = or_shape(g->order, x1g - (i0 + a)) - S0x[a];
        S0y[a] = or_shape(g->order, y0g - (j0 + a));
        DSy[a] = or_shape(g->order, y1g - (j0 + a)) - S0y[a];
    }
    const double area = g->dx * g->dy;
    const double fx = qw * g->dx / (g->dt * area);
    const double fy = qw * g->dy / (g->dt * area);
    const double fz = qw * vz / area;
    for (int b = 0; b < W; b++) {
        double acc = 0.0;
        for (int a = 0; a < W; a++) {
            const double Wx = DSx[a] * (S0y[b] + 0.5 * DSy[b]);
            acc -= fx * Wx;
            add_at(g, Jx, 1, 1, i0 + a, j0 + b, acc);
        }
    }
    for (int a = 0; a < W; a++) {
        double acc = 0.0;
        for (int b = 0; b < W; b++) {
            const double Wy = DSy[b] * (S0x[a] + 0.5 * DSx[a]);
            acc -= fy * Wy;
            add_at(g, Jy, 0, 0, i0 + a, j0 + b, acc);
        }
    }
    for (int b = 0; b < W; b++) {
        for (int a = 0; a < W; a++) {
            const double Wz = S0x[a] * S0y[b] + 0.5 * DSx[a] * S0y[b] + 0.5 * S0x[a] * DSy[b] +
                              DSx[a] * DSy[b] / 3.0;
            add_at(g, Jz, 0, 0, i0 + a, j0 + b, fz * Wz);
        }
    }
}

/* Periodic wrap of a grid coordinate that moved by less than one cell (Sec. 3:
 * periodic in x and y). */
static double wrap_coord(double s, int n) {
    if (s < 0.0) s += n;
    if (s >= n) s -= n;
    if (s >= n) s = 0.0; /* s was a tiny negative number that rounded up to n */
    return s;
}

/* The particle half of one step n -> n+1 for one species: gather E^n, B^n at x^n,
 * push u^{n-1/2} -> u^{n+1/2}, move x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2},
 * deposit J^{n+1/2} from the unwrapped move, then wrap into the periodic box, or, with
 * walls, reflect a particle that crossed one: x -> -x (or 2 nx dx - x) and ux -> -ux.
 * Its deposit is that of the unreflected move folded back at the wall: the particle
 * and its mirror image, which carries on after the reflection. */
int64_t or_push_deposit(const or_grid* g, const double* F, double qm, double qw, int64_t n,
                        double* x, double* y, double* ux, double* uy, double* uz,
                        double* J, int32_t deposit) {
    int64_t bad = 0;
    for (int64_t k = 0; k < n; k++) {
        double f[6];
        gather_one(g, F, x[k], y[k], f);
        double u[3] = {ux[k], uy[k], uz[k]};
        boris_one(qm, g->dt, f, f + 3, u);
        const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double x0g = x[k] / g->dx, y0g = y[k] / g->dy;
        const double x1g = x0g + g->dt * u[0] / (gam * g->dx);
        const double y1g = y0g + g->dt * u[1] / (gam * g->dy);
        if (!(fabs(x1g - x0g) < 1.0 && fabs(y1g - y0g) < 1.0)) bad++;
        if (deposit)
            or_deposit_move(g, qw, x[k], y[k], x1g * g->dx, y1g * g->dy, u[2] / gam, J);
        double xn = x1g;
        if (g->walls && xn < 0.0) {
            xn = -xn;
            u[0] = -u[0];
        } else if (g->walls && xn >= g->nx) {
            xn = 2.0 * g->nx - xn;
            u[0] = -u[0];
        }
        x[k] = (g->walls ? xn : wrap_coord(xn, g->nx)) * g->dx;
        y[k] = wrap_coord(y1g, g->ny) * g->dy;
        ux[k] = u[0];
        uy[k] = u[1];
        uz[k] = u[2];
    }
    return bad;
}

void or_deposit_rho(const or_grid* g, double qw, int64_t n, const double* x,
                    const double* y, double* rho) {
    const double area = g->dx * g->dy;
    for (int64_t k = 0; k < n; k++) {
        const double xg = x[k] / g->dx, yg = y[k] / g->dy;
        const int i0 = (int)floor(xg) - 2, j0 = (int)floor(yg) - 2;
        for (int j = j0; j <= j0 + 5; j++)
            for (int i = i0; i <= i0 + 5; i++)
                add_at(g, rho, 0, 0, i, j, qw * or_shape(g->order, xg - i) * or_shape(g->order, yg - j) / area);
    }
}

/* ---- Yee-grid difference operators (Sec. 2; each a one-cell centred difference) ---- */

/* curl of an E-lattice vector (Ex,Ey,Ez layout), evaluated on the B lattices. */
static void curl_E_lattice(const or_grid* g, const double* V, double* out) {
    const int nx = g->nx, ny = g->ny;
    const int64_t N = (int64_t)nx * ny;
    const double *Vx = V, *Vy = V + N, *Vz = V + 2 * N;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t k = at(g, i, j);
            /* x at (i, j+1/2):      d/dy Vz      (Vz, Vy on integer-x lattices) */
            out[k] = (val(g, Vz, 0, i, j + 1) - val(g, Vz, 0, i, j)) / g->dy;
            /* y at (i+1/2, j):     -d/dx Vz */
            out[N + k] = -(val(g, Vz, 0, i + 1, j) - val(g, Vz, 0, i, j)) / g->dx;
            /* z at (i+1/2, j+1/2):  d/dx Vy - d/dy Vx */
            out[2 * N + k] = (val(g, Vy, 0, i + 1, j) - val(g, Vy, 0, i, j)) / g->dx -
                             (val(g, Vx, 1, i, j + 1) - val(g, Vx, 1, i, j)) / g->dy;
        }
}

/* curl of a B-lattice vector (Bx,By,Bz layout), evaluated on the E lattices. */
static void curl_B_lattice(const or_grid* g, const double* V, double* out) {
    const int nx = g->nx, ny = g->ny;
    const int64_t N = (int64_t)nx * ny;
    const double *Vx = V, *Vy = V + N, *Vz = V + 2 * N;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t k = at(g, i, j);
            /* x at (i+1/2, j):      d/dy Vz      (Vz, Vy on half-integer-x lattices) */
            out[k] = (val(g, Vz, 1, i, j) - val(g, Vz, 1, i, j - 1)) / g->dy;
            /* y at (i, j+1/2):     -d/dx Vz */
            out[N + k] = -(val(g, Vz, 1, i, j) - val(g, Vz, 1, i - 1, j)) / g->dx;
            /* z at (i, j):          d/dx Vy - d/dy Vx */
            out[2 * N + k] = (val(g, Vy, 1, i, j) - val(g, Vy, 1, i - 1, j)) / g->dx -
                             (val(g, Vx, 0, i, j) - val(g, Vx, 0, i, j - 1)) / g->dy;
            if (g->walls && i == 0) out[N + k] = out[2 * N + k] = 0.0; /* Ey, Ez on the wall */
        }
}

/* Five-point Laplacian of each of the 3 components of V, on its own lattice. */
static void laplacian3(const or_grid* g, const double* V, double* out) {
    const int nx = g->nx, ny = g->ny;
    const int64_t N = (int64_t)nx * ny;
    for (int c = 0; c < 3; c++) {
        const double* v = V + c * N;
        const int half = c > 0; /* Bx on an integer-x lattice, By and Bz on half-integer ones */
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int64_t k = at(g, i, j);
                const double vc = val(g, v, half, i, j);
                out[c * N + k] = (val(g, v, half, i + 1, j) - 2.0 * vc + val(g, v, half, i - 1, j)) /
                                     (g->dx * g->dx) +
                                 (val(g, v, half, i, j + 1) - 2.0 * vc + val(g, v, half, i, j - 1)) /
                                     (g->dy * g->dy);
            }
    }
}

/* Eq. (7), right-hand side: theta (c dt)^2 (Lap B^n + (4 pi / c) curl J^{n+1/2})
 *                           - c dt curl E^n, with c = 1. */
void or_rhs(const or_grid* g, const double* F, const double* J, double* b) {
    const int64_t N = (int64_t)g->nx * g->ny;
    double* lapB = malloc(3 * N * sizeof(double));
    double* curlJ = malloc(3 * N * sizeof(double));
    double* curlE = malloc(3 * N * sizeof(double));
    laplacian3(g, F + 3 * N, lapB);
    curl_E_lattice(g, J, curlJ); /* J lives on the E lattices */
    curl_E_lattice(g, F, curlE);
    const double dt = g->dt, th = g->theta;
    for (int64_t k = 0; k < 3 * N; k++)
        b[k] = th * dt * dt * (lapB[k] + 4.0 * PI * curlJ[k]) - dt * curlE[k];
    free(lapB);
    free(curlJ);
    free(curlE);
}

/* Eq. (7), left-hand operator: [1 - (theta c dt)^2 Lap] x. */
void or_apply_A(const or_grid* g, const double* x, double* Ax) {
    const int64_t N = (int64_t)g->nx * g->ny;
    laplacian3(g, x, Ax);
    const double a = (g->theta * g->dt) * (g->theta * g->dt);
    for (int64_t k = 0; k < 3 * N; k++) Ax[k] = x[k] - a * Ax[k];
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t k = 0; k < n; k++) s += a[k] * b[k];
    return s;
}

/* Conjugate-gradient solve of Eq. (7) after discretising in space with periodic
 * boundaries (Sec. 2, citing Hoshino 2013). The paper names no preconditioner; the
 * Jacobi (diagonal) one is used: the diagonal of A is the constant
 * 1 + 2 (theta dt)^2 (1/dx^2 + 1/dy^2). Textbook PCG: r = b - Ax, z = r/d, p = z;
 * alpha = (r.z)/(p.Ap); x += alpha p; r -= alpha Ap; beta = (r.z)_new/(r.z); p = z + beta p. */
int32_t or_pcg(const or_grid* g, const double* b, double* x, double rtol, int32_t maxit,
               double* rel_resid) {
    const int64_t n = 3 * (int64_t)g->nx * g->ny;
    const double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, n * sizeof(double));
        *rel_resid = 0.0;
        return 0;
    }
    const double a = (g->theta * g->dt) * (g->theta * g->dt);
    const double d = 1.0 + 2.0 * a * (1.0 / (g->dx * g->dx) + 1.0 / (g->dy * g->dy));
    double* r = malloc(n * sizeof(double));
    double* z = malloc(n * sizeof(double));
    double* p = malloc(n * sizeof(double));
    double* q = malloc(n * sizeof(double));
    or_apply_A(g, x, q);
    for (int64_t k = 0; k < n; k++) r[k] = b[k] - q[k];
    double rnorm = sqrt(dot(n, r, r));
    int32_t it = 0, result = -1;
    if (rnorm <= rtol * bnorm) {
        result = 0;
    } else {
        for (int64_t k = 0; k < n; k++) z[k] = r[k] / d;
        memcpy(p, z, n * sizeof(double));
        double rz = dot(n, r, z);
        for (it = 1; it <= maxit; it++) {
            or_apply_A(g, p, q);
            const double alpha = rz / dot(n, p, q);
            for (int64_t k = 0; k < n; k++) {
                x[k] += alpha * p[k];
                r[k] -= alpha * q[k];
            }
            rnorm = sqrt(dot(n, r, r));
            if (rnorm <= rtol * bnorm) {
                result = it;
                break;
            }
            for (int64_t k = 0; k < n; k++) z[k] = r[k] / d;
            const double rz_new = dot(n, r, z);
            const double beta = rz_new / rz;
            rz = rz_new;
            for (int64_t k = 0; k < n; k++) p[k] = z[k] + beta * p[k];
        }
    }
    *rel_resid = rnorm / bnorm;
    free(r);
    free(z);
    free(p);
    free(q);
    return result;
}

/* Eqs. (5)-(6) with B^{n+1} = B^n + dB: Ampere's law (6) gives
 *   E^{n+1} = E^n + c dt curl(theta B^{n+1} + (1-theta) B^n) - 4 pi dt J^{n+1/2}
 *           = E^n + c dt curl(B^n + theta dB) - 4 pi dt J^{n+1/2},
 * and then B^{n+1} = B^n + dB (the definition of dB above Eq. (7)). */
void or_field_update(const or_grid* g, double* F, const double* dB, const double* J) {
    const int64_t N = (int64_t)g->nx * g->ny;
    double* Bh = malloc(3 * N * sizeof(double));
    double* curlBh = malloc(3 * N * sizeof(double));
    for (int64_t k = 0; k < 3 * N; k++) Bh[k] = F[3 * N + k] + g->theta * dB[k];
    curl_B_lattice(g, Bh, curlBh);
    for (int64_t k = 0; k < 3 * N; k++) F[k] += g->dt * (curlBh[k] - 4.0 * PI * J[k]);
    for (int64_t k = 0; k < 3 * N; k++) F[3 * N + k] += dB[k];
    if (g->walls) /* the conductor keeps Ey = Ez = 0 on the wall: it carries that current */
        for (int j = 0; j < g->ny; j++) F[N + at(g, 0, j)] = F[2 * N + at(g, 0, j)] = 0.0;
    free(Bh);
    free(curlBh);
}

/* Explicit FDTD (Eqs. 3-4). Eq. (3) advances B between half-integer time levels; the
 * particle push needs B at integer levels, so each step splits Eq. (3) into two halves
 * around Eq. (4): B^{n+1/2} - B^{n-1/2} = -c dt curl E^n still holds step to step. */
void or_explicit_update(const or_grid* g, double* F, const double* J) {
    const int64_t N = (int64_t)g->nx * g->ny;
    double* curl = malloc(3 * N * sizeof(double));
    curl_E_lattice(g, F, curl); /* curl E^n on the B lattices */
    for (int64_t k = 0; k < 3 * N; k++) F[3 * N + k] -= 0.5 * g->dt * curl[k];
    curl_B_lattice(g, F + 3 * N, curl); /* curl B^{n+1/2} on the E lattices */
    for (int64_t k = 0; k < 3 * N; k++) F[k] += g->dt * (curl[k] - 4.0 * PI * J[k]);
    if (g->walls) /* the conductor keeps Ey = Ez = 0 on the wall */
        for (int j = 0; j < g->ny; j++) F[N + at(g, 0, j)] = F[2 * N + at(g, 0, j)] = 0.0;
    curl_E_lattice(g, F, curl); /* curl E^{n+1} */
    for (int64_t k = 0; k < 3 * N; k++) F[3 * N + k] -= 0.5 * g->dt * curl[k];
    free(curl);
}

void or_div_E(const or_grid* g, const double* F, double* out) {
    const int64_t N = (int64_t)g->nx * g->ny;
    const double *Ex = F, *Ey = F + N;
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            const int64_t k = at(g, i, j);
            out[k] = (val(g, Ex, 1, i, j) - val(g, Ex, 1, i - 1, j)) / g->dx +
                     (val(g, Ey, 0, i, j) - val(g, Ey, 0, i, j - 1)) / g->dy;
        }
}

void or_div_J(const or_grid* g, const double* J, double* out) {
    or_div_E(g, J, out); /* J shares the E lattices */
}

void or_div_B(const or_grid* g, const double* F, double* out) {
    const int64_t N = (int64_t)g->nx * g->ny;
    const double *Bx = F + 3 * N, *By = F + 4 * N;
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            const int64_t k = at(g, i, j);
            out[k] = (val(g, Bx, 0, i + 1, j) - val(g, Bx, 0, i, j)) / g->dx +
                     (val(g, By, 1, i, j + 1) - val(g, By, 1, i, j)) / g->dy;
        }
}

void or_field_energy(const or_grid* g, const double* F, double* UE, double* UB) {
    const int64_t N = (int64_t)g->nx * g->ny;
    const double w = g->dx * g->dy / (8.0 * PI);
    *UE = w * dot(3 * N, F, F);
    *UB = w * dot(3 * N, F + 3 * N, F + 3 * N);
}
