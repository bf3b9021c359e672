/*
 * oracle.h -- plain FP64 CPU reference of the 2D implicit-FDTD PIC particle cycle
 * (Ikeya & Matsumoto, "Stability Property of Numerical Cherenkov Radiation and its
 * Application to Relativistic Shock Simulations", PASJ 2015, arXiv:1412.2480).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library. The product (the CUDA library
 * under paper_1412_2480_gb300/) never links, loads or calls it; the two share no
 * code, header, table or helper.
 *
 * Units and conventions (the paper's Sec. 2 uses Gaussian units; c = 1 here):
 *   grid     nx x ny cells of size dx x dy; node (i,j) sits at (i dx, j dy); periodic in
 *            y, and in x either periodic or closed by two conducting, reflecting walls
 *            at x = 0 and x = nx dx (walls != 0; the shock configuration, Sec. 4).
 *   walls    mirror images (the method of images for a perfect conductor): a quantity
 *            on an integer-x lattice (Ey, Ez, Bx, Jy, Jz, rho) is odd under reflection
 *            at a wall, so it vanishes on the wall nodes; one on a half-integer lattice
 *            (Ex, By, Bz, Jx) is even. Values beyond a wall are read from the image;
 *            deposits beyond a wall fold back with the image's sign. This gives the
 *            conductor conditions Ey = Ez = Bx = 0 on the walls, Neumann conditions for
 *            By and Bz, and a symmetric positive definite operator in Eq. (7).
 *   storage  every grid quantity is an nx*ny array, index k = j*nx + i; the value
 *            stored at k lives at the quantity's own staggered position (Fig. 1 of
 *            the paper has no content; the standard 2D Yee arrangement is used):
 *              Ez, Jz, rho at (i    , j    )
 *              Ex, Jx, By  at (i+1/2, j    )
 *              Ey, Jy, Bx  at (i    , j+1/2)
 *              Bz          at (i+1/2, j+1/2)
 *   fields   one array of 6*nx*ny doubles: Ex, Ey, Ez, Bx, By, Bz (component-major).
 *   current  one array of 3*nx*ny doubles: Jx, Jy, Jz.
 *   dB, rhs  arrays of 3*nx*ny doubles on the B lattices: x, y, z components.
 *   particles  physical positions x in [0, nx dx), y in [0, ny dy); momenta
 *            u = gamma v (units of c); charge per macro-particle q = s*w,
 *            mass per macro-particle w (so q/m = s = +-1).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t nx, ny;   /* cells; both must be >= 8 */
    double dx, dy;    /* cell size */
    double dt;        /* time step; CFL number sigma = c dt / dx (Sec. 3.1) */
    double theta;     /* implicitness factor of Eqs. (5)-(6), 0.5 <= theta <= 1 */
    int32_t order;    /* particle shape order 1, 2 or 3 */
    int32_t walls;    /* 0: periodic in x; 1: conducting, reflecting walls at x = 0, nx dx */
    int32_t nodal;    /* gather reading: 0 each component on its own staggered lattice;
                         1 the fields averaged to the nodes first (periodic only) */
} or_grid;

/* Centred cardinal B-spline of order p (degree p): the particle shape. */
double or_shape(int32_t p, double d);

/* Momentum-conserving gather of the 6 field components for n particles (Sec. 1).
 * out is 6*n, component-major (Ex..Bz). */
void or_gather(const or_grid* g, const double* F, int64_t n, const double* x,
               const double* y, double* out);

/* Relativistic Buneman-Boris push of n momenta with given E (3n) and B (3n),
 * component-major per particle ([E0x,E0y,E0z,E1x,...]). */
void or_boris(double qm, double dt, int64_t n, const double* E, const double* B, double* u);

/* Esirkepov (density decomposition) current of one macro-particle of charge qw
 * moving in a straight line from (x0,y0) to (x1,y1) (physical units, unwrapped,
 * |x1-x0| < dx and |y1-y0| < dy) with out-of-plane velocity vz. Adds into J. */
void or_deposit_move(const or_grid* g, double qw, double x0, double y0, double x1,
                     double y1, double vz, double* J);

/* One species' gather, push, move, deposit and periodic wrap (the particle half of
 * the step). Updates x, y, ux, uy, uz in place; adds the current into J when
 * deposit != 0. Returns the number of particles whose displacement was not
 * below one cell in x or y (or was NaN). */
int64_t or_push_deposit(const or_grid* g, const double* F, double qm, double qw, int64_t n,
                        double* x, double* y, double* ux, double* uy, double* uz,
                        double* J, int32_t deposit);

/* Node charge density rho (nx*ny) of n macro-particles of charge qw, added into rho. */
void or_deposit_rho(const or_grid* g, double qw, int64_t n, const double* x,
                    const double* y, double* rho);

/* Right-hand side of Eq. (7): b = theta (c dt)^2 (Lap B + (4 pi/c) curl J) - c dt curl E. */
void or_rhs(const or_grid* g, const double* F, const double* J, double* b);

/* Operator of Eq. (7): Ax = x - (theta c dt)^2 Lap x on each B lattice. */
void or_apply_A(const or_grid* g, const double* x, double* Ax);

/* Jacobi-preconditioned conjugate gradient on Eq. (7) (Sec. 2). x holds the initial
 * guess on entry and the solution on exit. Stops when ||r||_2 <= rtol ||b||_2.
 * Returns the iteration count, or -1 if maxit was reached first. If ||b|| = 0 the
 * solution is x = 0. *rel_resid receives ||r||/||b|| (0 when ||b|| = 0). */
int32_t or_pcg(const or_grid* g, const double* b, double* x, double rtol, int32_t maxit,
               double* rel_resid);

/* Field update from Eqs. (5)-(6) with dB: E += c dt curl(B + theta dB) - 4 pi dt J,
 * then B += dB. */
void or_field_update(const or_grid* g, double* F, const double* dB, const double* J);

/* Explicit FDTD update, Eqs. (3)-(4), B kept at integer time levels: B^{n+1/2} =
 * B^n - (c dt/2) curl E^n; E^{n+1} = E^n + c dt curl B^{n+1/2} - 4 pi dt J^{n+1/2};
 * B^{n+1} = B^{n+1/2} - (c dt/2) curl E^{n+1}. theta is not used. */
void or_explicit_update(const or_grid* g, double* F, const double* J);

/* Discrete divergences: div E at nodes (nx*ny), div B at cell centres (nx*ny). */
void or_div_E(const or_grid* g, const double* F, double* out);
void or_div_B(const or_grid* g, const double* F, double* out);

/* Discrete divergence of J at nodes (nx*ny). */
void or_div_J(const or_grid* g, const double* J, double* out);

/* Field energies U_E = sum |E|^2 dx dy / 8 pi and U_B likewise. */
void or_field_energy(const or_grid* g, const double* F, double* UE, double* UB);

#ifdef __cplusplus
}
#endif
#endif
