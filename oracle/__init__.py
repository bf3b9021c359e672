"""Plain FP64 CPU oracle of the 2D implicit-FDTD PIC particle cycle.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this package. The CUDA product never imports, links or
calls it, and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, single-threaded, FP64); this module
compiles it with gcc, loads it with ctypes and sequences one time step the way the
paper orders it (Ikeya & Matsumoto, PASJ 2015, Sec. 2 and Sec. 3): gather and push with
E^n, B^n; deposit J^{n+1/2}; right-hand side and CG solve of Eq. (7); field update from
Eqs. (5)-(6).

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: the paper's dispersion relation Eqs. (10) and (15), discrete charge
conservation, exact Boris gyration, a spectral solve of Eq. (7), scipy's B-splines
and closed-form current sums.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, -O2, no fast-math)."""
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest_src:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("dx", C.c_double),
                ("dy", C.c_double), ("dt", C.c_double), ("theta", C.c_double),
                ("order", C.c_int32), ("walls", C.c_int32), ("nodal", C.c_int32)]


_P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            G = C.POINTER(Grid)
            L.or_shape.restype = C.c_double
            L.or_shape.argtypes = [C.c_int32, C.c_double]
            L.or_gather.argtypes = [G, _P, C.c_int64, _P, _P, _P]
            L.or_boris.argtypes = [C.c_double, C.c_double, C.c_int64, _P, _P, _P]
            L.or_deposit_move.argtypes = [G, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, _P]
            L.or_push_deposit.restype = C.c_int64
            L.or_push_deposit.argtypes = [G, _P, C.c_double, C.c_double, C.c_int64, _P, _P, _P,
                                          _P, _P, _P, C.c_int32]
            L.or_deposit_rho.argtypes = [G, C.c_double, C.c_int64, _P, _P, _P]
            L.or_rhs.argtypes = [G, _P, _P, _P]
            L.or_apply_A.argtypes = [G, _P, _P]
            L.or_pcg.restype = C.c_int32
            L.or_pcg.argtypes = [G, _P, _P, C.c_double, C.c_int32, C.POINTER(C.c_double)]
            L.or_field_update.argtypes = [G, _P, _P, _P]
            L.or_explicit_update.argtypes = [G, _P, _P]
            for name in ("or_div_E", "or_div_B", "or_div_J"):
                getattr(L, name).argtypes = [G, _P, _P]
            L.or_field_energy.argtypes = [G, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            _lib = L
    return _lib


def grid(nx, ny, dt, theta, order, dx=1.0, dy=1.0, walls=False, gather="staggered") -> Grid:
    """gather: "staggered" (each component on its own lattice) or "nodal" (fields
    averaged to the nodes first; periodic only)."""
    if nx < 8 or ny < 8:
        raise ValueError("the oracle needs nx, ny >= 8")
    if gather not in ("staggered", "nodal") or (gather == "nodal" and walls):
        raise ValueError("gather must be 'staggered' or 'nodal' (nodal without walls)")
    return Grid(int(nx), int(ny), float(dx), float(dy), float(dt), float(theta), int(order),
                1 if walls else 0, 1 if gather == "nodal" else 0)


def wall_nodes_zeroed(F, nx, ny):
    """Fields with the conductor's zeros on the wall column (Ey, Ez, Bx at x = 0)."""
    F = _c(F).reshape(6, ny, nx).copy()
    F[[1, 2, 3], :, 0] = 0.0
    return F.ravel()


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- thin wrappers (one call = one C function) ----------------------------------

def shape(p, d):
    L = lib()
    return np.array([L.or_shape(int(p), float(v)) for v in np.ravel(d)]).reshape(np.shape(d))


def gather(g, F, x, y):
    x, y = _c(x), _c(y)
    out = np.zeros(6 * x.size)
    lib().or_gather(C.byref(g), _c(F).ravel(), x.size, x, y, out)
    return out.reshape(6, x.size)


def boris(qm, dt, E, B, u):
    """E, B, u: arrays of shape (n, 3). Returns the pushed momenta (n, 3)."""
    u = _c(u).copy()
    lib().or_boris(float(qm), float(dt), u.shape[0], _c(E).ravel(), _c(B).ravel(), u.ravel())
    return u


def deposit_move(g, qw, x0, y0, x1, y1, vz, J=None):
    if J is None:
        J = np.zeros(3 * g.nx * g.ny)
    lib().or_deposit_move(C.byref(g), qw, x0, y0, x1, y1, vz, J)
    return J


def push_deposit(g, F, qm, qw, x, y, ux, uy, uz, J=None, deposit=True):
    """One species' gather, push, move, deposit and wrap. Updates x..uz in place
    (they must be float64 C-contiguous) and returns (J, number of bad moves)."""
    if J is None:
        J = np.zeros(3 * g.nx * g.ny)
    for a in (x, y, ux, uy, uz):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("particle arrays must be C-contiguous float64")
    bad = lib().or_push_deposit(C.byref(g), _c(F).ravel(), float(qm), float(qw), x.size, x, y,
                                ux, uy, uz, J, 1 if deposit else 0)
    return J, int(bad)


def deposit_rho(g, qw, x, y, rho=None):
    x, y = _c(x), _c(y)
    if rho is None:
        rho = np.zeros(g.nx * g.ny)
    lib().or_deposit_rho(C.byref(g), float(qw), x.size, x, y, rho)
    return rho


def rhs(g, F, J):
    b = np.zeros(3 * g.nx * g.ny)
    lib().or_rhs(C.byref(g), _c(F).ravel(), _c(J).ravel(), b)
    return b


def apply_A(g, x):
    out = np.zeros(3 * g.nx * g.ny)
    lib().or_apply_A(C.byref(g), _c(x).ravel(), out)
    return out


def pcg(g, b, x0=None, rtol=1e-10, maxit=1000):
    x = np.zeros(3 * g.nx * g.ny) if x0 is None else _c(x0).ravel().copy()
    rr = C.c_double(0.0)
    it = lib().or_pcg(C.byref(g), _c(b).ravel(), x, float(rtol), int(maxit), C.byref(rr))
    return x, int(it), rr.value


def field_update(g, F, dB, J):
    F = _c(F).ravel().copy()
    lib().or_field_update(C.byref(g), F, _c(dB).ravel(), _c(J).ravel())
    return F


def explicit_update(g, F, J):
    """Explicit FDTD step of the fields, Eqs. (3)-(4) (see oracle.h)."""
    F = _c(F).ravel().copy()
    lib().or_explicit_update(C.byref(g), F, _c(J).ravel())
    return F


def div_E(g, F):
    out = np.zeros(g.nx * g.ny)
    lib().or_div_E(C.byref(g), _c(F).ravel(), out)
    return out


def div_B(g, F):
    out = np.zeros(g.nx * g.ny)
    lib().or_div_B(C.byref(g), _c(F).ravel(), out)
    return out


def div_J(g, J):
    out = np.zeros(g.nx * g.ny)
    lib().or_div_J(C.byref(g), _c(J).ravel(), out)
    return out


# ---- Fourier diagnostics (Sec. 3.1, Fig. 3) --------------------------------------------
def spectrum(F2d):
    """Amplitude |sum_{l,m} F(l,m) exp(-2 pi i (p l/nx + q m/ny))| / (nx ny) of an (ny, nx)
    grid quantity, p and q in FFT order; numpy's FFT is the library step."""
    F2d = np.asarray(F2d, dtype=np.float64)
    return np.abs(np.fft.fft2(F2d)) / F2d.size


def resonance_ky(cfl_x, cfl_y, beta, kx_dx):
    """Eq. (17): the k_y dy >= 0 at which the flow's mode omega = V k_x (beta = V/c) lies
    on the theta = 1/2 vacuum dispersion surface, Eq. (15), with S_x = cfl_x sin(k_x dx/2)
    and cfl = c dt / d. None where the square root or the arcsine has no real value."""
    half_phase = beta * cfl_x * kx_dx / 2.0  # V k_x dt / 2
    if not (0.0 < half_phase < math.pi / 2):
        return None
    radicand = math.tan(half_phase) ** 2 - (cfl_x * math.sin(kx_dx / 2.0)) ** 2
    if radicand < 0.0:
        return None
    s = math.sqrt(radicand) / cfl_y
    if s > 1.0:
        return None
    return 2.0 * math.asin(s)


def field_energy(g, F):
    ue, ub = C.c_double(), C.c_double()
    lib().or_field_energy(C.byref(g), _c(F).ravel(), C.byref(ue), C.byref(ub))
    return ue.value, ub.value


# ---- one whole step --------------------------------------------------------------

class Species:
    """One particle species: charge-to-mass sign qm = +-1, macro weight w (charge
    per macro-particle q = qm*w, mass w), physical positions and momenta u = gamma v."""

    def __init__(self, qm, w, x, y, ux, uy, uz):
        self.qm, self.w = float(qm), float(w)
        self.x, self.y = _c(x).copy(), _c(y).copy()
        self.ux, self.uy, self.uz = _c(ux).copy(), _c(uy).copy(), _c(uz).copy()

    @property
    def n(self):
        return self.x.size

    def kinetic_energy(self):
        return self.w * float(np.sum(np.sqrt(1.0 + self.ux**2 + self.uy**2 + self.uz**2) - 1.0))


# ---- the moving injector of the shock set-up ------------------------------------------
# A plane starting at x_f(0) = x0 (cells) moves toward +x at c, x_f(n) = x0 + n cfl, and
# keeps the beam flowing toward the wall at x = 0 uninterrupted behind it: at the end of
# step n the slab [x_f(n+1) - w, x_f(n+1)) of every row, w = (1 + v) cfl (uncovered
# because the beam moved -v dt while the plane moved c dt), receives
# floor(ppc w (n+1)) - floor(ppc w n) co-located pairs (the beam density over time), at
# uniform random positions, with rest-frame Gaussian momenta of spread u_th boosted to
# gamma0 toward -x; none once x_f(n+1) > nx. Random numbers: splitmix64 (Steele, Lea &
# Flood 2014) of the counter seed K0 + n K1 + j K2 + k K3 + s K4 + d, uniform
# ((h >> 11) + 1/2) 2^-53; Box-Muller for the Gaussians.
_INJ_K = (0xD1B54A32D192ED03, 0xABC98388FB8FAC03, 0x8CB92BA72F3D8DD7, 0x9E3779B97F4A7C15,
          0xC2B2AE3D27D4EB4F)


def splitmix64(z):
    """The splitmix64 output function of the counter z (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def inject_uniform(seed, n, j, k, s, d):
    """Uniform in (0, 1) for draw d of pair k (array) of row j (array) at step n, species s."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(_INJ_K[0]) + np.uint64(n) * np.uint64(_INJ_K[1]) +
               np.asarray(j, dtype=np.uint64) * np.uint64(_INJ_K[2]) +
               np.asarray(k, dtype=np.uint64) * np.uint64(_INJ_K[3]) +
               np.uint64(s) * np.uint64(_INJ_K[4]) + np.uint64(d))
    h = splitmix64(key)
    return ((h >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def inject_pairs(n, nx, ny, cfl, x0, ppc, gamma0, u_th, seed):
    """Pairs entering at the end of step n: (x, y) in cells and [(ux, uy, uz)] per species."""
    w = (1.0 + math.sqrt(1.0 - 1.0 / (gamma0 * gamma0))) * cfl
    xf = x0 + (n + 1) * cfl
    if xf > nx:
        return None
    per_row = int(math.floor((ppc * w) * (n + 1))) - int(math.floor((ppc * w) * n))
    if per_row <= 0:
        return None
    j = np.repeat(np.arange(ny), per_row)
    k = np.tile(np.arange(per_row), ny)
    x = xf - w * inject_uniform(seed, n, j, k, 0, 0)
    y = j + inject_uniform(seed, n, j, k, 0, 1)
    beta0 = math.sqrt(1.0 - 1.0 / (gamma0 * gamma0))
    mom = []
    for s in (0, 1):
        r0 = np.sqrt(-2.0 * np.log(inject_uniform(seed, n, j, k, s, 2)))
        a0 = 2.0 * math.pi * inject_uniform(seed, n, j, k, s, 3)
        r1 = np.sqrt(-2.0 * np.log(inject_uniform(seed, n, j, k, s, 4)))
        a1 = 2.0 * math.pi * inject_uniform(seed, n, j, k, s, 5)
        upx, upy, upz = u_th * r0 * np.cos(a0), u_th * r0 * np.sin(a0), u_th * r1 * np.cos(a1)
        gp = np.sqrt(1.0 + upx * upx + upy * upy + upz * upz)
        mom.append((-gamma0 * (upx + beta0 * gp), upy, upz))
    return x, y, mom


class OracleSim:
    """The per-step particle cycle, in the paper's order (Sec. 2, Sec. 3):

    1. every species: gather E^n, B^n at x^n; Boris push u^{n-1/2} -> u^{n+1/2};
       move; Esirkepov deposit of J^{n+1/2}; periodic wrap;
    2. right-hand side b of Eq. (7) from B^n, E^n, J^{n+1/2};
    3. PCG solve of [1 - (theta c dt)^2 Lap] dB = b from the initial guess
       (zero, or the previous step's dB when warm_start == "prev");
    4. E^{n+1}, B^{n+1} from Eqs. (5)-(6).
    """

    def __init__(self, nx, ny, cfl, theta, order, species, dx=1.0, dy=1.0,
                 cg_rtol=1e-10, cg_max_iter=1000, warm_start="zero", fields=None,
                 deposit=True, walls=False, injector=None, solver="implicit", gather="staggered"):
        self.g = grid(nx, ny, cfl * dx, theta, order, dx, dy, walls, gather)
        # "implicit": Eq. (7) by PCG and Eqs. (5)-(6); "explicit": Eqs. (3)-(4)
        if solver not in ("implicit", "explicit"):
            raise ValueError("solver must be 'implicit' or 'explicit'")
        self.solver = solver
        self.N = nx * ny
        self.species = list(species)
        self.F = np.zeros(6 * self.N) if fields is None else _c(fields).ravel().copy()
        if walls:
            self.F = wall_nodes_zeroed(self.F, nx, ny)
        # injector: dict(x0=, ppc=, gamma0=, u_th=, seed=) (with walls); needs both species
        self.injector = dict(injector) if injector else None
        self.cfl = float(cfl)
        self.J = np.zeros(3 * self.N)
        self.dB = np.zeros(3 * self.N)
        self.cg_rtol, self.cg_max_iter = float(cg_rtol), int(cg_max_iter)
        self.warm_start = warm_start
        self.deposit = bool(deposit)
        self.step_count = 0
        self.last_cg_iters = 0
        self.last_cg_resid = 0.0
        self.bad_moves = 0

    def push_deposit(self):
        L = lib()
        self.J[:] = 0.0
        for s in self.species:
            self.bad_moves += int(L.or_push_deposit(
                C.byref(self.g), self.F, s.qm, s.qm * s.w, s.n, s.x, s.y, s.ux, s.uy,
                s.uz, self.J, 1 if self.deposit else 0))

    def field_solve(self):
        if self.solver == "explicit":
            self.F = explicit_update(self.g, self.F, self.J)
            self.last_cg_iters, self.last_cg_resid = 0, 0.0
            return
        b = rhs(self.g, self.F, self.J)
        x0 = self.dB if self.warm_start == "prev" else None
        dB, it, rr = pcg(self.g, b, x0, self.cg_rtol, self.cg_max_iter)
        if it < 0:
            raise RuntimeError(f"oracle PCG did not converge in {self.cg_max_iter} iterations")
        self.dB = dB
        self.last_cg_iters, self.last_cg_resid = it, rr
        self.F = field_update(self.g, self.F, dB, self.J)

    def inject(self):
        q = self.injector
        new = inject_pairs(self.step_count, self.g.nx, self.g.ny, self.cfl, q["x0"], q["ppc"],
                           q["gamma0"], q["u_th"], q["seed"])
        if new is None:
            return
        x, y, mom = new
        for s, sp in enumerate(self.species):
            sp.x = np.concatenate([sp.x, x * self.g.dx])
            sp.y = np.concatenate([sp.y, y * self.g.dy])
            sp.ux = np.concatenate([sp.ux, mom[s][0]])
            sp.uy = np.concatenate([sp.uy, mom[s][1]])
            sp.uz = np.concatenate([sp.uz, mom[s][2]])

    def step(self, n=1):
        for _ in range(int(n)):
            self.push_deposit()
            if self.injector:
                self.inject()
            self.field_solve()
            self.step_count += 1

    # diagnostics
    def fields(self):
        return self.F.reshape(6, self.g.ny, self.g.nx)

    def energies(self):
        ue, ub = field_energy(self.g, self.F)
        return ue, ub, sum(s.kinetic_energy() for s in self.species)

    def rho(self):
        r = np.zeros(self.N)
        for s in self.species:
            deposit_rho(self.g, s.qm * s.w, s.x, s.y, r)
        return r

