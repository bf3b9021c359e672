"""Runs the same seeded workload through the CUDA library (C ABI) and through the oracle.

Inputs come only from paper_1412_2480_gb300.inputs; nothing the CUDA path produces is
ever fed to the oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import inputs


def workload(nx, ny, ppc, gamma0=20.0, u_th=1e-3, seed=1, field_amp=0.0, colocated=True):
    w, sp = inputs.drifting_pair_plasma(nx, ny, ppc, gamma0, u_th, seed, colocated=colocated)
    F0 = inputs.random_fields(nx, ny, field_amp, seed) if field_amp else np.zeros((6, ny, nx))
    return w, sp, F0


def run_gpu(nx, ny, ppc, sp, F0, steps, order, cfl=1.0, theta=0.5, gamma0=20.0,
            precision=pic.PIC_FP64, want_particles=True, **kw):
    prm = pic.pic_params_default(nx=nx, ny=ny, cfl=cfl, theta=theta, shape_order=order,
                                 gamma0=gamma0, ppc=ppc, precision=precision, **kw)
    h = pic.pic_init(prm)
    try:
        if np.any(F0):
            for c in range(6):
                pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c], dtype=np.float64).ravel())
        for s in range(len(sp)):
            d = sp[s]
            pic.pic_load_particles(h, s, d["x"], d["y"], d["ux"], d["uy"], d["uz"])
        pic.pic_step(h, steps)
        F = np.stack([pic.fields_numpy(h, c, nx, ny) for c in range(12)])
        parts = [pic.pic_particles(h, s) for s in range(len(sp))] if want_particles else None
        mom = pic.pic_moments(h)
    finally:
        pic.pic_free(h)
    return F, parts, mom


def run_oracle(nx, ny, w, sp, F0, steps, order, cfl=1.0, theta=0.5, cg_rtol=1e-10,
               warm_start="zero", deposit=True, walls=False, solver="implicit", gather="staggered"):
    species = [oracle.Species(d["qm"], w, d["x"], d["y"], d["ux"], d["uy"], d["uz"]) for d in sp]
    sim = oracle.OracleSim(nx, ny, cfl, theta, order, species, cg_rtol=cg_rtol, fields=F0,
                           warm_start=warm_start, deposit=deposit, walls=walls, solver=solver,
                           gather=gather)
    sim.step(steps)
    F = np.concatenate([sim.fields(), sim.J.reshape(3, ny, nx), sim.dB.reshape(3, ny, nx)])
    parts = [np.stack([s.x, s.y, s.ux, s.uy, s.uz]) for s in sim.species]
    return F, parts, sim


def rel(a, b):
    """Norm-wise relative difference ||a - b|| / ||b||."""
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def relmax(a, b, scale=None):
    """Element-wise relative difference max|a - b| / max|b| (or / scale when given):
    a wrong tile-edge column or wall node is not diluted by the grid size here."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    m = float(np.abs(b).max()) if scale is None else float(scale)
    return float(np.abs(a - b).max() / (m if m > 0 else 1.0))


def check(a, b, tol, what="", scale=None):
    """Parity of one quantity: both the norm-wise and the element-wise relative
    difference within tol. With scale (the largest magnitude of the summed terms, e.g.
    one species' largest current where two species cancel) only the element-wise bound
    max|a - b| / scale is checked here; the caller bounds the norm-wise one itself."""
    if scale is None:
        r, m = rel(a, b), relmax(a, b)
        assert r < tol and m < tol, f"{what}: norm-wise {r:.2e}, element-wise {m:.2e} (bound {tol:.0e})"
    else:
        m = relmax(a, b, scale)
        assert m < tol, f"{what}: element-wise {m:.2e} of the scale (bound {tol:.0e})"


def check_rows(a, b, tol, what=""):
    """check() for each row (component) of two arrays shaped (components, n)."""
    for k in range(np.asarray(b).shape[0]):
        check(np.asarray(a)[k], np.asarray(b)[k], tol, f"{what} row {k}")


def match_particles(g, o, scale):
    """Pairs every particle of g (5 x n: x, y, ux, uy, uz) with its nearest particle of o
    in coordinates divided by scale (5 values) and returns the largest paired distance,
    or infinity when the pairing is not one to one. Unlike a comparison of sorted arrays
    it does not break when two particles closer than the round-off swap their order."""
    from scipy.spatial import cKDTree
    if g.shape != o.shape:
        return float("inf")
    if g.shape[1] == 0:
        return 0.0
    sc = np.asarray(scale, dtype=np.float64)[:, None]
    d, idx = cKDTree((o / sc).T).query((g / sc).T)
    if np.unique(idx).size != idx.size:
        return float("inf")
    return float(d.max())


def periodic_pos_err(a, b, L):
    """Largest position difference modulo the box length."""
    d = np.abs(a - b)
    return float(np.max(np.minimum(d, L - d))) if d.size else 0.0
