"""Config 5 as stated, at reduced size, over a long run: the relativistic shock of Sec. 4
(a magnetised pair beam, sigma_B = 0.1, gamma0 = 40, 16 particles per cell per species,
flowing into the conducting wall at x = 0 and fed by the moving injector; CFL 1,
theta = 0.501, shape order 3) on 1024 x 128 cells for 400 steps, in the form config 5
names: FP32 particles (MIXED32) with the learned warm start. The network is trained on
the GPU first, from this CFL and theta, by the library's own kernels.

The paper measures the magnetic noise the upstream beam carries. Reading: the noise
energy sum |B - B0 z|^2 dx dy / (8 pi) over the band 256 <= x < 512, which holds
upstream beam throughout (the shock stays below x = 256 within 400 steps). The oracle's
record (tests/golden/shock_noise_reduced.json, written by tests/golden/
make_shock_noise.py from the oracle alone: an hour of one host core) is compared with
the GPU run from the same seeded inputs (their SHA-256 is checked) in 50-step windows
once the noise has grown out of the particles' shot noise, within 5 %; the particle
count (loaded plus injected) must match exactly."""
import importlib.util
import json
import os

import numpy as np
import pytest

import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import warmstart

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_shock_noise", os.path.join(HERE, "make_shock_noise.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    return mk


def _digest(sp):
    import hashlib
    h = hashlib.sha256()
    for d in sp:
        for k in ("x", "y", "ux", "uy", "uz"):
            h.update(np.ascontiguousarray(d[k], dtype=np.float64).tobytes())
    return h.hexdigest()


def test_reduced_shock_upstream_noise_matches_oracle():
    path = os.path.join(HERE, "shock_noise_reduced.json")
    d = json.load(open(path))
    mk = _maker()
    w, sp, F0, inj = mk.setup()
    assert _digest(sp) == d["input_sha256"], "the seeded inputs differ from the stored oracle run's"
    b0 = d["b0"]
    # the learned warm start of this CFL and theta
    B, X = warmstart.generate_pairs(steps=2500, seeds=(11, 12), cfl=mk.CFL, theta=mk.THETA, order=1, ppc=8,
                                    gamma0=20.0)
    net, loss, _ = warmstart.train(B, X, iters=2000)
    try:
        prm = pic.pic_params_default(nx=mk.NX, ny=mk.NY, ppc=mk.PPC, shape_order=mk.ORDER, gamma0=mk.GAMMA0,
                                     u_th=mk.UTH, cfl=mk.CFL, theta=mk.THETA, precision=pic.PIC_MIXED32,
                                     cg_rtol=1e-10, warm_start=pic.PIC_WS_LEARNED, bc_x=pic.PIC_BC_WALLS,
                                     inject_x0=float(mk.X0), seed=mk.INJ_SEED)
        h = pic.pic_init(prm)
        noise, npart, iters = [], [], 0
        try:
            pic.pic_set_cnn(h, net)
            for c in range(6):
                pic.pic_set_fields(h, c, np.ascontiguousarray(F0[c]).ravel())
            for s, x in enumerate(sp):
                pic.pic_load_particles(h, s, x["x"], x["y"], x["ux"], x["uy"], x["uz"])
            for _ in range(mk.STEPS):
                pic.pic_step(h, 1)
                m = pic.pic_moments(h)
                assert m["cg_rel_resid"] <= 1e-10
                iters += m["cg_iters_last"]
                F = np.zeros((6, mk.NY, mk.NX))
                for c in (3, 4, 5):
                    F[c] = pic.fields_numpy(h, c, mk.NX, mk.NY)
                noise.append(mk.band_noise(F, b0))
                npart.append(m["n_particles"][0])
        finally:
            pic.pic_free(h)
    finally:
        pic.pic_cnn_free(net)
    ref = np.array(d["after_step"]["band_noise"])
    got = np.array(noise)
    assert npart == d["after_step"]["n_per_species"]
    wo, wg = ref.reshape(-1, 50).mean(axis=1), got.reshape(-1, 50).mean(axis=1)
    grown = wo > 1e3 * ref[:10].mean()  # past the particles' shot noise
    rel = np.abs(wg - wo) / wo
    print(f"network loss {loss:.2e}; inner PCG iterations {iters / mk.STEPS:.2f} per step; band noise per "
          f"50-step window, oracle {np.array2string(wo, precision=3)}, GPU/oracle - 1 "
          f"{np.array2string(wg / wo - 1, precision=4)}")
    assert grown.sum() >= 4
    assert np.all(rel[grown] <= 0.05), rel
