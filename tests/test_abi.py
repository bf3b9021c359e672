"""The C-ABI library loads and exports every symbol include/pic.h declares; host-side
parameter validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_1412_2480_gb300 as pic
from paper_1412_2480_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            names |= set(re.findall(r"PIC_API\s+[\w\s\*]+?\b(pic_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpic():
    pkg_build.build()
    return ctypes.CDLL(pkg_build.LIB)


def test_every_declared_symbol_is_exported(libpic):
    names = declared_symbols()
    assert "pic_step" in names and "pic_init" in names and len(names) >= 12
    for n in names:
        assert hasattr(libpic, n), n
    assert set(pic.EXPORTED) <= names


def test_struct_layouts_match_header():
    # sizes computed by the C compiler must equal the ctypes mirrors
    import subprocess
    import tempfile
    src = '#include <stdio.h>\n#include "pic.h"\nint main(void){printf("%zu %zu", sizeof(pic_params), sizeof(pic_moments_t));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        a, b = map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split())
    assert a == ctypes.sizeof(pic.pic_params)
    assert b == ctypes.sizeof(pic.pic_moments_t)


def test_defaults_and_validation_on_host():
    p = pic.pic_params_default()
    assert (p.nx, p.ny, p.cfl, p.theta, p.shape_order) == (64, 64, 1.0, 0.5, 1)
    assert p.cg_rtol == 1e-10 and p.cg_max_iter == 200
    bad = [dict(nx=4), dict(cfl=1.5), dict(cfl=0.0), dict(theta=0.4), dict(theta=1.2),
           dict(shape_order=4), dict(gamma0=0.5), dict(ppc=0), dict(precision=7),
           dict(cg_rtol=0.0), dict(cg_max_iter=0), dict(warm_start=5), dict(dx=-1.0),
           dict(cfl=1.0, dx=2.0, dy=1.0)]
    for kw in bad:
        with pytest.raises(pic.PicError) as e:
            pic.pic_init(pic.pic_params_default(**kw))
        assert e.value.code == pic.PIC_EINVAL, kw
        assert pic.pic_last_error(None)


def test_init_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pic.PicError) as e:
        pic.pic_init(pic.pic_params_default())
    assert e.value.code in (pic.PIC_ECUDA, pic.PIC_ENOMEM)


def test_batch_validation_on_host():
    mixed = pic.pic_params_default(precision=pic.PIC_MIXED32)
    fp64 = pic.pic_params_default()
    cases = [[fp64, fp64],                                   # FP64 batches of > 1 are refused
             [mixed, pic.pic_params_default(precision=pic.PIC_MIXED32, flags=pic.PIC_NO_GRAPH)],
             [mixed, pic.pic_params_default(precision=pic.PIC_MIXED32, nx=4)],
             [pic.pic_params_default(precision=pic.PIC_MIXED32, nx=256, ny=256, tile_x=200, tile_y=200)]]
    for ps in cases:
        with pytest.raises(pic.PicError) as e:
            pic.pic_init_batch(ps)
        assert e.value.code == pic.PIC_EINVAL
        assert pic.pic_last_error(None)
    with pytest.raises(pic.PicError) as e:
        pic.pic_init_batch([])
    assert e.value.code == pic.PIC_EINVAL
    with pytest.raises(pic.PicError) as e:
        pic.pic_autotune_tiles([mixed], steps=0)
    assert e.value.code == pic.PIC_EINVAL
    assert pic.pic_batch_size(None) == 0


def test_walls_parameter_validation_on_host():
    for kw in (dict(bc_x=2), dict(bc_x=pic.PIC_BC_WALLS, precision=pic.PIC_FP64,
                                  warm_start=pic.PIC_WS_LEARNED)):
        with pytest.raises(pic.PicError) as e:
            pic.pic_init(pic.pic_params_default(**kw))
        assert e.value.code == pic.PIC_EINVAL


def test_return_codes_match_header():
    text = open(os.path.join(ROOT, "include", "pic.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"#define (PIC_E\w+|PIC_OK) \((-?\d+)\)", text))
    codes.update((k, int(v)) for k, v in re.findall(r"#define (PIC_OK) (\d+)", text))
    assert "PIC_ETIMEOUT" in codes and len(codes) >= 9
    for name, value in codes.items():
        assert getattr(pic, name) == value, name
