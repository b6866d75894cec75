"""CPU checks of the C ABI: the library builds and loads, exports every
function include/sdeb.h declares, the ctypes struct matches the C layout,
and argument validation fails cleanly without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdeb.h")


@pytest.fixture(scope="module")
def L():
    sdeb_build.build()
    return sdeb.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SDEB_API\s+[\w\s\*]*?\b(sdeb_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(sdeb.EXPORTED_SYMBOLS)


def test_problem_struct_layout_matches_header(L):
    fields = [f for f, _ in sdeb.Problem._fields_]
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "sdeb.h"', "int main(void){",
           'printf("%zu\\n", sizeof(sdeb_problem));']
    for f in fields:
        src.append('printf("%%zu\\n", offsetof(sdeb_problem, %s));' % f)
    src.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write("\n".join(src))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(sdeb.Problem)
    for f, off in zip(fields, out[1:]):
        assert getattr(sdeb.Problem, f).offset == off, f


def _status(L, pb):
    ctx = ctypes.c_void_p()
    st = L.sdeb_create(ctypes.byref(pb), ctypes.byref(ctx))
    if st == sdeb.SDEB_OK:
        L.sdeb_destroy(ctx)
    else:
        assert not ctx.value
    return st


def test_validation_rejects_bad_problems(L):
    good = dict(model="kuramoto", n=8, orbits=16, dt=0.01, steps=100, stride=10)
    bad = [
        dict(good, n=0), dict(good, orbits=0), dict(good, dt=0.0), dict(good, dt=float("nan")),
        dict(good, dt=float("inf")), dict(good, steps=-1), dict(good, steps=2**32), dict(good, stride=0),
        dict(good, precision=7), dict(good, ckpt_every=-1), dict(good, m=7), dict(good, d=3),
        dict(good, model=99), dict(good, model="fhn_net", n=7), dict(good, orbit_offset=2**32 - 8),
    ]
    for kw in bad:
        assert _status(L, sdeb.Problem.make(**kw)) == sdeb.SDEB_EINVAL, kw
        assert sdeb.sdeb_last_error()
    pb = sdeb.Problem.make(**good)
    pb.flags = 0x80
    assert _status(L, pb) == sdeb.SDEB_EINVAL
    # at most one step scheme: Milstein, RK4, implicit Euler, implicit midpoint
    for flags in (sdeb.SDEB_FLAG_MILSTEIN | sdeb.SDEB_FLAG_RK4,
                  sdeb.SDEB_FLAG_RK4 | sdeb.SDEB_FLAG_IMPLICIT_EULER,
                  sdeb.SDEB_FLAG_MILSTEIN | sdeb.SDEB_FLAG_IMPLICIT_MIDPOINT,
                  sdeb.SDEB_FLAG_IMPLICIT_EULER | sdeb.SDEB_FLAG_IMPLICIT_MIDPOINT):
        pb = sdeb.Problem.make(**good)
        pb.flags = flags
        assert _status(L, pb) == sdeb.SDEB_EINVAL, flags
    pb = sdeb.Problem.make(**good)
    pb.reserved = 1
    assert _status(L, pb) == sdeb.SDEB_EINVAL
    assert _status(L, sdeb.Problem.make(**dict(good, n=300))) == sdeb.SDEB_EUNSUPPORTED
    assert L.sdeb_create(None, None) == sdeb.SDEB_EINVAL


def test_null_arguments_are_errors(L):
    assert L.sdeb_set_params(None, None, None, 0, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_integrate(None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_integrate_range(None, 0, 1, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_read_orbits(None, None, 0, 0, 0, 0, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_read_final(None, None, 0, 0, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_grad(None, None, None, None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_orbit_flags(None, None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_philox_fill(0, 0, -1, 0, 1, 0, 1, 0, None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_philox_fill(0, 0, 1, 0, 1, 0, 1, 0, None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_normals_fill(0, 0, 1, 0, 1, 4, 5, None, None) == sdeb.SDEB_EINVAL
    assert L.sdeb_order_param(None, 1, 0, 0, None, None, None) == sdeb.SDEB_EINVAL
    L.sdeb_destroy(None)
    for s in range(8):
        assert sdeb.sdeb_status_string(s)


def test_valid_problem_without_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st = _status(L, sdeb.Problem.make("kuramoto", 8, 16, 0.01, 100, 10))
    assert st == sdeb.SDEB_ECUDA
    # the stand-alone kernels fail the same way instead of falling back to the CPU
    assert L.sdeb_philox_fill(0, 0, 1, 0, 1, 0, 1, 0, ctypes.c_void_p(16), None) == sdeb.SDEB_ECUDA


def test_binding_raises_on_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(sdeb, "_lib", None)
    monkeypatch.setattr(sdeb, "library_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        sdeb.lib()
