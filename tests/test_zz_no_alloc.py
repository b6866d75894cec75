"""The allocation-free entry point sdeb_integrate_noalloc.

It exists for callers that cannot allocate device memory (graph capture,
host-owned allocators, real-time hosts): they pass every input and output
buffer, and the library keeps its only scratch in a fixed array of its own.
These tests call it through the C ABI twice in a row -- the shared scratch
keeps the previous call's contents, so the second call checks that what must
start at zero is cleared -- and compare each result with the context API's
(sdeb_create / sdeb_set_params / sdeb_integrate at the layout sdeb_create
picks).  Both run the same kernel at the same layout, so frames and final
states must be identical bit for bit: a compensation word left over from the
previous call would move a state by one rounding, which a tolerance check
could miss.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import np_dtype, run_gpu

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _noalloc(pb, p, x0, with_frames=True):
    import torch
    dt = torch.float64 if pb.precision == sdeb.SDEB_FP64 else torch.float32
    pt = torch.tensor(p, dtype=dt, device="cuda")
    xt = torch.tensor(x0, dtype=dt, device="cuda")
    xf = torch.empty_like(xt)
    fr = torch.empty((pb.steps // pb.stride + 1, pb.orbits, pb.n), dtype=dt, device="cuda") if with_frames else None
    sdeb.sdeb_integrate_noalloc(pb, ctypes.c_void_p(pt.data_ptr()), ctypes.c_void_p(xt.data_ptr()),
                                ctypes.c_void_p(xf.data_ptr()),
                                ctypes.c_void_p(fr.data_ptr()) if fr is not None else None,
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return (fr.cpu().numpy() if fr is not None else None), xf.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_context_api_twice(precision):
    n, orbits, dt, steps, stride, seed = 32, 4099, 0.01, 600, 50, 3
    p, x0 = inputs.kuramoto(n, orbits, seed=21)
    p, x0 = p.astype(np_dtype(precision)), x0.astype(np_dtype(precision))
    ref_fr, ref_fin = run_gpu("kuramoto", n, p, x0, dt, steps, stride, seed=seed, precision=precision)
    pb = sdeb.Problem.make("kuramoto", n, orbits, dt, steps, stride, seed, precision)
    for _ in range(2):
        fr, fin = _noalloc(pb, p, x0)
        np.testing.assert_array_equal(fr, ref_fr)
        np.testing.assert_array_equal(fin, ref_fin)


def test_noalloc_other_model_without_frames():
    n, orbits, dt, steps = 128, 1000, 0.01, 300
    p, x0 = inputs.fhn(n // 2, orbits, seed=4)
    p, x0 = p.astype(np.float32), x0.astype(np.float32)
    _, ref_fin = run_gpu("fhn_net", n, p, x0, dt, steps, 10, seed=1, precision="fp32")
    pb = sdeb.Problem.make("fhn_net", n, orbits, dt, steps, 10, 1, "fp32")
    for _ in range(2):
        _, fin = _noalloc(pb, p, x0, with_frames=False)
        np.testing.assert_array_equal(fin, ref_fin)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", [dict(rk4=True), dict(implicit="euler"), dict(implicit="midpoint"),
                                    dict(milstein=True)])
def test_noalloc_step_schemes_match_the_context_api(scheme, precision):
    """The scheme flags reach the same kernels through this entry point."""
    model = "gbm" if "milstein" in scheme else "kuramoto"
    n, orbits, dt, steps, stride = (8, 700, 0.01, 200, 20)
    if model == "gbm":
        p, x0 = inputs.scalar_model(n, orbits, [0.3, 0.3], 0.5, 1.5, seed=5)
    else:
        p, x0 = inputs.kuramoto(n, orbits, seed=6)
    p, x0 = p.astype(np_dtype(precision)), x0.astype(np_dtype(precision))
    ref_fr, ref_fin = run_gpu(model, n, p, x0, dt, steps, stride, seed=2, precision=precision, **scheme)
    pb = sdeb.Problem.make(model, n, orbits, dt, steps, stride, 2, precision, **scheme)
    for _ in range(2):
        fr, fin = _noalloc(pb, p, x0)
        np.testing.assert_array_equal(fr, ref_fr)
        np.testing.assert_array_equal(fin, ref_fin)


def test_noalloc_rejects_sizes_beyond_its_limit():
    L = sdeb.lib()
    pb = sdeb.Problem.make("kuramoto", 8, 16, 0.01, 10, 10, 0, "fp32", rk4=True)
    pb.flags |= sdeb.SDEB_FLAG_IMPLICIT_EULER                   # two step schemes
    st = L.sdeb_integrate_noalloc(ctypes.byref(pb), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None, None)
    assert st == sdeb.SDEB_EINVAL
    n = 64
    orbits = (1 << 21) // n + 1        # one orbit past the scratch limit
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 10, 10, 0, "fp32")
    st = L.sdeb_integrate_noalloc(ctypes.byref(pb), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None, None)
    assert st == sdeb.SDEB_EINVAL
    assert "limit" in sdeb.sdeb_last_error()
    pb = sdeb.Problem.make("kuramoto", n, 16, 0.01, 10, 10, 0, "fp32", ckpt_every=5)
    st = L.sdeb_integrate_noalloc(ctypes.byref(pb), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None, None)
    assert st == sdeb.SDEB_EUNSUPPORTED
