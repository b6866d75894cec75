"""The copy calls' memory kinds (SDEB_MEM_HOST / _DEVICE / _HOST_ASYNC):
inputs enqueued from page-locked host memory and frames / final states read
into host memory without waiting give the same bits as the waiting copies,
with the horizon run in ranges whose frames are read while the next range
computes on the same stream; any other kind is EINVAL."""
import ctypes

import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_async_host_copies_give_the_waiting_copies_bits(precision):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits, steps, stride = 32, 3000, 400, 10
    p, x0 = inputs.kuramoto(n, orbits, seed=61)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pt, xt = torch.tensor(p, dtype=dt), torch.tensor(x0, dtype=dt)
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, steps, stride, 4, precision)
    with Integrator(pb) as it:
        it.set_params(pt, xt)                               # waiting host copies
        it.integrate()
        ref_frames = it.frames(device="cpu")
        ref_final = it.final(device="cpu")
    s = torch.cuda.Stream()
    ph, xh = pt.pin_memory(), xt.pin_memory()
    frames = torch.empty_like(ref_frames).pin_memory()
    final = torch.empty_like(ref_final).pin_memory()
    with Integrator(pb) as it:
        it.set_params(ph, xh, stream=s, async_host=True)
        done = 0
        for k0, k1 in ((0, 130), (130, 260), (260, 400)):
            it.integrate_range(k0, k1, stream=s)
            f_end = k1 // stride + 1
            it.frames(begin=done, count=f_end - done, out=frames[done:f_end], stream=s, async_host=True)
            done = f_end
        it.final(out=final, stream=s, async_host=True)
        s.synchronize()
    np.testing.assert_array_equal(frames.numpy(), ref_frames.numpy())
    np.testing.assert_array_equal(final.numpy(), ref_final.numpy())


def test_unknown_memory_kind_is_refused():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 8, 16
    p, x0 = inputs.kuramoto(n, orbits, seed=62)
    pt, xt = torch.tensor(p, dtype=torch.float32).cuda(), torch.tensor(x0, dtype=torch.float32).cuda()
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 20, 10, 4, "fp32")
    L = sdeb.lib()
    with Integrator(pb) as it:
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())   # noqa: E731
        assert L.sdeb_set_params(it.ctx, ptr(pt), ptr(xt), 3, None) == sdeb.SDEB_EINVAL
        it.set_params(pt, xt)
        it.integrate()
        out = torch.empty((3, orbits, n), dtype=torch.float32, device="cuda")
        assert L.sdeb_read_orbits(it.ctx, ptr(out), out.numel() * 4, 0, 3, -1, None) == sdeb.SDEB_EINVAL
        fin = torch.empty((orbits, n), dtype=torch.float32, device="cuda")
        assert L.sdeb_read_final(it.ctx, ptr(fin), fin.numel() * 4, 7, None) == sdeb.SDEB_EINVAL
        torch.cuda.synchronize()
