"""GPU ensemble moments of the stored frames (sdeb_frame_moments): the mean
and population variance over orbits of every state component and of the
order parameter r of Eq. 7 (Sec. 2.3), accumulated in FP64 on the GPU.

* Against the oracle's moments of the oracle's own trajectories: Kuramoto
  n = 32 with 4133 orbits (two chunks, the second ragged) to t = 10 and the
  benchmark's 2^18 orbits to t = 2: FP64 path <= 1e-12, FP32 path <= 1e-6
  for r's mean and variance and <= 1e-5 for the state's.
* Against the oracle's moments of the GPU's own frames: the reduction alone,
  <= 1e-13 (FP32 r: 1e-6, its sines and cosines come from the SFU).
* The benchmark's n = 32 problem at full size (2^18 orbits, 10^4 steps): the
  FP32 moments track the FP64 ones -- r's mean and standard deviation to
  1e-6 up to t = 10 and 1e-5 over the horizon.
* Components beyond one pass of 256 threads (a FitzHugh-Nagumo network of
  256 units, n = 512), one orbit, frame subranges that give the bits of the
  whole range, host and device outputs alike, and the error statuses.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import NTHREADS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _rel(x, ref):
    x, ref = np.asarray(x, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)))


def _gpu_run(model, n, p, x0, dt, steps, stride, precision, seed=0, frames=True):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    dt_t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make(model, n, x0.shape[0], dt, steps, stride, seed, precision)
    it = Integrator(pb)
    it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
    it.integrate()
    fr = it.frames().cpu().numpy().astype(np.float64) if frames else None
    return it, fr


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("orbits,steps", [(4133, 2000), (1 << 18, 400)])
def test_moments_match_the_oracle(precision, orbits, steps):
    n, dt, stride = 32, 0.005, 100
    p, x0 = inputs.kuramoto(n, orbits, seed=12)
    p, x0 = p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64)
    it, fr = _gpu_run("kuramoto", n, p, x0, dt, steps, stride, precision)
    with it:
        mom, rmom = [t.cpu().numpy() for t in it.moments(order_param=True)]
    pb = oracle.make_problem("kuramoto", n, n, n + 2, dt, steps, stride, 0, mean_field=True)
    ofr, _ = oracle.integrate(pb, p, x0, nthreads=NTHREADS)
    omom, ormom = oracle.frame_moments(ofr, order_parameter=True)
    e_state, e_r = _rel(mom, omom), _rel(rmom, ormom)
    # the reduction alone: the oracle's moments of the GPU's frames
    gmom, grmom = oracle.frame_moments(fr, order_parameter=True)
    e_red, e_red_r = _rel(mom, gmom), _rel(rmom, grmom)
    print("%s orbits=%d: vs oracle state %.1e r %.1e; reduction state %.1e r %.1e" % (
        precision, orbits, e_state, e_r, e_red, e_red_r))
    assert e_red < 1e-13
    if precision == "fp64":
        assert e_red_r < 1e-13
        assert e_state < 1e-12 and e_r < 1e-12
    else:
        assert e_red_r < 1e-6
        assert e_state < 1e-5 and e_r < 1e-6


def test_moments_full_size_fp32_tracks_fp64():
    W = inputs.WORKLOADS["kuramoto_n32"]
    n, orbits = 32, 1 << 18
    p, x0 = inputs.kuramoto(n, orbits, seed=1)
    p, x0 = p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64)
    res = {}
    for precision in ("fp64", "fp32"):
        it, _ = _gpu_run("kuramoto", n, p, x0, W["dt"], W["steps"], W["stride"], precision, frames=False)
        with it:
            res[precision] = [t.cpu().numpy() for t in it.moments(order_param=True)]
            # the reduction against the oracle's definition on a few frames of the GPU's own frames
            for f in (0, 20, 100):
                fr = it.frames(begin=f, count=1).cpu().numpy()
                gm, gr = oracle.frame_moments(fr, order_parameter=True)
                assert _rel(res[precision][0][f:f + 1], gm) < 1e-13, (precision, f)
                assert _rel(res[precision][1][f:f + 1], gr) < (1e-13 if precision == "fp64" else 1e-6), (precision, f)
    r64, r32 = res["fp64"][1], res["fp32"][1]
    d_mean = np.abs(r32[:, 0] - r64[:, 0])
    d_sd = np.abs(np.sqrt(r32[:, 1]) - np.sqrt(r64[:, 1]))
    h = 21                                                   # frames up to t = 10
    print("full size <r>: fp32-fp64 up to t=10 %.1e, over the horizon %.1e; sd(r) %.1e / %.1e" % (
        d_mean[:h].max(), d_mean.max(), d_sd[:h].max(), d_sd.max()))
    assert d_mean[:h].max() < 1e-6 and d_sd[:h].max() < 1e-6
    assert d_mean.max() < 1e-5 and d_sd.max() < 1e-5


def test_moments_many_components_one_orbit_subranges_and_host_output():
    import torch
    # FitzHugh-Nagumo network of 256 units: n = 512 state components
    units, orbits = 256, 300
    p, x0 = inputs.fhn(units, orbits, seed=9)
    it, fr = _gpu_run("fhn_net", 2 * units, p, x0, 0.01, 300, 50, "fp64", seed=4)
    with it:
        mom, _ = it.moments()
        np.testing.assert_allclose(mom.cpu().numpy(), oracle.frame_moments(fr)[0], rtol=1e-13, atol=1e-13)
        with pytest.raises(sdeb.SdebError) as e:
            it.moments(order_param=True)
        assert e.value.status == sdeb.SDEB_EUNSUPPORTED
    # one orbit: mean = the state, variance 0
    p1, x1 = inputs.kuramoto(8, 1, seed=3)
    it, fr = _gpu_run("kuramoto", 8, p1, x1, 0.01, 200, 10, "fp32")
    with it:
        mom, rmom = [t.cpu().numpy() for t in it.moments(order_param=True)]
        np.testing.assert_array_equal(mom[:, :, 0], fr[:, 0, :])
        np.testing.assert_array_equal(mom[:, :, 1], 0.0)
        np.testing.assert_array_equal(rmom[:, 1], 0.0)
    # subranges give the bits of the whole range; host output equals device output
    p, x0 = inputs.kuramoto(16, 9000, seed=5)
    it, _ = _gpu_run("kuramoto", 16, p, x0, 0.01, 1000, 20, "fp64", frames=False)
    with it:
        whole = [t.cpu().numpy() for t in it.moments(order_param=True)]
        part = [t.cpu().numpy() for t in it.moments(begin=17, count=9, order_param=True)]
        host = [t.numpy() for t in it.moments(order_param=True, device="cpu")]
        again = [t.cpu().numpy() for t in it.moments(order_param=True)]
        for a, b, c, d in zip(whole, part, host, again):
            np.testing.assert_array_equal(a[17:26], b)
            np.testing.assert_array_equal(a, c)
            np.testing.assert_array_equal(a, d)


def test_moments_errors():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 8, 64
    p, x0 = inputs.kuramoto(n, orbits, seed=2)
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 100, 10, 0, "fp64")
    with Integrator(pb) as it:
        with pytest.raises(sdeb.SdebError) as e:
            it.moments()                                  # before set_params
        assert e.value.status == sdeb.SDEB_ESTATE
        it.set_params(torch.tensor(p).cuda(), torch.tensor(x0).cuda())
        it.integrate_range(0, 50)
        with pytest.raises(sdeb.SdebError) as e:
            it.moments(begin=0, count=7)                  # frame 6 = step 60 is past step 50
        assert e.value.status == sdeb.SDEB_ESTATE
        it.moments(begin=0, count=6)
        with pytest.raises(sdeb.SdebError) as e:
            it.moments(begin=5, count=7)                  # outside [0, 11)
        assert e.value.status == sdeb.SDEB_EINVAL
        buf = torch.empty((2, n, 2), dtype=torch.float64, device="cuda")
        st = sdeb.lib().sdeb_frame_moments(it.ctx, 0, 2, ctypes.c_void_p(buf.data_ptr()), buf.numel() * 8 - 8,
                                           None, 0, sdeb.SDEB_MEM_DEVICE, None)
        assert st == sdeb.SDEB_EINVAL                     # wrong size
        st = sdeb.lib().sdeb_frame_moments(it.ctx, 0, 2, None, 0, None, 0, sdeb.SDEB_MEM_DEVICE, None)
        assert st == sdeb.SDEB_EINVAL                     # nothing asked for
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 100, 10, 0, "fp64", no_frames=True)
    with Integrator(pb) as it:
        it.set_params(torch.tensor(p).cuda(), torch.tensor(x0).cuda())
        it.integrate()
        with pytest.raises(sdeb.SdebError) as e:
            it.moments(count=1)
        assert e.value.status == sdeb.SDEB_ESTATE
