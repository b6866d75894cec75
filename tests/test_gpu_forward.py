"""GPU parity of the forward Euler-Maruyama path against the CPU oracle.

Tolerances (max |x - x_ref| / max(|x_ref|, 1) over orbits, frames, states):
FP64 path 1e-12, FP32 Kahan path 1e-4, against the FP64 oracle.
"""
import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import max_rel_err, np_dtype, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _cast(precision, *arrays):
    t = np_dtype(precision)
    return [np.asarray(a).astype(t) for a in arrays]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kuramoto_n4_1024_orbits(precision):
    # 1024 orbits, n = 4, dt = 0.01, 1000 steps, a frame every 10 steps
    p, x0 = _cast(precision, *inputs.kuramoto(4, 1024, seed=1))
    fr, fin = run_gpu("kuramoto", 4, p, x0, 0.01, 1000, 10, seed=0, precision=precision)
    rfr, rfin = run_oracle("kuramoto", 4, p, x0, 0.01, 1000, 10, seed=0)
    assert fr.shape == (101, 1024, 4)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 9, 16, 17, 31, 32, 33, 64, 65, 100, 128, 129, 200, 256])
def test_kuramoto_all_layouts_ragged(precision, n):
    # every lane-group layout, ragged unit counts and orbit counts, a non-zero
    # global orbit offset
    orbits, steps, stride = 37, 150, 50
    p, x0 = _cast(precision, *inputs.kuramoto(n, orbits, seed=n))
    fr, fin = run_gpu("kuramoto", n, p, x0, 0.01, steps, stride, seed=5, precision=precision, orbit_offset=1000)
    rfr, rfin = run_oracle("kuramoto", n, p, x0, 0.01, steps, stride, seed=5, orbit_offset=1000,
                           mean_field=n > 64)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n", [("kuramoto_paper", 12), ("fhn_net", 128), ("fhn_net", 6), ("ou", 5),
                                     ("gbm", 3), ("linear_ode", 4)])
def test_other_models(precision, model, n):
    orbits, steps, stride, dt = 45, 400, 100, 0.01
    if model == "kuramoto_paper":
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=2)
        p[:, 0] = 2.5
        p[:, n + 1:] = 0.3
    elif model == "fhn_net":
        p, x0 = inputs.fhn(n // 2, orbits, seed=3)
    elif model == "ou":
        p, x0 = inputs.scalar_model(n, orbits, [0.7, 0.4], -1, 1, seed=4)
    elif model == "gbm":
        p, x0 = inputs.scalar_model(n, orbits, [0.1, 0.3], 0.5, 1.5, seed=5)
    else:
        p, x0 = inputs.scalar_model(n, orbits, [0.9], -2, 2, seed=6)
    p, x0 = _cast(precision, p, x0)
    fr, fin = run_gpu(model, n, p, x0, dt, steps, stride, seed=9, precision=precision)
    rfr, rfin = run_oracle(model, n, p, x0, dt, steps, stride, seed=9)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_is_bit_exact(precision):
    n, orbits, steps, stride = 32, 300, 500, 25
    p, x0 = _cast(precision, *inputs.kuramoto(n, orbits, seed=8))
    fr, fin = run_gpu("kuramoto", n, p, x0, 0.01, steps, stride, precision=precision)
    fr2, fin2 = run_gpu("kuramoto", n, p, x0, 0.01, steps, stride, precision=precision,
                        ranges=[(0, 137), (137, 138), (138, 400), (400, 500)])
    np.testing.assert_array_equal(fr, fr2)
    np.testing.assert_array_equal(fin, fin2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shared_params_and_no_frames(precision):
    n, orbits, steps = 8, 50, 200
    p, x0 = inputs.kuramoto(n, orbits, seed=3, shared=True)
    p, x0 = _cast(precision, p, x0)
    _, fin = run_gpu("kuramoto", n, p, x0, 0.01, steps, 1, precision=precision, shared=True, no_frames=True)
    _, rfin = run_oracle("kuramoto", n, p, x0, 0.01, steps, 1, shared=True)
    assert max_rel_err(fin, rfin) < TOL[precision]


def test_zero_steps_and_long_stride():
    p, x0 = inputs.kuramoto(4, 10, seed=1)
    fr, fin = run_gpu("kuramoto", 4, p, x0, 0.01, 0, 5)
    np.testing.assert_array_equal(fr[0], x0)
    np.testing.assert_array_equal(fin, x0)
    fr, fin = run_gpu("kuramoto", 4, p, x0, 0.01, 30, 1000)
    assert fr.shape[0] == 1
    np.testing.assert_array_equal(fr[0], x0)
    _, rfin = run_oracle("kuramoto", 4, p, x0, 0.01, 30, 1000)
    assert max_rel_err(fin, rfin) < 1e-12


def test_call_order_and_read_errors():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    pb = sdeb.Problem.make("kuramoto", 4, 8, 0.01, 100, 10, precision="fp64")
    with Integrator(pb) as it:
        with pytest.raises(sdeb.SdebError) as e:
            it.integrate()
        assert e.value.status == sdeb.SDEB_ESTATE
        p, x0 = inputs.kuramoto(4, 8, seed=1)
        it.set_params(torch.tensor(p), torch.tensor(x0))  # host tensors
        it.integrate_range(0, 50)
        with pytest.raises(sdeb.SdebError) as e:
            it.frames(0, 7)  # frame 6 is at step 60 > 50
        assert e.value.status == sdeb.SDEB_ESTATE
        with pytest.raises(sdeb.SdebError) as e:
            it.integrate_range(40, 60)
        assert e.value.status == sdeb.SDEB_ESTATE
        it.frames(0, 6)
        it.integrate_range(50, 100)
        with pytest.raises(sdeb.SdebError) as e:
            it.integrate()
        assert e.value.status == sdeb.SDEB_ESTATE
        out = torch.empty((2, 8, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(sdeb.SdebError) as e:
            sdeb.sdeb_read_orbits(it.ctx, out.data_ptr(), out.numel() * 8 - 8, 0, 2, 1)
        assert e.value.status == sdeb.SDEB_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_flag(precision):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    # dx = -theta x dt with theta = -1e30: |x| overflows within a few steps;
    # the second orbit (theta = 0.5) stays finite
    p = np.array([[-1e30], [0.5]])
    x0 = np.ones((2, 3))
    pb = sdeb.Problem.make("linear_ode", 3, 2, 1.0, 40, 10, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    with Integrator(pb) as it:
        it.set_params(torch.tensor(p, dtype=dt).cuda(), torch.tensor(x0, dtype=dt).cuda())
        it.integrate()
        flags = it.flags().numpy()
    assert flags.tolist() == [1, 0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_layouts_and_autotune(precision):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits, steps, stride = 32, 301, 200, 50
    p, x0 = _cast(precision, *inputs.kuramoto(n, orbits, seed=31))
    rfr, _ = run_oracle("kuramoto", n, p, x0, 0.01, steps, stride, seed=2)
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    pt, xt = torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda()
    for layout in [(4, 8), (8, 4), (2, 16), (16, 4), (4, 16), (32, 4)]:
        pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, steps, stride, 2, precision)
        with Integrator(pb) as it:
            if layout == (2, 16):
                with pytest.raises(sdeb.SdebError) as e:      # no kernel for this layout
                    it.set_layout(*layout)
                assert e.value.status == sdeb.SDEB_EUNSUPPORTED
                continue
            it.set_layout(*layout)
            assert it.layout() == layout
            it.set_params(pt, xt)
            it.integrate()
            assert max_rel_err(it.frames().cpu().numpy(), rfr) < TOL[precision]
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, steps, stride, 2, precision)
    with Integrator(pb) as it:
        with pytest.raises(sdeb.SdebError) as e:
            it.set_layout(2, 8)                               # 16 units < 32
        assert e.value.status == sdeb.SDEB_EINVAL
        it.set_params(pt, xt)
        chosen = it.autotune(trial_steps=32)
        assert chosen[0] * chosen[1] >= n
        it.integrate()
        assert max_rel_err(it.frames().cpu().numpy(), rfr) < TOL[precision]
        with pytest.raises(sdeb.SdebError) as e:
            it.autotune()
        assert e.value.status == sdeb.SDEB_ESTATE
