"""GPU parity of the ODE path (SDEB_FLAG_RK4: classical fourth-order
Runge-Kutta on the drift alone; the paper lists Runge-Kutta among its ODE
integrators, Sec. 1.5) against the oracle's pinned RK4 step.

* Every model: FP64 <= 1e-12 over 400 steps and FP32 <= 1e-4 over 200 steps
  of dt = 0.01 (frames and final state).  Without noise the n = 128
  Kuramoto orbits are chaotic enough that the FP64 oracle itself, with x0
  perturbed by 2^-24 relative (one FP32 rounding), departs by 2.6e-6 at
  t = 1.5, 6.4e-6 at t = 2 and 1.7e-4 at t = 3: the FP32 horizon is t <= 2
  (pinned in test_oracle_sensitivity.py).
* No noise: Kuramoto with sigma > 0 gives the bits of sigma = 0.
* Resume over step ranges is bit-exact.
* Errors: a tuner-only layout (EUNSUPPORTED at integration), RK4 with
  Milstein (EINVAL), sdeb_grad on an RK4 context and an RK4 instance in a
  batch (EUNSUPPORTED)."""
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
    return [np.asarray(a).astype(t).astype(np.float64) for a in arrays]


def _inputs(model, n, orbits):
    if model == "kuramoto":
        return inputs.kuramoto(n, orbits, seed=31)
    if model == "kuramoto_paper":
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=32)
        p[:, 0] = 2.0
        return p, x0
    if model == "fhn_net":
        return inputs.fhn(n // 2, orbits, seed=33)
    if model == "ou":
        return inputs.scalar_model(n, orbits, [0.7, 0.4], -1, 1, seed=34)
    if model == "gbm":
        return inputs.scalar_model(n, orbits, [0.3, 0.3], 0.5, 1.5, seed=35)
    return inputs.scalar_model(n, orbits, [0.9], -2, 2, seed=36)


def _rk4(model, n, p, x0, precision, dt=0.01, steps=400, stride=50, **kw):
    return run_gpu(model, n, p, x0, dt, steps, stride, seed=2, precision=precision, orbit_offset=3, rk4=True,
                   **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n", [("kuramoto", 8), ("kuramoto", 32), ("kuramoto", 128), ("kuramoto_paper", 12),
                                     ("fhn_net", 32), ("ou", 5), ("gbm", 3), ("linear_ode", 4)])
def test_rk4_matches_oracle(precision, model, n):
    orbits = 200
    steps = 400 if precision == "fp64" else 200
    p, x0 = _cast(precision, *_inputs(model, n, orbits))
    fr, fin = _rk4(model, n, p, x0, precision, steps=steps)
    rfr, rfin = run_oracle(model, n, p, x0, 0.01, steps, 50, seed=2, orbit_offset=3, rk4=True)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rk4_applies_no_noise_and_resumes_bit_exactly(precision):
    n, orbits = 32, 150
    p, x0 = _cast(precision, *inputs.kuramoto(n, orbits, seed=37))
    p0 = p.copy()
    p0[:, 1] = 0.0
    a = _rk4("kuramoto", n, p, x0, precision)
    b = _rk4("kuramoto", n, p0, x0, precision)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    c = _rk4("kuramoto", n, p, x0, precision, ranges=[(0, 99), (99, 250), (250, 400)])
    np.testing.assert_array_equal(a[0], c[0])
    np.testing.assert_array_equal(a[1], c[1])


def test_rk4_errors():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 32, 64
    p, x0 = inputs.kuramoto(n, orbits, seed=38)
    pt, xt = torch.tensor(p, dtype=torch.float32).cuda(), torch.tensor(x0, dtype=torch.float32).cuda()
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 50, 10, 1, "fp32", rk4=True, ckpt_every=10)
    with Integrator(pb) as it:
        it.set_params(pt, xt)
        it.set_layout(8, 4)                     # a layout only the layout tuner instantiates
        with pytest.raises(sdeb.SdebError) as e:
            it.integrate()
        assert e.value.status == sdeb.SDEB_EUNSUPPORTED
        it.set_layout(4, 8)
        it.set_params(pt, xt)
        it.integrate()
        with pytest.raises(sdeb.SdebError) as e:
            it.grad(torch.zeros(orbits, n, device="cuda"))
        assert e.value.status == sdeb.SDEB_EUNSUPPORTED
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create(sdeb.Problem.make("gbm", 2, 4, 0.01, 10, 1, 1, "fp32", rk4=True, milstein=True))
    assert e.value.status == sdeb.SDEB_EINVAL
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create_batch([sdeb.Problem.make("kuramoto", 8, 1, 0.01, 10, 1, 1, "fp32", rk4=True)])
    assert e.value.status == sdeb.SDEB_EUNSUPPORTED
