"""GPU parity of the implicit ODE schemes (SDEB_FLAG_IMPLICIT_EULER and
SDEB_FLAG_IMPLICIT_MIDPOINT: implicit Euler and the implicit midpoint rule on
the drift alone, the paper's ODE integrators of Sec. 1.5) against the
oracle's pinned implicit step: 4 Newton iterations from the old state, a
dense LU solve in the oracle, the closed-form structured solve of each model
(Woodbury for the Kuramoto models, block Sherman-Morrison for the
FitzHugh-Nagumo network) on the GPU -- the same Newton iterates, so the two
agree to rounding whether or not Newton has converged.

* Every model, both schemes: FP64 <= 1e-12 over 400 steps and FP32 <= 1e-4
  over 200 steps of dt = 0.01 (frames and final state); the FP32 horizon is
  the one the Runge-Kutta path uses.  The n = 128 Kuramoto orbits without
  noise are chaotic: the FP64 oracle itself, with x0 perturbed by one
  rounding (2^-52 relative), stays below 1e-12 through t = 3 and departs by
  3.8e-12 (midpoint) and 2.9e-11 (Euler) by t = 4, so their FP64 horizon is
  300 steps (pinned in test_oracle_sensitivity.py).
* Large steps (dt = 0.2, K dt up to 0.8 for the Kuramoto orbits): FP64
  <= 1e-12 over a horizon per case, where Newton's later iterates matter:
  30 steps (t = 6) where the oracle itself, with x0 perturbed by one
  rounding, departs past 1e-12 by t = 12 (Kuramoto n = 32 under Euler,
  n = 100 under both schemes), 60 steps where that departure stays below
  1e-13 (Kuramoto n = 32 under the midpoint rule, the FitzHugh-Nagumo
  network); pinned in test_oracle_sensitivity.py (LARGE_STEP_HORIZON).
* Every lane layout that covers an n = 32 orbit gives the oracle's orbit.
* A stiff linear ODE (rate dt = 5): the closed forms (1 + h rate)^-k and
  ((1 - h rate / 2) / (1 + h rate / 2))^k, where Euler-Maruyama diverges.
* No noise is applied; resume over step ranges is bit-exact.
* Errors: the schemes with each other, RK4 or Milstein (EINVAL); sdeb_grad
  and a batch instance (EUNSUPPORTED)."""
import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import max_rel_err, np_dtype, run_gpu, run_oracle
from test_oracle_sensitivity import LARGE_STEP_HORIZON

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-4}
SCHEMES = ["euler", "midpoint"]


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
        return inputs.kuramoto(n, orbits, seed=41)
    if model == "kuramoto_paper":
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=42)
        p[:, 0] = 2.0
        return p, x0
    if model == "fhn_net":
        return inputs.fhn(n // 2, orbits, seed=43)
    if model == "ou":
        return inputs.scalar_model(n, orbits, [0.7, 0.4], -1, 1, seed=44)
    if model == "gbm":
        return inputs.scalar_model(n, orbits, [0.3, 0.3], 0.5, 1.5, seed=45)
    return inputs.scalar_model(n, orbits, [0.9], -2, 2, seed=46)


def _implicit(scheme, model, n, p, x0, precision, dt=0.01, steps=400, stride=50, **kw):
    return run_gpu(model, n, p, x0, dt, steps, stride, seed=2, precision=precision, orbit_offset=3,
                   implicit=scheme, **kw)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n", [("kuramoto", 8), ("kuramoto", 32), ("kuramoto", 128), ("kuramoto_paper", 12),
                                     ("fhn_net", 32), ("ou", 5), ("gbm", 3), ("linear_ode", 4)])
def test_implicit_matches_oracle(scheme, precision, model, n):
    orbits = 200
    steps = (300 if n == 128 else 400) if precision == "fp64" else 200
    p, x0 = _cast(precision, *_inputs(model, n, orbits))
    fr, fin = _implicit(scheme, model, n, p, x0, precision, steps=steps)
    rfr, rfin = run_oracle(model, n, p, x0, 0.01, steps, 50, seed=2, orbit_offset=3, implicit=scheme)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("model,n", [("kuramoto", 32), ("kuramoto", 100), ("fhn_net", 64)])
def test_implicit_large_steps_match_oracle(scheme, model, n):
    orbits = 128
    p, x0 = _inputs(model, n, orbits)
    if model == "kuramoto":
        p[:, 0] = np.linspace(0.0, 4.0, orbits)     # K dt up to 0.8
    steps = LARGE_STEP_HORIZON[(model, n, scheme)]
    fr, fin = _implicit(scheme, model, n, p, x0, "fp64", dt=0.2, steps=steps, stride=10)
    rfr, rfin = run_oracle(model, n, p, x0, 0.2, steps, 10, seed=2, orbit_offset=3, implicit=scheme)
    assert max_rel_err(fr, rfr) < 1e-12
    assert max_rel_err(fin, rfin) < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("layout", [(4, 8), (8, 8), (16, 8), (32, 8)])
def test_implicit_every_layout_matches_oracle(scheme, layout):
    n, orbits = 32, 96
    p, x0 = inputs.kuramoto(n, orbits, seed=47)
    fr, fin = _implicit(scheme, "kuramoto", n, p, x0, "fp64", steps=300, layout=layout)
    rfr, rfin = run_oracle("kuramoto", n, p, x0, 0.01, 300, 50, seed=2, orbit_offset=3, implicit=scheme)
    assert max_rel_err(fr, rfr) < 1e-12
    assert max_rel_err(fin, rfin) < 1e-12


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_implicit_stiff_linear_ode_closed_form(precision, rtol):
    n, orbits, rate, dt, steps = 4, 64, 50.0, 0.1, 20
    p, x0 = _cast(precision, *inputs.scalar_model(n, orbits, [rate], -2, 2, seed=48))
    h = dt * rate
    factors = {"euler": 1.0 / (1.0 + h), "midpoint": (1.0 - 0.5 * h) / (1.0 + 0.5 * h)}
    for scheme, f in factors.items():
        fr, fin = _implicit(scheme, "linear_ode", n, p, x0, precision, dt=dt, steps=steps, stride=1)
        k = np.arange(steps + 1, dtype=np.float64)[:, None, None]
        expect = x0[None, :, :] * f ** k
        np.testing.assert_allclose(fr, expect, rtol=rtol, atol=0.0)
        np.testing.assert_allclose(fin, expect[-1], rtol=rtol, atol=0.0)
    # the explicit step on the same problem grows like |1 - h|^k = 4^k
    _, em = run_gpu("linear_ode", n, p, x0, dt, steps, steps, precision=precision)
    assert np.all(np.abs(em) > 1e10 * np.abs(x0))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_implicit_applies_no_noise_and_resumes_bit_exactly(precision):
    n, orbits = 32, 150
    p, x0 = _cast(precision, *inputs.kuramoto(n, orbits, seed=49))
    p0 = p.copy()
    p0[:, 1] = 0.0
    for scheme in SCHEMES:
        a = _implicit(scheme, "kuramoto", n, p, x0, precision)
        b = _implicit(scheme, "kuramoto", n, p0, x0, precision)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        c = _implicit(scheme, "kuramoto", n, p, x0, precision, ranges=[(0, 99), (99, 250), (250, 400)])
        np.testing.assert_array_equal(a[0], c[0])
        np.testing.assert_array_equal(a[1], c[1])


def test_implicit_errors():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 32, 64
    p, x0 = inputs.kuramoto(n, orbits, seed=50)
    pt, xt = torch.tensor(p, dtype=torch.float32).cuda(), torch.tensor(x0, dtype=torch.float32).cuda()
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 50, 10, 1, "fp32", implicit="euler", ckpt_every=10)
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
    for kw in (dict(rk4=True), dict(milstein=True)):
        with pytest.raises(sdeb.SdebError) as e:
            sdeb.sdeb_create(sdeb.Problem.make("gbm", 2, 4, 0.01, 10, 1, 1, "fp32", implicit="midpoint", **kw))
        assert e.value.status == sdeb.SDEB_EINVAL
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_create_batch([sdeb.Problem.make("kuramoto", 8, 1, 0.01, 10, 1, 1, "fp32", implicit="euler")])
    assert e.value.status == sdeb.SDEB_EUNSUPPORTED


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("model,n,orbits,steps", [("kuramoto", 1, 5, 50), ("kuramoto", 2, 1, 50),
                                                  ("kuramoto", 33, 7, 40), ("fhn_net", 2, 3, 50),
                                                  ("kuramoto", 8, 4, 0)])
def test_implicit_edge_shapes(scheme, model, n, orbits, steps):
    """One oscillator (the coupling vanishes), one orbit, a ragged n = 33
    (a lane with one live unit), one FHN unit, and no steps at all."""
    p, x0 = _inputs(model, n, orbits)
    fr, fin = _implicit(scheme, model, n, p, x0, "fp64", steps=steps, stride=10)
    rfr, rfin = run_oracle(model, n, p, x0, 0.01, steps, 10, seed=2, orbit_offset=3, implicit=scheme)
    assert max_rel_err(fr, rfr) < 1e-12
    assert max_rel_err(fin, rfin) < 1e-12
    if steps == 0:
        np.testing.assert_array_equal(fin, x0)
