"""GPU parity of the Milstein step (SDEB_FLAG_MILSTEIN; the scheme the paper
names as the next integrator, Sec. 2.1 and Sec. 3) against the oracle's
pinned Milstein step on the same inputs and the same Philox noise.

* GBM (g = sigma x) and the FitzHugh-Nagumo network (g = sigma v on v):
  FP64 <= 1e-12 and FP32 <= 1e-4 over the stated horizons, in several
  lane-group layouts, frames and final state.
* The Milstein result differs from Euler-Maruyama on these models (the
  correction is really applied), and on the additive-noise models (Kuramoto,
  OU) the flag changes nothing, bit for bit.
* Resume over step ranges is bit-exact under Milstein as under
  Euler-Maruyama."""
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
    if model == "gbm":
        rng = np.random.Generator(np.random.PCG64(21))
        p = np.stack([rng.uniform(-0.5, 0.5, orbits), rng.uniform(0.1, 0.6, orbits)], axis=1)
        x0 = rng.uniform(0.5, 2.0, (orbits, n))
        return p, x0
    return inputs.fhn(n // 2, orbits, seed=22)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n,layouts", [("gbm", 4, [None, (1, 8)]), ("gbm", 24, [None, (8, 8)]),
                                             ("fhn_net", 32, [None, (4, 8)]), ("fhn_net", 128, [None, (16, 8)])])
def test_milstein_matches_oracle(precision, model, n, layouts):
    orbits, steps, stride, dt = 300, 400, 50, 0.01
    p, x0 = _cast(precision, *_inputs(model, n, orbits))
    rfr, rfin = run_oracle(model, n, p, x0, dt, steps, stride, seed=4, orbit_offset=9, milstein=True)
    efr, _ = run_oracle(model, n, p, x0, dt, steps, stride, seed=4, orbit_offset=9, milstein=False)
    assert max_rel_err(efr, rfr) > 1e-6            # the correction is not negligible here
    for lay in layouts:
        fr, fin = run_gpu(model, n, p, x0, dt, steps, stride, seed=4, precision=precision, orbit_offset=9,
                          milstein=True, layout=lay)
        assert max_rel_err(fr, rfr) < TOL[precision], lay
        assert max_rel_err(fin, rfin) < TOL[precision], lay


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n", [("kuramoto", 32), ("ou", 6), ("kuramoto_paper", 8)])
def test_additive_noise_flag_changes_nothing(precision, model, n):
    orbits, steps, stride = 200, 300, 30
    if model == "kuramoto":
        p, x0 = inputs.kuramoto(n, orbits, seed=23)
    elif model == "kuramoto_paper":
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=24)
    else:
        p, x0 = inputs.scalar_model(n, orbits, [0.7, 0.4], -1, 1, seed=25)
    p, x0 = _cast(precision, p, x0)
    a = run_gpu(model, n, p, x0, 0.01, steps, stride, seed=6, precision=precision)
    b = run_gpu(model, n, p, x0, 0.01, steps, stride, seed=6, precision=precision, milstein=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_milstein_resume_is_bit_exact(precision):
    n, orbits, steps, stride = 32, 200, 500, 25
    p, x0 = _cast(precision, *inputs.fhn(n // 2, orbits, seed=26))
    fr, fin = run_gpu("fhn_net", n, p, x0, 0.01, steps, stride, precision=precision, milstein=True)
    fr2, fin2 = run_gpu("fhn_net", n, p, x0, 0.01, steps, stride, precision=precision, milstein=True,
                        ranges=[(0, 137), (137, 138), (138, 400), (400, 500)])
    np.testing.assert_array_equal(fr, fr2)
    np.testing.assert_array_equal(fin, fin2)
