"""GPU parity of user-defined models (sdeb_create_user: the caller's drift
and diffusion compiled at run time with the library's step kernel, the GPU
counterpart of the paper's run-time assembly of the OpenCL source,
Sec. 2.1.3).

* Sources restating GBM, Kuramoto (pairwise, Eq. 6) and the FitzHugh-Nagumo
  network (dense and diagonal noise forms) against the oracle's built-in
  models on the same inputs and noise: FP64 <= 1e-12, FP32 <= 1e-4 (frames
  and final state).
* Dense noise (a 2-state linear SDE driven by 3 Wiener channels) against
  Euler-Maruyama written out in numpy on the oracle's normals: FP64 1e-12.
* The ODE path (SDEB_FLAG_RK4) on the Kuramoto source against the oracle's
  fourth-order Runge-Kutta: FP64 1e-12.
* Resume over step ranges is bit-exact; set_layout and sdeb_grad refuse."""
import math

import numpy as np
import pytest

import oracle
import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

import user_models
from helpers import max_rel_err, np_dtype, run_oracle

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _run_user(source, n, m, d, p, x0, dt, steps, stride, precision, seed=5, orbit_offset=2, ranges=None, rk4=False):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make("user", n, x0.shape[0], dt, steps, stride, seed, precision, m=m, d=d,
                           orbit_offset=orbit_offset, rk4=rk4)
    with Integrator(pb, user_source=source) as it:
        it.set_params(torch.tensor(p, dtype=t).cuda(), torch.tensor(x0, dtype=t).cuda())
        if ranges is None:
            it.integrate()
        else:
            for a, b in ranges:
                it.integrate_range(a, b)
        return it.frames().cpu().numpy(), it.final().cpu().numpy()


def _cast(precision, *arrays):
    t = np_dtype(precision)
    return [np.asarray(a).astype(t).astype(np.float64) for a in arrays]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["gbm", "kuramoto", "fhn_net", "fhn_net_diagonal"])
def test_user_sources_match_the_oracle_models(precision, name):
    orbits, steps, stride, dt = 160, 300, 50, 0.01
    if name == "gbm":
        n, src = 4, user_models.GBM
        p, x0 = inputs.scalar_model(n, orbits, [0.2, 0.4], 0.5, 1.5, seed=41)
    elif name == "kuramoto":
        n, src = 8, user_models.KURAMOTO_PAIRWISE
        p, x0 = inputs.kuramoto(n, orbits, seed=42)
    else:
        n = 16
        src = user_models.FHN if name == "fhn_net" else user_models.FHN_DIAGONAL
        name = "fhn_net"
        p, x0 = inputs.fhn(n // 2, orbits, seed=43)
    m, d = sdeb.model_shape(name, n)
    p, x0 = _cast(precision, p, x0)
    fr, fin = _run_user(src, n, m, d, p, x0, dt, steps, stride, precision)
    rfr, rfin = run_oracle(name, n, p, x0, dt, steps, stride, seed=5, orbit_offset=2)
    assert max_rel_err(fr, rfr) < TOL[precision]
    assert max_rel_err(fin, rfin) < TOL[precision]


def test_dense_noise_against_euler_maruyama_on_the_oracle_normals():
    orbits, steps, stride, dt, seed = 64, 200, 20, 0.01, 9
    rng = np.random.Generator(np.random.PCG64(44))
    A = np.array([[-0.5, 0.3], [-0.2, -0.4]])
    B = rng.uniform(-0.5, 0.5, (2, 3))
    p = np.tile(np.concatenate([A.ravel(), B.ravel()]), (orbits, 1))
    x0 = rng.uniform(-1, 1, (orbits, 2))
    fr, fin = _run_user(user_models.LINEAR_DENSE, 2, 3, 10, p, x0, dt, steps, stride, "fp64", seed=seed,
                        orbit_offset=0)
    N = oracle.normals_fill(seed, 0, steps, 0, orbits, 3)          # [k][o][3]
    x = x0.copy()
    ref = [x.copy()]
    for k in range(steps):
        x = x + (x @ A.T) * dt + math.sqrt(dt) * (N[k] @ B.T)
        if (k + 1) % stride == 0:
            ref.append(x.copy())
    assert max_rel_err(fr, np.stack(ref)) < 1e-12
    assert max_rel_err(fin, x) < 1e-12


def test_user_model_rk4_matches_the_oracle():
    n, orbits, steps, stride, dt = 8, 96, 300, 50, 0.01
    p, x0 = inputs.kuramoto(n, orbits, seed=45)
    fr, fin = _run_user(user_models.KURAMOTO_PAIRWISE, n, n, n + 2, p, x0, dt, steps, stride, "fp64", rk4=True)
    rfr, rfin = run_oracle("kuramoto", n, p, x0, dt, steps, stride, seed=5, orbit_offset=2, rk4=True)
    assert max_rel_err(fr, rfr) < 1e-12
    assert max_rel_err(fin, rfin) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_user_model_resume_and_refusals(precision):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 16, 64
    p, x0 = _cast(precision, *inputs.fhn(n // 2, orbits, seed=46))
    a = _run_user(user_models.FHN, n, n // 2, 6, p, x0, 0.01, 250, 25, precision)
    b = _run_user(user_models.FHN, n, n // 2, 6, p, x0, 0.01, 250, 25, precision,
                  ranges=[(0, 101), (101, 102), (102, 250)])
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    pb = sdeb.Problem.make("user", n, orbits, 0.01, 10, 5, 1, precision, m=n // 2, d=6)
    with Integrator(pb, user_source=user_models.FHN) as it:
        with pytest.raises(sdeb.SdebError) as e:
            it.set_layout(1, 8)
        assert e.value.status == sdeb.SDEB_EUNSUPPORTED
        t = torch.float64 if precision == "fp64" else torch.float32
        it.set_params(torch.tensor(p, dtype=t).cuda(), torch.tensor(x0, dtype=t).cuda())
        it.autotune()                                     # nothing to tune: one kernel shape
        it.integrate()
        with pytest.raises(sdeb.SdebError) as e:
            it.grad(torch.zeros(orbits, n, dtype=t, device="cuda"))
        assert e.value.status in (sdeb.SDEB_EUNSUPPORTED, sdeb.SDEB_ESTATE)
