"""The oracle alone shows that some Kuramoto orbits amplify a rounding-size
perturbation by orders of magnitude over the benchmark horizon (t = 50),
while synchronised orbits damp it.  This is why the GPU parity tests state a
pathwise horizon (t <= 10) and bound the error beyond it by the dynamics'
own sensitivity.  CPU only: oracle against oracle."""
import numpy as np
import pytest

import oracle
from paper_1908_03869_gb300 import inputs


def _divergence(n, orbits, orbit, ulp, steps=10000):
    p, x0 = inputs.kuramoto(n, orbits, seed=1)
    p = p[orbit:orbit + 1].astype(np.float32).astype(np.float64)
    x0 = x0[orbit:orbit + 1].astype(np.float32).astype(np.float64)
    pb = oracle.make_problem("kuramoto", n, n, n + 2, 0.005, steps, 100, 0, mean_field=True)
    fr, _ = oracle.integrate(pb, p, x0, orbit_begin=orbit)
    sign = np.where(np.sin(np.arange(n) * 7.1) >= 0, 1.0, -1.0)
    frp, _ = oracle.integrate(pb, p, x0 * (1 + ulp * sign), orbit_begin=orbit)
    d = (np.abs(frp - fr) / np.maximum(np.abs(fr), 1.0)).max(axis=(1, 2))
    return d, p[0, 0]


def test_near_critical_orbit_amplifies_one_ulp():
    # n = 32, orbit 56352 (K ~ 3.08): 2^-24 at t = 0 grows past 1e-2 within
    # the horizon (the common noise can later pull the two copies together)
    d, K = _divergence(32, 1 << 18, 56352, 2.0 ** -24)
    assert d[0] < 1e-7
    assert d.max() > 1e-2
    assert d.max() / d[0] > 1e5


def test_synchronised_orbit_damps_one_ulp():
    # n = 128, orbit 65535 (K ~ 3.93, strongly locked): stays at rounding level
    d, K = _divergence(128, 1 << 16, 65535, 2.0 ** -24)
    assert d.max() < 1e-5


def test_fhn_network_amplifies_one_ulp():
    # 64 FitzHugh-Nagumo units with multiplicative noise (orbit 4099 of the
    # 2^18-orbit workload): a 2^-24 relative perturbation of the initial
    # state grows more than 20-fold within t = 200 (spike timing), so the
    # pathwise tolerances have a horizon.
    units, steps, orb = 64, 20000, 4099
    p, x0 = inputs.fhn(units, orb + 1, seed=1)
    p = p[orb:orb + 1].astype(np.float32).astype(np.float64)
    x0 = x0[orb:orb + 1].astype(np.float32).astype(np.float64)
    pb = oracle.make_problem("fhn_net", 2 * units, units, 6, 0.01, steps, 1000, 0)
    fr, _ = oracle.integrate(pb, p, x0, orbit_begin=orb)
    sign = np.where(np.sin(np.arange(2 * units) * 7.1) >= 0, 1.0, -1.0)
    frp, _ = oracle.integrate(pb, p, x0 * (1 + 2.0 ** -24 * sign), orbit_begin=orb)
    d = (np.abs(frp - fr) / np.maximum(np.abs(fr), 1.0)).max(axis=(1, 2))
    assert d[0] < 1e-7
    assert d.max() > 20 * 2.0 ** -24


# ---------------------------------------------------------------------------
# The ODE-path parity horizons.  Each GPU test of the Runge-Kutta and implicit
# schemes states a horizon; these pins show, on the oracle alone, how far a
# one-rounding perturbation of the initial state carries on the same inputs
# (the GPU tests' seeds and orbit offsets), so each horizon ends where the
# dynamics, not the kernel, would push an implementation that differs from
# the oracle by roundings past the tolerance.
# ---------------------------------------------------------------------------

def _ode_divergence(model, n, p, x0, dt, steps, stride, rel, orbit_begin=3, **kw):
    """max over state components of |x' - x| / max(|x|, 1), per frame and
    orbit, x' integrated from x0 (1 + rel s) with a fixed sign pattern s."""
    import concurrent.futures
    m, d = {"kuramoto": (n, n + 2), "fhn_net": (n // 2, 6)}[model]
    pb = oracle.make_problem(model, n, m, d, dt, steps, stride, 2, **kw)
    sign = np.where(np.sin(np.arange(n) * 7.1) >= 0, 1.0, -1.0)
    with concurrent.futures.ThreadPoolExecutor(2) as ex:   # the oracle releases the GIL
        runs = list(ex.map(lambda x: oracle.integrate(pb, p, x, orbit_begin=orbit_begin, nthreads=2)[0],
                           [x0, x0 * (1 + rel * sign)]))
    return (np.abs(runs[1] - runs[0]) / np.maximum(np.abs(runs[0]), 1.0)).max(axis=2)


def test_rk4_noiseless_n128_fp32_horizon():
    # tests/test_gpu_rk4.py, Kuramoto n = 128 (inputs seed 31, FP32-rounded),
    # dt = 0.01, no noise: one FP32 rounding (2^-24) of x0 stays below the
    # 1e-4 tolerance through t = 2 (the FP32 horizon, 200 steps) and passes
    # it by t = 3.5.  Orbit 171 is the most sensitive of the test's 200.
    p, x0 = inputs.kuramoto(128, 200, seed=31)
    sub = [171, 25]
    p = p[sub].astype(np.float32).astype(np.float64)
    x0 = x0[sub].astype(np.float32).astype(np.float64)
    d = _ode_divergence("kuramoto", 128, p, x0, 0.01, 350, 50, 2.0 ** -24, rk4=True).max(axis=1)
    # frames every 0.5: t = 0, 0.5, ..., 3.5
    assert d[:5].max() < 1e-5          # t <= 2: 6.4e-6
    assert d[3] > 1e-6                 # t = 1.5: 2.6e-6, growing
    assert d[6:].max() > 1e-4          # t = 3 .. 3.5: 1.7e-4 .. 3.2e-4


@pytest.mark.parametrize("scheme,orbit", [("euler", 15), ("midpoint", 33)])
def test_implicit_noiseless_n128_fp64_horizon(scheme, orbit):
    # tests/test_gpu_implicit.py, Kuramoto n = 128 (inputs seed 41), dt =
    # 0.01, 4 Newton iterations a step: one FP64 rounding (2^-52) of x0 stays
    # below the 1e-12 tolerance through t = 3 (the FP64 horizon, 300 steps)
    # and passes it by t = 4 (orbit 15 under implicit Euler, 33 under the
    # midpoint rule: the most sensitive of the test's 200 orbits).
    p, x0 = inputs.kuramoto(128, 200, seed=41)
    d = _ode_divergence("kuramoto", 128, p[[orbit]], x0[[orbit]], 0.01, 400, 50, 2.0 ** -52,
                        orbit_begin=3 + orbit, implicit=scheme)[:, 0]
    # frames every 0.5: t = 0 .. 4
    assert d[:7].max() < 1e-12         # t <= 3
    assert d[7:].max() > 3e-12         # t = 3.5 .. 4: 3.8e-12 .. 2.9e-11


@pytest.mark.parametrize("scheme", ["euler", "midpoint"])
@pytest.mark.parametrize("model,n", [("kuramoto", 32), ("kuramoto", 100), ("fhn_net", 64)])
def test_implicit_large_step_fp64_horizons(scheme, model, n):
    # tests/test_gpu_implicit.py, dt = 0.2 (K dt up to 0.8 for the Kuramoto
    # orbits), 128 orbits: where one FP64 rounding of x0 carries past 1e-12
    # within t = 12 the GPU test's horizon is 30 steps (t = 6); where it
    # stays below 1e-13 through t = 12 the horizon is 60 steps.
    orbits = 128
    if model == "kuramoto":
        p, x0 = inputs.kuramoto(n, orbits, seed=41)
        p[:, 0] = np.linspace(0.0, 4.0, orbits)
        kw = dict(mean_field=n > 64)
    else:
        p, x0 = inputs.fhn(n // 2, orbits, seed=43)
        kw = {}
    d = _ode_divergence(model, n, p, x0, 0.2, 60, 5, 2.0 ** -52, implicit=scheme, **kw).max(axis=1)
    # frames every t = 1, t = 0 .. 12
    if LARGE_STEP_HORIZON[(model, n, scheme)] == 30:
        assert d.max() > 1e-12
    else:
        assert d.max() < 1e-13


# Horizons (steps of dt = 0.2) of the large-step FP64 parity test of the
# implicit schemes, as the pins above support them.
LARGE_STEP_HORIZON = {
    ("kuramoto", 32, "euler"): 30,       # 1.7e-12 at t = 10
    ("kuramoto", 32, "midpoint"): 60,    # below 1e-13 through t = 12
    ("kuramoto", 100, "euler"): 30,      # 2.0e-12 at t = 8
    ("kuramoto", 100, "midpoint"): 30,   # 1.0e-12 at t = 4
    ("fhn_net", 64, "euler"): 60,        # below 1e-13 through t = 12
    ("fhn_net", 64, "midpoint"): 60,
}


def _adjoint_workload_orbit(o, ulp):
    """FP64 oracle gradient of orbit o's order parameter at T = 20 on the
    adjoint workload (n = 32, shared parameters, dt = 0.01, 2000 steps), x0
    moved by ulp (relative, signs fixed per component)."""
    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    n = W["n"]
    p, x0 = inputs.kuramoto(n, W["orbits"], seed=1, shared=True)
    p = p.astype(np.float32).astype(np.float64)
    x = x0[o:o + 1].astype(np.float32).astype(np.float64)
    sign = np.where(np.sin(np.arange(n) * 7.1) >= 0, 1.0, -1.0)
    x = x * (1 + ulp * sign)
    pb = oracle.make_problem("kuramoto", n, n, n + 2, W["dt"], W["steps"], 1, W["seed"])
    _, xK = oracle.integrate(pb, p[None, :], x, orbit_begin=o, frames=False)
    _, dr = oracle.order_param(xK[0])
    dp, _ = oracle.adjoint(pb, p[None, :], x, dr[None, :], orbit_begin=o)
    return dp[0]


def test_adjoint_workload_gradient_sensitivity_at_T20():
    # One FP32 ulp of x0 moves the FP64 gradient of orbit 4 at T = 20 by
    # more than 1e-4 of its largest component (orbit 1: below 1e-6).  An
    # FP32 adjoint takes a rounding in each of its 2000 steps, so on such an
    # orbit it cannot be held to 1e-3 of the FP64 gradient; the GPU tests
    # check the FP32 gradients at T = 20 per orbit statistically (median
    # 1e-4, at most 5 % of orbits beyond 1e-3) and orbit by orbit at T = 5.
    def sens(o):
        g0 = _adjoint_workload_orbit(o, 0.0)
        return np.abs(_adjoint_workload_orbit(o, 2.0 ** -24) - g0).max() / np.abs(g0).max()
    assert sens(4) > 1e-4
    assert sens(1) < 1e-6
