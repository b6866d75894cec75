"""The oracle alone shows that some Kuramoto orbits amplify a rounding-size
perturbation by orders of magnitude over the benchmark horizon (t = 50),
while synchronised orbits damp it.  This is why the GPU parity tests state a
pathwise horizon (t <= 10) and bound the error beyond it by the dynamics'
own sensitivity.  CPU only: oracle against oracle."""
import numpy as np

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
