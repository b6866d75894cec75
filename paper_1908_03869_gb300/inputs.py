"""Seeded synthetic inputs for the Euler-Maruyama workloads.

This module holds no arithmetic of the method itself: it only draws initial
states and parameter vectors with numpy's PCG64 generator, so the CUDA path
and the CPU oracle can be fed identical inputs.  (The Wiener increments are
not drawn here; both sides derive them from the Philox counter.)

Distributions:
  * Kuramoto workloads (scalar-sigma layout p = (K, sigma, omega_1..omega_n)):
    omega_i ~ N(0, 1), K ~ U(0, 4), sigma ~ U(0.1, 0.5), theta_i(0) ~ U(0, 2 pi).
  * The paper's speed protocol (Sec. 2.2.1, layout p = (K, omega, p)):
    theta_i(0) ~ U(-pi, pi), omega_i ~ U(0.01, 0.03), p_i ~ U(0.001, 0.003), K = 1.
  * The paper's accuracy protocol (Sec. 2.3.1): N = 100, omega_i ~ U(0.2, 0.4),
    theta_i(0) ~ U(-pi, pi), p_i ~ U(0.01, 0.03), K in {0.02, 0.2}.
  * FitzHugh-Nagumo network (p = (a, b, eps, I, c, sigma)): a ~ U(0.6, 0.8),
    b ~ U(0.7, 0.9), eps ~ U(0.05, 0.1), I ~ U(0.3, 0.6), c ~ U(0, 0.5),
    sigma ~ U(0.01, 0.1); v_i(0) ~ U(-2, 2), w_i(0) ~ U(-0.5, 1.5).
  * Batched heterogeneous instances: n ~ U{2..256},
    steps = round(exp(U(ln 1e3, ln 1e5))), dt in {0.001, 0.01} with
    probability 1/2 each, parameters as for the Kuramoto workloads.
"""
import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def kuramoto(n, orbits, seed=1, shared=False):
    """Scalar-sigma Kuramoto inputs.  Returns (params, x0): params is [orbits][n+2]
    (or [n+2] when shared) and x0 is [orbits][n], both float64."""
    g = _rng(seed)
    rows = 1 if shared else orbits
    p = np.empty((rows, n + 2))
    p[:, 0] = g.uniform(0.0, 4.0, rows)
    p[:, 1] = g.uniform(0.1, 0.5, rows)
    p[:, 2:] = g.standard_normal((rows, n))
    x0 = g.uniform(0.0, 2.0 * math.pi, (orbits, n))
    return (p[0].copy() if shared else p), x0


def kuramoto_paper_speed(n, orbits, seed=1):
    """Paper layout p = (K, omega_1..omega_n, p_1..p_n), Sec. 2.2.1 distributions."""
    g = _rng(seed)
    p = np.empty((orbits, 2 * n + 1))
    p[:, 0] = 1.0
    p[:, 1:n + 1] = g.uniform(0.01, 0.03, (orbits, n))
    p[:, n + 1:] = g.uniform(0.001, 0.003, (orbits, n))
    x0 = g.uniform(-math.pi, math.pi, (orbits, n))
    return p, x0


def kuramoto_paper_accuracy(K, orbits=64, n=100, seed=1):
    """Paper layout, Sec. 2.3.1 distributions (N = 100, 64 realisations)."""
    g = _rng(seed)
    p = np.empty((orbits, 2 * n + 1))
    p[:, 0] = K
    p[:, 1:n + 1] = g.uniform(0.2, 0.4, (orbits, n))
    p[:, n + 1:] = g.uniform(0.01, 0.03, (orbits, n))
    x0 = g.uniform(-math.pi, math.pi, (orbits, n))
    return p, x0


def fhn(units, orbits, seed=1):
    """FitzHugh-Nagumo network inputs: params [orbits][6], x0 [orbits][2*units]
    ordered (v_1..v_u, w_1..w_u)."""
    g = _rng(seed)
    p = np.empty((orbits, 6))
    p[:, 0] = g.uniform(0.6, 0.8, orbits)
    p[:, 1] = g.uniform(0.7, 0.9, orbits)
    p[:, 2] = g.uniform(0.05, 0.1, orbits)
    p[:, 3] = g.uniform(0.3, 0.6, orbits)
    p[:, 4] = g.uniform(0.0, 0.5, orbits)
    p[:, 5] = g.uniform(0.01, 0.1, orbits)
    x0 = np.empty((orbits, 2 * units))
    x0[:, :units] = g.uniform(-2.0, 2.0, (orbits, units))
    x0[:, units:] = g.uniform(-0.5, 1.5, (orbits, units))
    return p, x0


def scalar_model(n, orbits, p, x_low, x_high, seed=1):
    """Inputs for the two-parameter test models (OU, GBM) and the linear ODE:
    params [orbits][len(p)] all equal to p, x0 ~ U(x_low, x_high)."""
    g = _rng(seed)
    params = np.tile(np.asarray(p, dtype=np.float64), (orbits, 1))
    x0 = g.uniform(x_low, x_high, (orbits, n))
    return params, x0


def batched_instances(count=4096, seed=1, n_low=2, n_high=256, k_low=1e3, k_high=1e5):
    """Heterogeneous single-orbit instances.  Returns a list of dicts with keys
    n, steps, dt, params [n+2], x0 [n]."""
    g = _rng(seed)
    out = []
    for _ in range(count):
        n = int(g.integers(n_low, n_high + 1))
        steps = int(round(math.exp(g.uniform(math.log(k_low), math.log(k_high)))))
        dt = 0.001 if g.uniform() < 0.5 else 0.01
        p = np.empty(n + 2)
        p[0] = g.uniform(0.0, 4.0)
        p[1] = g.uniform(0.1, 0.5)
        p[2:] = g.standard_normal(n)
        x0 = g.uniform(0.0, 2.0 * math.pi, n)
        out.append(dict(n=n, steps=steps, dt=dt, params=p, x0=x0))
    return out


# The workload table.  Sizes are those the library is benchmarked and tested on.
WORKLOADS = {
    "kuramoto_n4_fp64": dict(model="kuramoto", n=4, orbits=1024, dt=0.01, steps=1000, stride=10,
                             precision="fp64", seed=0),
    "kuramoto_n8": dict(model="kuramoto", n=8, orbits=1 << 20, dt=0.005, steps=10000, stride=100, seed=0),
    "kuramoto_n32": dict(model="kuramoto", n=32, orbits=1 << 18, dt=0.005, steps=10000, stride=100, seed=0),
    "kuramoto_n128": dict(model="kuramoto", n=128, orbits=1 << 16, dt=0.005, steps=10000, stride=100, seed=0),
    "kuramoto_adjoint_n32": dict(model="kuramoto", n=32, orbits=16384, dt=0.01, steps=2000, ckpt_every=100,
                                 seed=0, shared=True),
    "fhn_64units": dict(model="fhn_net", n=128, orbits=1 << 18, dt=0.01, steps=100000, stride=1000, seed=0),
    "batched_4096": dict(model="kuramoto", count=4096, stride=100, seed=0),
}
