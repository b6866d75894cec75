"""Pins of the oracle's Milstein step (the scheme the paper names as the
next one to add, Sec. 2.1 and Sec. 3; Kloeden and Platen, Sec. 10.3), for
diagonal noise: X_j += f_j dt + g_jj dW_j + 1/2 g_jj g_jj' (dW_j^2 - dt).

* The diffusion derivative against central differences of the diffusion.
* GBM: the Milstein recursion written out as a product over the oracle's own
  normals, x0 prod_k (1 + mu dt + sigma dW_k + sigma^2 (dW_k^2 - dt) / 2).
* Additive noise (Kuramoto, OU) and no noise: Milstein equals Euler-Maruyama
  bit for bit.
* Strong convergence on GBM against the exact solution on the same Brownian
  path, x0 exp((mu - sigma^2/2) T + sigma W_T): the mean pathwise error falls
  as dt^1 for Milstein and as dt^(1/2) for Euler-Maruyama (the textbook
  strong orders 1 and 1/2).
"""
import math

import numpy as np
import pytest

import oracle


def test_diffusion_derivative_matches_central_differences():
    rng = np.random.Generator(np.random.PCG64(1))
    cases = [("gbm", 3, 3, 2, np.array([0.3, 0.7])),
             ("fhn_net", 8, 4, 6, np.array([0.7, 0.8, 0.08, 0.5, 0.3, 0.05])),
             ("ou", 2, 2, 2, np.array([0.5, 0.4])),
             ("kuramoto", 3, 3, 5, np.array([1.0, 0.3, 0.1, -0.2, 0.4]))]
    for model, n, m, d, p in cases:
        pb = oracle.make_problem(model, n, m, d, 0.01, 1)
        x = rng.uniform(-1.5, 1.5, n)
        dg = oracle.diffusion_diag_derivative(pb, x, p)
        g0 = oracle.diffusion(pb, x, p)
        h = 1e-6
        for j in range(m):
            xp, xm = x.copy(), x.copy()
            xp[j] += h
            xm[j] -= h
            fd = (oracle.diffusion(pb, xp, p)[j, j] - oracle.diffusion(pb, xm, p)[j, j]) / (2 * h)
            assert abs(fd - dg[j]) < 1e-8, (model, j, fd, dg[j])
            # diagonal noise: channel j drives component j only
            off = np.delete(g0[:, j], j)
            assert np.all(off == 0.0)


def test_gbm_milstein_is_the_product_formula():
    mu, sigma, dt, steps, seed, orbits = 0.4, 0.9, 0.02, 150, 11, 6
    pb = oracle.make_problem("gbm", 2, 2, 2, dt, steps, 50, seed, milstein=True)
    p = np.tile([mu, sigma], (orbits, 1))
    x0 = np.array([[1.0, 0.5]] * orbits) * np.arange(1, orbits + 1)[:, None]
    _, xK = oracle.integrate(pb, p, x0, orbit_begin=7)
    N = oracle.normals_fill(seed, 0, steps, 7, orbits, 2)   # [k][o][m]
    dW = math.sqrt(dt) * N
    factor = np.prod(1.0 + mu * dt + sigma * dW + 0.5 * sigma ** 2 * (dW ** 2 - dt), axis=0)
    np.testing.assert_allclose(xK, x0 * factor, rtol=1e-12, atol=0)


@pytest.mark.parametrize("model,n,m,d,p", [
    ("kuramoto", 4, 4, 6, [1.5, 0.3, 0.2, -0.1, 0.5, 0.0]),
    ("ou", 3, 3, 2, [0.7, 0.4]),
    ("linear_ode", 2, 0, 1, [0.3]),
])
def test_additive_noise_milstein_equals_euler_maruyama(model, n, m, d, p):
    x0 = np.linspace(-1.0, 1.0, 3 * n).reshape(3, n)
    p = np.tile(p, (3, 1))
    outs = []
    for mil in (False, True):
        pb = oracle.make_problem(model, n, m, d, 0.01, 200, 20, 5, milstein=mil)
        outs.append(oracle.integrate(pb, p, x0))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


def _strong_error(milstein, dt, orbits=4096, T=1.0, mu=1.0, sigma=1.0, seed=3):
    steps = int(round(T / dt))
    pb = oracle.make_problem("gbm", 1, 1, 2, dt, steps, steps, seed, milstein=milstein)
    p = np.tile([mu, sigma], (orbits, 1))
    x0 = np.ones((orbits, 1))
    _, xK = oracle.integrate(pb, p, x0, nthreads=8)
    W = math.sqrt(dt) * oracle.normals_fill(seed, 0, steps, 0, orbits, 1).sum(axis=0)   # [o][1]
    exact = np.exp((mu - 0.5 * sigma ** 2) * T + sigma * W)
    return float(np.mean(np.abs(xK - exact)))


def test_strong_orders_one_and_one_half_on_gbm():
    dts = [2.0 ** -4, 2.0 ** -6, 2.0 ** -8]
    for milstein, order in ((True, 1.0), (False, 0.5)):
        errs = [_strong_error(milstein, dt) for dt in dts]
        slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
        assert abs(slope - order) < 0.15, (milstein, errs, slope)
    # at the finest step Milstein is far more accurate than Euler-Maruyama
    assert _strong_error(True, dts[-1]) < 0.2 * _strong_error(False, dts[-1])
