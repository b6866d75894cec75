"""Pins for the oracle's discrete adjoint and the order parameter (Eq. 7).

The adjoint is checked against the analytic pathwise OU gradient and against
central finite differences of the (separately pinned) forward integrator
with common random numbers: the same seed, hence the same Wiener increments.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1908_03869_gb300 import inputs


def _pb(model, n, dt, steps, seed=0, shared=False):
    m = {"kuramoto": n, "kuramoto_paper": n, "fhn_net": n // 2, "ou": n, "gbm": n, "linear_ode": 0}[model]
    d = {"kuramoto": n + 2, "kuramoto_paper": 2 * n + 1, "fhn_net": 6, "ou": 2, "gbm": 2, "linear_ode": 1}[model]
    return oracle.make_problem(model, n, m, d, dt, steps, 1, seed, shared_params=shared)


def test_ou_adjoint_matches_analytic_gradient():
    # L = X^K, a = 1 - theta dt, X^K = a^K x0 + sigma sqrt(dt) sum_i a^{K-1-i} N_i:
    # dL/dx0 = a^K, dL/dsigma = sqrt(dt) sum a^{K-1-i} N_i,
    # dL/dtheta = -K dt a^{K-1} x0 - sigma sqrt(dt) sum (K-1-i) dt a^{K-2-i} N_i
    K, dt, theta, sigma, x_init, seed = 250, 0.01, 0.6, 0.35, 0.8, 31
    pb = _pb("ou", 1, dt, K, seed=seed)
    params = np.array([[theta, sigma]])
    x0 = np.array([[x_init]])
    dp, dx0 = oracle.adjoint(pb, params, x0, np.ones((1, 1)))
    N = oracle.normals_fill(seed, 0, K, 0, 1, 1)[:, 0, 0]
    a = 1 - theta * dt
    i = np.arange(K)
    dsigma = math.sqrt(dt) * np.sum(a ** (K - 1 - i) * N)
    j = i[:-1]
    dtheta = -K * dt * a ** (K - 1) * x_init - sigma * math.sqrt(dt) * np.sum((K - 1 - j) * dt * a ** (K - 2 - j) * N[:-1])
    assert dx0[0, 0] == pytest.approx(a ** K, rel=1e-12)
    assert dp[0, 1] == pytest.approx(dsigma, rel=1e-11)
    assert dp[0, 0] == pytest.approx(dtheta, rel=1e-11)


def _loss(pb, params, x0, c):
    _, xK = oracle.integrate(pb, params, x0, frames=False)
    return float((xK * c).sum())


def _fd_check(pb, params, x0, rtol=1e-6):
    rng = np.random.Generator(np.random.PCG64(5))
    c = rng.standard_normal(x0.shape)
    dp, dx0 = oracle.adjoint(pb, params, x0, c)
    scale_p = np.abs(dp).max()
    for q in range(params.shape[-1]):
        h = 1e-6 * max(abs(params.reshape(-1, params.shape[-1])[0, q]), 1.0)
        pp, pm = params.copy(), params.copy()
        pp[..., q] += h
        pm[..., q] -= h
        fd = (_loss(pb, pp, x0, c) - _loss(pb, pm, x0, c)) / (2 * h)
        got = dp[:, q].sum()
        assert abs(got - fd) <= rtol * max(abs(fd), scale_p, 1e-8), (q, got, fd)
    for l in range(x0.shape[1]):
        h = 1e-6 * max(abs(x0[0, l]), 1.0)
        xp, xm = x0.copy(), x0.copy()
        xp[0, l] += h
        xm[0, l] -= h
        fd = (_loss(pb, params, xp, c) - _loss(pb, params, xm, c)) / (2 * h)
        assert abs(dx0[0, l] - fd) <= rtol * max(abs(fd), np.abs(dx0).max()), (l, dx0[0, l], fd)


def test_kuramoto_adjoint_vs_central_fd():
    params, x0 = inputs.kuramoto(6, 1, seed=2)
    _fd_check(_pb("kuramoto", 6, 0.01, 300, seed=4), params, x0)


def test_kuramoto_shared_params_adjoint_vs_central_fd():
    params, x0 = inputs.kuramoto(5, 3, seed=3, shared=True)
    pb = _pb("kuramoto", 5, 0.01, 200, seed=6, shared=True)
    rng = np.random.Generator(np.random.PCG64(1))
    c = rng.standard_normal(x0.shape)
    dp, _ = oracle.adjoint(pb, params, x0, c)
    for q in range(params.size):
        h = 1e-6 * max(abs(params[q]), 1.0)
        pp, pm = params.copy(), params.copy()
        pp[q] += h
        pm[q] -= h
        fd = (_loss(pb, pp, x0, c) - _loss(pb, pm, x0, c)) / (2 * h)
        assert dp[:, q].sum() == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(dp).max())


def test_kuramoto_paper_layout_adjoint_vs_central_fd():
    params, x0 = inputs.kuramoto_paper_speed(4, 1, seed=5)
    params[:, 0] = 2.0
    params[:, 5:] = 0.3
    _fd_check(_pb("kuramoto_paper", 4, 0.02, 200, seed=7), params, x0)


def test_fhn_adjoint_vs_central_fd():
    params, x0 = inputs.fhn(3, 1, seed=4)
    params[:, 5] = 0.3
    _fd_check(_pb("fhn_net", 6, 0.01, 300, seed=9), params, x0)


def test_gbm_and_linear_adjoint_vs_central_fd():
    params, x0 = inputs.scalar_model(3, 1, [0.2, 0.5], 0.5, 1.5, seed=1)
    _fd_check(_pb("gbm", 3, 0.01, 200, seed=2), params, x0)
    params, x0 = inputs.scalar_model(2, 1, [0.7], -1.0, 1.0, seed=2)
    _fd_check(_pb("linear_ode", 2, 0.01, 200), params, x0)


def test_order_parameter_special_cases_and_gradient():
    r, dr = oracle.order_param(np.full(7, 1.234))
    assert r == pytest.approx(1.0, rel=1e-15)
    np.testing.assert_allclose(dr, 0.0, atol=1e-15)
    r, _ = oracle.order_param(2 * math.pi * np.arange(8) / 8 + 0.3)
    assert r < 1e-15
    # two phases: r = |cos((a - b) / 2)|
    r, _ = oracle.order_param(np.array([0.4, 1.5]))
    assert r == pytest.approx(abs(math.cos(0.55)), rel=1e-14)
    th = np.random.Generator(np.random.PCG64(3)).uniform(0, 2 * math.pi, 11)
    r, dr = oracle.order_param(th)
    for l in range(11):
        tp, tm = th.copy(), th.copy()
        tp[l] += 1e-6
        tm[l] -= 1e-6
        fd = (oracle.order_param(tp)[0] - oracle.order_param(tm)[0]) / 2e-6
        assert dr[l] == pytest.approx(fd, rel=1e-6, abs=1e-10)
