"""Pins of the oracle's fourth-order Runge-Kutta step on the drift alone
(the ODE path: the paper lists Runge-Kutta among its ODE integrators,
Sec. 1.5; classical RK4):

* Linear ODE dx/dt = -theta x: RK4 multiplies x by the degree-4 Taylor
  polynomial of exp(-h theta) every step, so x_K = R(h theta)^K x0 with
  R(z) = 1 - z + z^2/2 - z^3/6 + z^4/24 (closed form).
* Kuramoto with K = 0: the drift is the constant omega, which RK4 integrates
  exactly: theta(t) = theta(0) + omega t.
* Self-convergence of order 4 on nonlinear drifts (Kuramoto n = 5, the
  FitzHugh-Nagumo network): halving dt divides the error against a
  64-times-finer RK4 run by ~16 (a wrong stage or weight drops the order).
* The diffusion is not applied: RK4 on Kuramoto with sigma > 0 equals RK4
  with sigma = 0 bit for bit; and RK4 and Milstein together are rejected.
"""
import math

import numpy as np
import pytest

import oracle


def _run(model, n, m, d, p, x0, dt, steps, **kw):
    pb = oracle.make_problem(model, n, m, d, dt, steps, steps, 3, rk4=True, **kw)
    return oracle.integrate(pb, np.atleast_2d(p), np.atleast_2d(x0), frames=False)[1]


def test_linear_ode_closed_form():
    theta, dt, steps = 0.7, 0.05, 300
    x0 = np.array([[1.5, -0.25, 3.0]])
    xK = _run("linear_ode", 3, 0, 1, [theta], x0, dt, steps)
    z = theta * dt
    R = 1 - z + z ** 2 / 2 - z ** 3 / 6 + z ** 4 / 24
    np.testing.assert_allclose(xK, x0 * R ** steps, rtol=1e-13, atol=0)


def test_uncoupled_kuramoto_is_integrated_exactly():
    n, dt, steps = 4, 0.01, 500
    omega = np.array([0.3, -1.2, 2.0, 0.05])
    p = np.concatenate([[0.0, 0.4], omega])
    th0 = np.array([[0.1, 2.0, -1.0, 4.0]])
    xK = _run("kuramoto", n, n, n + 2, p, th0, dt, steps)
    np.testing.assert_allclose(xK, th0 + omega * dt * steps, rtol=0, atol=1e-12)


@pytest.mark.parametrize("model,n,m,d,p,x0", [
    ("kuramoto", 5, 5, 7, [2.5, 0.0, 0.4, -0.3, 1.1, 0.0, -0.8], [0.3, 1.9, -2.2, 0.5, 3.0]),
    ("fhn_net", 8, 4, 6, [0.7, 0.8, 0.08, 0.5, 0.3, 0.05], [1.2, -0.5, 0.3, -1.7, 0.1, 0.9, -0.2, 0.4]),
])
def test_fourth_order_self_convergence(model, n, m, d, p, x0):
    T = 4.0
    ref = _run(model, n, m, d, p, x0, T / (64 * 400), 64 * 400)
    errs = []
    for steps in (50, 100, 200):
        errs.append(np.abs(_run(model, n, m, d, p, x0, T / steps, steps) - ref).max())
    slope = np.polyfit(np.log([T / 50, T / 100, T / 200]), np.log(errs), 1)[0]
    assert 3.7 < slope < 4.4, (errs, slope)


def test_diffusion_is_not_applied_and_flags_are_exclusive():
    n = 6
    p0 = np.concatenate([[1.3, 0.0], np.linspace(-1, 1, n)])
    p1 = p0.copy()
    p1[1] = 0.8
    x0 = np.linspace(0, 5, n)
    a = _run("kuramoto", n, n, n + 2, p0, x0, 0.01, 300)
    b = _run("kuramoto", n, n, n + 2, p1, x0, 0.01, 300)
    np.testing.assert_array_equal(a, b)
    pb = oracle.make_problem("gbm", 2, 2, 2, 0.01, 10, 10, 0, milstein=True, rk4=True)
    assert oracle.lib().oracle_check_problem(pb) != 0
