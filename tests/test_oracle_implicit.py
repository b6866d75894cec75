"""Pins of the oracle's implicit ODE schemes on the drift alone (the paper
lists implicit Euler and implicit midpoint among its ODE integrators,
Sec. 1.5), each step solved by a fixed count of Newton iterations:

* The drift Jacobian against central differences of the drift, every model.
* Linear ODE dx/dt = -theta x (closed forms): implicit Euler gives
  x0 / (1 + h theta)^K, implicit midpoint x0 ((1 - h theta/2)/(1 + h theta/2))^K;
  with h theta = 10 (stiff) both stay bounded where explicit Euler's factor
  1 - h theta = -9 would explode.
* Self-convergence on nonlinear drifts (Kuramoto n = 6, the FHN network):
  order 1 for implicit Euler and 2 for implicit midpoint; and the Newton
  iterations have converged (the step equation's residual is at rounding).
"""
import numpy as np
import pytest

import oracle

MODELS = [
    ("kuramoto", 6, 6, 8, [2.0, 0.0, 0.4, -0.3, 1.1, 0.0, -0.8, 0.2], [0.3, 1.9, -2.2, 0.5, 3.0, -1.0]),
    ("fhn_net", 8, 4, 6, [0.7, 0.8, 0.08, 0.5, 0.3, 0.05], [1.2, -0.5, 0.3, -1.7, 0.1, 0.9, -0.2, 0.4]),
]


def _run(model, n, m, d, p, x0, dt, steps, implicit):
    pb = oracle.make_problem(model, n, m, d, dt, steps, steps, 3, implicit=implicit)
    return oracle.integrate(pb, np.atleast_2d(p), np.atleast_2d(x0), frames=False)[1][0]


@pytest.mark.parametrize("model,n,m,d,p,x0", MODELS + [
    ("gbm", 3, 3, 2, [0.4, 0.2], [1.0, 0.5, 2.0]), ("ou", 3, 3, 2, [0.7, 0.3], [1.0, -0.5, 2.0]),
    ("kuramoto_paper", 4, 4, 9, [1.5, 0.1, -0.2, 0.3, 0.0, 0.01, 0.02, 0.01, 0.02], [0.1, 1.0, 2.0, -1.0])])
def test_jacobian_against_central_differences(model, n, m, d, p, x0):
    pb = oracle.make_problem(model, n, m, d, 0.01, 1)
    x0, p = np.asarray(x0, float), np.asarray(p, float)
    J = oracle.drift_jacobian(pb, x0, p)
    h = 1e-6
    for j in range(n):
        xp, xm = x0.copy(), x0.copy()
        xp[j] += h
        xm[j] -= h
        fd = (oracle.drift(pb, xp, p) - oracle.drift(pb, xm, p)) / (2 * h)
        np.testing.assert_allclose(J[:, j], fd, rtol=0, atol=1e-8)


@pytest.mark.parametrize("theta_h", [0.05, 10.0])
def test_linear_ode_closed_forms(theta_h):
    theta, steps = 0.5, 60
    dt = theta_h / theta
    x0 = np.array([1.5, -0.25, 3.0])
    be = _run("linear_ode", 3, 0, 1, [theta], x0, dt, steps, "euler")
    mp = _run("linear_ode", 3, 0, 1, [theta], x0, dt, steps, "midpoint")
    np.testing.assert_allclose(be, x0 / (1 + theta_h) ** steps, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(mp, x0 * ((1 - theta_h / 2) / (1 + theta_h / 2)) ** steps, rtol=1e-12, atol=1e-300)
    assert np.all(np.abs(be) <= np.abs(x0)) and np.all(np.abs(mp) <= np.abs(x0))   # stable, also when stiff


@pytest.mark.parametrize("model,n,m,d,p,x0", MODELS)
def test_orders_one_and_two(model, n, m, d, p, x0):
    T = 2.0
    ref = _run(model, n, m, d, p, x0, T / 6400, 6400, "midpoint")
    for scheme, order in (("euler", 1.0), ("midpoint", 2.0)):
        errs = [np.abs(_run(model, n, m, d, p, x0, T / s, s, scheme) - ref).max() for s in (50, 100, 200)]
        slope = np.polyfit(np.log([T / 50, T / 100, T / 200]), np.log(errs), 1)[0]
        assert abs(slope - order) < 0.15, (model, scheme, errs, slope)


@pytest.mark.parametrize("model,n,m,d,p,x0", MODELS)
def test_newton_iterations_converge(model, n, m, d, p, x0):
    dt = 0.05
    x0, p = np.asarray(x0, float), np.asarray(p, float)
    pb = oracle.make_problem(model, n, m, d, dt, 1)
    for scheme, theta in (("euler", 1.0), ("midpoint", 0.5)):
        y = _run(model, n, m, d, p, x0, dt, 1, scheme)
        residual = y - x0 - dt * oracle.drift(pb, x0 + theta * (y - x0), p)
        assert np.abs(residual).max() < 1e-13, (scheme, residual)
