"""Pins for the oracle's Euler-Maruyama integrator (Eq. 2) and its models.

Each test checks the oracle against something other than itself: closed
forms of linear SDEs (OU, GBM, the g = 0 linear ODE), the exact discrete
moments of OU, the closed-form Adler solution for two coupled phases,
conservation laws of the coupling terms, the analytic FitzHugh-Nagumo
fixed point, and a hand-expanded high-precision recursion on tiny inputs.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_1908_03869_gb300 import inputs


def _pb(model, n, dt, steps, stride=1, seed=0, **kw):
    m = {"kuramoto": n, "kuramoto_paper": n, "fhn_net": n // 2, "ou": n, "gbm": n, "linear_ode": 0}[model]
    d = {"kuramoto": n + 2, "kuramoto_paper": 2 * n + 1, "fhn_net": 6, "ou": 2, "gbm": 2, "linear_ode": 1}[model]
    return oracle.make_problem(model, n, m, d, dt, steps, stride, seed, **kw)


def test_ou_pathwise_closed_form():
    # X^K = a^K x0 + sigma sqrt(dt) sum_i a^{K-1-i} N^i, a = 1 - theta dt
    n, orbits, K, dt, theta, sigma = 3, 6, 400, 0.01, 0.7, 0.4
    pb = _pb("ou", n, dt, K, seed=21)
    params, x0 = inputs.scalar_model(n, orbits, [theta, sigma], -1, 1, seed=2)
    _, xK = oracle.integrate(pb, params, x0, frames=False)
    N = oracle.normals_fill(21, 0, K, 0, orbits, n)          # [K][orbits][n]
    a = 1.0 - theta * dt
    weights = a ** (K - 1 - np.arange(K))
    want = a ** K * x0 + sigma * math.sqrt(dt) * np.einsum("k,kon->on", weights, N)
    np.testing.assert_allclose(xK, want, rtol=1e-12, atol=1e-13)


def test_ou_exact_discrete_moments():
    # mean a^K x0 and variance sigma^2 dt (1 - a^{2K}) / (1 - a^2) over orbits
    orbits, K, dt, theta, sigma, x_init = 40000, 150, 0.02, 0.8, 0.5, 1.5
    pb = _pb("ou", 1, dt, K, seed=5)
    params = np.tile([theta, sigma], (orbits, 1))
    x0 = np.full((orbits, 1), x_init)
    _, xK = oracle.integrate(pb, params, x0, frames=False, nthreads=4)
    a = 1.0 - theta * dt
    mean = a ** K * x_init
    var = sigma ** 2 * dt * (1 - a ** (2 * K)) / (1 - a ** 2)
    se_mean = math.sqrt(var / orbits)
    se_var = var * math.sqrt(2.0 / (orbits - 1))
    assert abs(xK.mean() - mean) < 5 * se_mean
    assert abs(xK.var(ddof=1) - var) < 5 * se_var


def test_gbm_pathwise_product():
    # multiplicative noise: X^K = x0 prod_i (1 + mu dt + sigma sqrt(dt) N^i)
    n, orbits, K, dt, mu, sigma = 5, 4, 300, 0.005, 0.3, 0.6
    pb = _pb("gbm", n, dt, K, seed=8)
    params, x0 = inputs.scalar_model(n, orbits, [mu, sigma], 0.5, 2.0, seed=4)
    _, xK = oracle.integrate(pb, params, x0, frames=False)
    N = oracle.normals_fill(8, 0, K, 0, orbits, n)
    want = x0 * np.prod(1.0 + mu * dt + sigma * math.sqrt(dt) * N, axis=0)
    np.testing.assert_allclose(xK, want, rtol=1e-12)


def test_linear_ode_g_zero():
    n, orbits, K, dt, theta = 4, 3, 1000, 0.01, 0.9
    pb = _pb("linear_ode", n, dt, K, stride=250)
    params, x0 = inputs.scalar_model(n, orbits, [theta], -3, 3, seed=6)
    fr, xK = oracle.integrate(pb, params, x0)
    np.testing.assert_allclose(xK, (1 - theta * dt) ** K * x0, rtol=1e-12)
    for f in range(fr.shape[0]):
        np.testing.assert_allclose(fr[f], (1 - theta * dt) ** (250 * f) * x0, rtol=1e-12)


def test_kuramoto_uncoupled_noiseless_is_free_rotation():
    n, orbits, K, dt = 6, 5, 2000, 0.005
    pb = _pb("kuramoto", n, dt, K)
    params, x0 = inputs.kuramoto(n, orbits, seed=3)
    params[:, 0] = 0.0   # K
    params[:, 1] = 0.0   # sigma
    _, xK = oracle.integrate(pb, params, x0, frames=False)
    np.testing.assert_allclose(xK, x0 + K * dt * params[:, 2:], rtol=1e-12, atol=1e-12)


def _adler_exact(psi0, a, b, t):
    # psi' = a - b sin psi, b > |a|: with u = tan(psi/2), (u - u+)/(u - u-) = C exp(lam t)
    lam = math.sqrt(b * b - a * a)
    up, um = (b + lam) / a, (b - lam) / a
    u0 = math.tan(psi0 / 2)
    E = (u0 - up) / (u0 - um) * math.exp(lam * t)
    return 2 * math.atan((up - E * um) / (1 - E))


def test_kuramoto_two_oscillators_adler_closed_form():
    # n = 2, sigma = 0: psi = theta_2 - theta_1 obeys psi' = (w2 - w1) - K sin psi;
    # EM converges to the closed form with order one in dt.
    w1, w2, Kc, T = 0.1, 0.4, 1.0, 6.0
    th0 = np.array([[0.2, 0.9]])
    errs = []
    for steps in (3000, 6000, 12000):
        dt = T / steps
        pb = _pb("kuramoto", 2, dt, steps)
        params = np.array([[Kc, 0.0, w1, w2]])
        _, xK = oracle.integrate(pb, params, th0, frames=False)
        psi = xK[0, 1] - xK[0, 0]
        errs.append(abs(psi - _adler_exact(0.7, w2 - w1, Kc, T)))
        # the mean phase rotates freely: theta_1 + theta_2 = const + (w1 + w2) t
        assert xK.sum() == pytest.approx(th0.sum() + (w1 + w2) * T, rel=1e-12)
    assert errs[0] < 1e-3
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


@pytest.mark.parametrize("model", ["kuramoto", "kuramoto_paper"])
def test_kuramoto_coupling_conserves_phase_sum(model):
    # sum_i sin(theta_j - theta_i) over all pairs cancels, so
    # sum theta^{k+1} - sum theta^k = dt sum omega + sqrt(dt) sum_i g_ii N_i.
    n, orbits, K, dt = 7, 3, 60, 0.01
    pb = _pb(model, n, dt, K, seed=13)
    if model == "kuramoto":
        params, x0 = inputs.kuramoto(n, orbits, seed=9)
        params[:, 0] = 3.5
        omega, g = params[:, 2:], params[:, 1:2] * np.ones((1, n))
    else:
        params, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=9)
        params[:, 0] = 3.5
        omega, g = params[:, 1:n + 1], params[:, n + 1:]
    fr, _ = oracle.integrate(pb, params, x0)
    N = oracle.normals_fill(13, 0, K, 0, orbits, n)
    for k in range(K):
        lhs = fr[k + 1].sum(axis=1) - fr[k].sum(axis=1)
        rhs = dt * omega.sum(axis=1) + math.sqrt(dt) * (g * N[k]).sum(axis=1)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


def test_kuramoto_pairwise_equals_mean_field():
    n, orbits, K, dt = 16, 4, 500, 0.01
    params, x0 = inputs.kuramoto(n, orbits, seed=10)
    _, a = oracle.integrate(_pb("kuramoto", n, dt, K, seed=1), params, x0, frames=False)
    _, b = oracle.integrate(_pb("kuramoto", n, dt, K, seed=1, mean_field=True), params, x0, frames=False)
    np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11)


def test_kuramoto_paper_layout_matches_scalar_layout():
    # p = (K, omega, p_i) with every p_i = sigma is the same SDE as p = (K, sigma, omega)
    n, orbits, K, dt = 5, 3, 200, 0.01
    ps, x0 = inputs.kuramoto(n, orbits, seed=12)
    pp = np.concatenate([ps[:, :1], ps[:, 2:], np.repeat(ps[:, 1:2], n, axis=1)], axis=1)
    _, a = oracle.integrate(_pb("kuramoto", n, dt, K, seed=4), ps, x0, frames=False)
    _, b = oracle.integrate(_pb("kuramoto_paper", n, dt, K, seed=4), pp, x0, frames=False)
    np.testing.assert_array_equal(a, b)


def test_kuramoto_brute_force_tiny():
    # Hand-expanded recursion in 40-digit arithmetic for n = 3, 4 steps.
    mpmath.mp.dps = 40
    n, steps, dt, seed = 3, 4, 0.05, 99
    params, x0 = inputs.kuramoto(n, 2, seed=14)
    _, xK = oracle.integrate(_pb("kuramoto", n, dt, steps, seed=seed), params, x0, frames=False)
    N = oracle.normals_fill(seed, 0, steps, 0, 2, n)
    for o in range(2):
        Kc, sig = mpmath.mpf(params[o, 0]), mpmath.mpf(params[o, 1])
        om = [mpmath.mpf(v) for v in params[o, 2:]]
        th = [mpmath.mpf(v) for v in x0[o]]
        h = mpmath.mpf(dt)
        for k in range(steps):
            t0, t1, t2 = th
            new = [
                t0 + h * (om[0] + Kc / 3 * (mpmath.sin(t1 - t0) + mpmath.sin(t2 - t0))) + sig * mpmath.sqrt(h) * mpmath.mpf(N[k, o, 0]),
                t1 + h * (om[1] + Kc / 3 * (mpmath.sin(t0 - t1) + mpmath.sin(t2 - t1))) + sig * mpmath.sqrt(h) * mpmath.mpf(N[k, o, 1]),
                t2 + h * (om[2] + Kc / 3 * (mpmath.sin(t0 - t2) + mpmath.sin(t1 - t2))) + sig * mpmath.sqrt(h) * mpmath.mpf(N[k, o, 2]),
            ]
            th = new
        np.testing.assert_allclose(xK[o], [float(v) for v in th], rtol=1e-14)


def test_fhn_fixed_point_is_stationary():
    # sigma = 0, c = 0: the FHN fixed point solves v - v^3/3 - w + I = 0 and
    # v + a - b w = 0, i.e. -v^3/3 + (1 - 1/b) v + (I - a/b) = 0.
    u, K, dt = 4, 500, 0.01
    params, x0 = inputs.fhn(u, 2, seed=3)
    params[:, 4] = 0.0
    params[:, 5] = 0.0
    for o in range(2):
        a, b, I = params[o, 0], params[o, 1], params[o, 3]
        roots = np.roots([-1.0 / 3.0, 0.0, 1.0 - 1.0 / b, I - a / b])
        v = float(np.real(roots[np.argmin(np.abs(np.imag(roots)))]))
        x0[o, :u] = v
        x0[o, u:] = (v + a) / b
    _, xK = oracle.integrate(_pb("fhn_net", 2 * u, dt, K), params, x0, frames=False)
    np.testing.assert_allclose(xK, x0, rtol=1e-10, atol=1e-10)


def test_fhn_uncoupled_units_are_independent():
    # c = 0, sigma = 0: each unit of a 3-unit network evolves like a 1-unit network
    K, dt = 400, 0.01
    params, x0 = inputs.fhn(3, 1, seed=5)
    params[:, 4] = 0.0
    params[:, 5] = 0.0
    _, big = oracle.integrate(_pb("fhn_net", 6, dt, K), params, x0, frames=False)
    for i in range(3):
        single = np.array([[x0[0, i], x0[0, 3 + i]]])
        _, s = oracle.integrate(_pb("fhn_net", 2, dt, K), params, single, frames=False)
        np.testing.assert_array_equal(big[0, [i, 3 + i]], s[0])


def test_fhn_coupling_conserves_v_sum_and_is_mean_field():
    # c mean(v) - c v_i sums to zero over units; and with two units the
    # coupling of unit 1 is (c / 2)(v_2 - v_1) (mean includes the unit itself).
    u, K, dt = 5, 40, 0.01
    params, x0 = inputs.fhn(u, 2, seed=6)
    params[:, 4] = 0.4
    fr, _ = oracle.integrate(_pb("fhn_net", 2 * u, dt, K, seed=3), params, x0)
    params0 = params.copy()
    params0[:, 4] = 0.0
    for k in range(K):
        # one step from the same state with c = 0: the v-sum must agree
        _, with_c = oracle.integrate(_pb("fhn_net", 2 * u, dt, K, seed=3), params, fr[k], k_begin=k, k_end=k + 1, frames=False)
        _, no_c = oracle.integrate(_pb("fhn_net", 2 * u, dt, K, seed=3), params0, fr[k], k_begin=k, k_end=k + 1, frames=False)
        np.testing.assert_array_equal(with_c, fr[k + 1])
        np.testing.assert_allclose(with_c[:, :u].sum(axis=1), no_c[:, :u].sum(axis=1), rtol=0, atol=1e-12)
        np.testing.assert_array_equal(with_c[:, u:], no_c[:, u:])
    p2, x2 = inputs.fhn(2, 1, seed=7)
    p2[:, 5] = 0.0
    pb = _pb("fhn_net", 4, dt, 1)
    _, one = oracle.integrate(pb, p2, x2, frames=False)
    p2c = p2.copy()
    p2c[:, 4] = 0.0
    _, base = oracle.integrate(pb, p2c, x2, frames=False)
    c = p2[0, 4]
    v1, v2 = x2[0, 0], x2[0, 1]
    assert one[0, 0] - base[0, 0] == pytest.approx(dt * c / 2 * (v2 - v1), rel=1e-9, abs=1e-15)


def test_fhn_epsilon_zero_freezes_w():
    params, x0 = inputs.fhn(4, 2, seed=8)
    params[:, 2] = 0.0
    fr, _ = oracle.integrate(_pb("fhn_net", 8, 0.01, 100, stride=10, seed=2), params, x0)
    for f in range(fr.shape[0]):
        np.testing.assert_array_equal(fr[f][:, 4:], x0[:, 4:])


def test_frames_resume_and_orbit_offset():
    n, orbits, K, s, dt = 9, 6, 120, 7, 0.01
    params, x0 = inputs.kuramoto(n, orbits, seed=15)
    pb = _pb("kuramoto", n, dt, K, stride=s, seed=77)
    fr, xK = oracle.integrate(pb, params, x0)
    assert fr.shape[0] == K // s + 1
    np.testing.assert_array_equal(fr[0], x0)
    for f in range(1, fr.shape[0]):
        _, xf = oracle.integrate(pb, params, x0, k_end=f * s, frames=False)
        np.testing.assert_array_equal(fr[f], xf)
    _, xj = oracle.integrate(pb, params, x0, k_end=50, frames=False)
    _, xr = oracle.integrate(pb, params, xj, k_begin=50, frames=False)
    np.testing.assert_array_equal(xr, xK)
    _, part = oracle.integrate(pb, params[3:], x0[3:], orbit_begin=3, frames=False)
    np.testing.assert_array_equal(part, xK[3:])
    _, thr = oracle.integrate(pb, params, x0, frames=False, nthreads=3)
    np.testing.assert_array_equal(thr, xK)


def test_problem_validation():
    assert oracle.lib().oracle_check_problem(oracle.make_problem("kuramoto", 4, 4, 6, 0.1, 1)) == 0
    assert oracle.lib().oracle_check_problem(oracle.make_problem("kuramoto", 4, 3, 6, 0.1, 1)) != 0
    assert oracle.lib().oracle_check_problem(oracle.make_problem("fhn_net", 6, 3, 6, 0.1, 1)) == 0
    assert oracle.lib().oracle_check_problem(oracle.make_problem("fhn_net", 5, 2, 6, 0.1, 1)) != 0
    with pytest.raises(ValueError):
        oracle.integrate(oracle.make_problem("ou", 2, 2, 2, 0.1, 10, stride=0), np.zeros((1, 2)), np.zeros((1, 2)))
