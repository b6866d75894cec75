"""Pins of the oracle's ensemble moments (frame_moments): the mean and
population variance over orbits of every state component, and of the order
parameter r of Eq. 7 (Sec. 2.3), checked against closed forms and against
the oracle's own per-orbit order parameter (oracle.c)."""
import numpy as np

import oracle


def test_constant_and_arithmetic_sequences():
    F, M, n = 3, 10, 4
    x = np.zeros((F, M, n))
    x[0] = 2.5                                        # a constant: its value, variance 0
    x[1] = np.arange(M)[:, None] * 1.0                # 0..M-1: mean (M-1)/2, variance (M^2-1)/12
    x[2] = 1e8 + np.arange(M)[:, None] * 3.0          # shifted and scaled: variance 9 (M^2-1)/12
    mom, _ = oracle.frame_moments(x)
    assert mom.shape == (F, n, 2)
    np.testing.assert_array_equal(mom[0, :, 0], 2.5)
    np.testing.assert_array_equal(mom[0, :, 1], 0.0)
    np.testing.assert_allclose(mom[1, :, 0], (M - 1) / 2, rtol=1e-15)
    np.testing.assert_allclose(mom[1, :, 1], (M * M - 1) / 12, rtol=1e-14)
    np.testing.assert_allclose(mom[2, :, 0], 1e8 + 3 * (M - 1) / 2, rtol=1e-15)
    np.testing.assert_allclose(mom[2, :, 1], 9 * (M * M - 1) / 12, rtol=1e-9)


def test_order_parameter_closed_forms():
    n = 6
    synced = np.full((1, 5, n), 0.7)                              # r = 1 for every orbit
    splay = (2 * np.pi * np.arange(n) / n + 0.3)[None, None, :]   # r = 0
    two = np.array([[[0.0, np.pi / 2]]])                          # r = |1 + i| / 2 = 1/sqrt(2)
    _, r1 = oracle.frame_moments(synced, order_parameter=True)
    _, r0 = oracle.frame_moments(splay, order_parameter=True)
    _, r2 = oracle.frame_moments(two, order_parameter=True)
    np.testing.assert_allclose(r1[0], [1.0, 0.0], atol=1e-15)
    assert abs(r0[0, 0]) < 1e-15 and r0[0, 1] == 0.0
    np.testing.assert_allclose(r2[0, 0], 2 ** -0.5, rtol=1e-15)
    # a mix of synchronised and splay orbits: mean 1/2, variance 1/4
    mix = np.concatenate([np.full((1, 4, n), 1.1), np.broadcast_to(splay, (1, 4, n))], axis=1)
    _, rm = oracle.frame_moments(mix, order_parameter=True)
    np.testing.assert_allclose(rm[0], [0.5, 0.25], atol=1e-15)


def test_order_parameter_matches_the_oracle_per_orbit():
    rng = np.random.Generator(np.random.PCG64(5))
    th = rng.uniform(-40, 40, (2, 50, 9))
    _, rm = oracle.frame_moments(th, order_parameter=True)
    for f in range(2):
        r = np.array([oracle.order_param(th[f, o])[0] for o in range(50)])
        np.testing.assert_allclose(rm[f, 0], r.mean(), rtol=1e-14)
        np.testing.assert_allclose(rm[f, 1], r.var(), rtol=1e-12)


def test_ou_moments_against_the_exact_discrete_law():
    # Euler-Maruyama on dX = -theta X dt + sigma dW from x0: the orbit mean
    # of X^k is a^k x0 (a = 1 - theta dt) and the variance is
    # sigma^2 dt (1 - a^2k) / (1 - a^2); over M orbits the sample moments
    # lie within a few standard errors of these.
    n, M, dt, steps, stride, theta, sigma, x0v = 2, 20000, 0.05, 60, 20, 0.8, 0.5, 1.5
    pb = oracle.make_problem("ou", n, n, 2, dt, steps, stride, 3)
    p = np.tile([theta, sigma], (M, 1))
    fr, _ = oracle.integrate(pb, p, np.full((M, n), x0v), nthreads=8)
    mom, _ = oracle.frame_moments(fr)
    a = 1 - theta * dt
    for f in range(fr.shape[0]):
        k = f * stride
        mean = a ** k * x0v
        var = sigma ** 2 * dt * (1 - a ** (2 * k)) / (1 - a ** 2)
        assert np.all(np.abs(mom[f, :, 0] - mean) <= 5 * np.sqrt(var / M) + 1e-15)
        if k > 0:
            assert np.all(np.abs(mom[f, :, 1] - var) <= 5 * var * np.sqrt(2.0 / M))
        else:
            np.testing.assert_array_equal(mom[f, :, 1], 0.0)
