"""Pins of the oracle's particle swarm (oracle/swarm.py): the inertia-weight
swarm of Kennedy and Eberhart with Shi and Eberhart's inertia weight, driving
the oracle integrator over parameter sets (the population-based parameter
search of the paper's Sec. 1.2).

* Special cases with a closed form: with c1 = c2 = 0 and w = 1 every particle
  moves on a straight line, x_g = x_0 + g v_0; a swarm whose particles sit
  at their own bests, all equal, with v = 0 stays where it is.
* With w = 0 and one attraction of coefficient 1 a particle ends between
  its position and the global best (social term) or its own best
  (cognitive term).
* The global best is the least personal best, the lowest index among
  equals; a NaN fitness never improves a personal best; personal-best
  fitness never increases; positions and velocities stay in their bounds.
* The uniforms are the Philox words of counter (g, j, i, 2) mapped into
  (0, 1), distinct for every generation, dimension and particle.
* The update converges on the sphere function (the textbook test of the
  swarm): the best fitness falls below 1e-10 in 200 generations.
* The fitness: a synchronised orbit has r = 1 and a splay state r = 0 (Eq. 7),
  so f = (1 - r*)^2 and r*^2.
* A search over the coupling K of the Kuramoto model (Eq. 5/6) reaches a
  target order parameter (0.9, within 0.01) with K above Kuramoto's critical
  coupling.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import swarm
from paper_1908_03869_gb300 import inputs

W, C1, C2 = 0.7298, 1.49618, 1.49618


def _state(P, D, seed=3, lo=-5.0, hi=5.0):
    g = np.random.default_rng(seed)
    return swarm.new_state(g.uniform(lo, hi, (P, D)), g.uniform(-1.0, 1.0, (P, D)))


def test_pure_inertia_is_a_straight_line():
    st = _state(6, 3)
    x0, v0 = st["x"].copy(), st["v"].copy()
    lo, hi = [-1e6] * 3, [1e6] * 3
    for g in range(20):
        swarm.update(st, np.arange(6.0), lo, hi, 1.0, 0.0, 0.0, 7, g)
        np.testing.assert_allclose(st["x"], x0 + (g + 1) * v0, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(st["v"], v0)


def test_swarm_at_rest_at_its_best_stays():
    x = np.tile([0.5, -1.25], (5, 1))
    st = swarm.new_state(x, np.zeros_like(x))
    for g in range(5):
        b = swarm.update(st, np.full(5, 2.0), [-5, -5], [5, 5], W, C1, C2, 11, g)
        assert b == 0
        np.testing.assert_array_equal(st["x"], x)
        np.testing.assert_array_equal(st["v"], 0.0)


def test_global_best_ties_nan_and_monotone_personal_bests():
    st = _state(8, 2)
    fit = np.array([3.0, 1.0, 5.0, 0.5, 2.0, 0.5, np.nan, 9.0])
    assert swarm.update(st, fit, [-5, -5], [5, 5], W, C1, C2, 1, 0) == 3        # 0.5 at 3 and 5: lowest index
    assert np.isinf(st["pbest_fit"][6])                                          # NaN never improves
    g = np.random.default_rng(9)
    prev = st["pbest_fit"].copy()
    for gen in range(1, 40):
        fit = g.uniform(0.0, 4.0, 8)
        fit[gen % 8] = np.nan
        b = swarm.update(st, fit, [-5, -5], [5, 5], 2.0, 2.5, 2.5, 1, gen)       # aggressive coefficients
        assert np.all(st["pbest_fit"] <= prev)
        assert st["pbest_fit"][b] == np.min(st["pbest_fit"])
        assert b == int(np.flatnonzero(st["pbest_fit"] == np.min(st["pbest_fit"]))[0])
        assert np.all(st["x"] >= -5) and np.all(st["x"] <= 5)
        assert np.all(np.abs(st["v"]) <= 10)
        prev = st["pbest_fit"].copy()


def test_uniforms_are_philox_words_of_the_swarm_counter():
    r1, r2 = swarm.uniforms(5, 3, 4, 2)
    for i in range(4):
        for j in range(2):
            words = oracle.philox([3, j, i, 2], [5, 0])
            assert r1[i, j] == (float(words[0]) + 0.5) * 2.0 ** -32
            assert r2[i, j] == (float(words[1]) + 0.5) * 2.0 ** -32
    assert np.all((r1 > 0) & (r1 < 1)) and np.all((r2 > 0) & (r2 < 1))
    other = swarm.uniforms(5, 4, 4, 2)[0]
    assert len(set(r1.ravel()) | set(other.ravel())) == 16


def test_converges_on_the_sphere_function():
    st = _state(20, 2, seed=4)
    best = []
    for g in range(200):
        fit = np.sum(st["x"] ** 2, axis=1)
        b = swarm.update(st, fit, [-5, -5], [5, 5], W, C1, C2, 2, g)
        best.append(st["pbest_fit"][b])
    assert best[-1] < 1e-10
    assert all(a >= b for a, b in zip(best, best[1:]))


def test_fitness_closed_forms():
    n, R = 8, 3
    sync = np.full((2 * R, n), 1.3)
    splay = 0.4 + 2 * math.pi * np.arange(n) / n
    theta = np.vstack([sync[:R], np.tile(splay, (R, 1))])
    fit = swarm.fitness(theta, 2, R, 0.3)
    assert abs(fit[0] - 0.7 ** 2) < 1e-14
    assert abs(fit[1] - 0.3 ** 2) < 1e-14


def test_expand_sets_the_searched_columns_of_every_realisation():
    base = np.arange(10.0)
    x = np.array([[7.5, -1.0], [8.5, -2.0]])
    rows = swarm.expand(x, [0, 1], base, 3)
    assert rows.shape == (6, 10)
    for o in range(6):
        np.testing.assert_array_equal(rows[o, 2:], base[2:])
        np.testing.assert_array_equal(rows[o, :2], x[o // 3])


@pytest.mark.parametrize("target", [0.9])
def test_search_over_the_coupling_reaches_a_synchronised_target(target):
    n, R, P = 8, 4, 8
    p, x0 = inputs.kuramoto(n, R, seed=5)
    base = p[0].copy()
    base[1] = 0.05                                   # weak noise
    base[2:] = np.linspace(-0.5, 0.5, n)             # spread natural frequencies
    pb = oracle.make_problem("kuramoto", n, n, n + 2, 0.02, 500, 500, 0)
    g = np.random.default_rng(6)
    hist = swarm.search(pb, base, x0, [0], [0.0], [6.0], g.uniform(0.0, 1.0, (P, 1)), np.zeros((P, 1)), 8,
                        W, C1, C2, 12, target, nthreads=4)
    first = hist[0]["pbest_fit"].min()
    last = hist[-1]["pbest_fit"].min()
    assert last < first
    assert last < 1e-4
    # above Kuramoto's critical coupling for frequencies uniform on [-a, a],
    # K_c = 2 / (pi g(0)) = 4 a / pi, below which r stays near 0
    k_best = hist[-1]["pbest"][hist[-1]["gbest"], 0]
    assert k_best > 4 * 0.5 / math.pi


def test_attraction_moves_toward_the_right_best():
    """w = 0 and one attraction with coefficient 1: a particle moves from x
    toward its target by a fraction r in (0, 1), so it ends between them --
    the global best's position for the social term, its own best for the
    cognitive one."""
    g = np.random.default_rng(8)
    for gen in range(10):
        st = _state(6, 2, seed=gen)
        st["pbest"] = g.uniform(-5, 5, (6, 2))
        st["pbest_fit"] = g.uniform(1.0, 2.0, 6)
        x_old = st["x"].copy()
        fit = np.full(6, 10.0)                      # no personal best improves
        b = swarm.update(st, fit, [-5, -5], [5, 5], 0.0, 0.0, 1.0, 3, gen)
        tgt = np.broadcast_to(st["pbest"][b], x_old.shape)
        assert np.all((st["x"] - x_old) * (tgt - x_old) >= 0)
        assert np.all(np.abs(st["x"] - x_old) <= np.abs(tgt - x_old))
        st2 = _state(6, 2, seed=gen)
        st2["pbest"] = st["pbest"].copy()
        st2["pbest_fit"] = st["pbest_fit"].copy()
        x_old = st2["x"].copy()
        swarm.update(st2, fit, [-5, -5], [5, 5], 0.0, 1.0, 0.0, 3, gen)
        assert np.all((st2["x"] - x_old) * (st2["pbest"] - x_old) >= 0)
        assert np.all(np.abs(st2["x"] - x_old) <= np.abs(st2["pbest"] - x_old))
