"""GPU parity of the particle swarm search (sdeb_swarm_*, the SwarmSearch
driver) against the oracle's swarm (oracle/swarm.py): the population-based
parameter search of the paper's Sec. 1.2.

* expand: bit-exact (FP64; FP32 rows are the oracle's rows rounded).
* fitness: within 1e-14 of the oracle on the same states (FP64 sums of FP64
  cos/sin, summed in another order).
* update: bit-exact over 12 chained generations on the same fitness values
  (ties, NaN fitness, clamped velocities and positions included): every
  product and sum is rounded on its own in the oracle's order, and r1, r2
  are the same Philox words.
* The whole search in FP64 against the oracle's: the same global best every
  generation and bit-identical positions, velocities and personal bests
  (they depend on the fitness only through its comparisons), personal-best
  fitness within 1e-12.
* FP32: personal-best fitness never increases, the global best is the least
  (lowest index), bounds hold, and the oracle's fitness of the best
  position is within 1e-4 of the GPU's.
"""
import numpy as np
import pytest

import oracle
from oracle import swarm as oswarm
import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

pytestmark = pytest.mark.gpu
W, C1, C2 = 0.7298, 1.49618, 1.49618


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _dev(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64).cuda()


def _p(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_expand_matches_oracle(precision):
    import torch
    g = np.random.default_rng(1)
    P, R, d, dims = 37, 5, 12, [3, 0, 11]
    x = g.uniform(-3, 3, (P, len(dims)))
    base = g.uniform(-1, 1, d)
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = torch.empty((P * R, d), dtype=dt, device="cuda")
    xd, bd = _dev(x), _dev(base, dt)        # held: the caching allocator must not reuse them
    sdeb.sdeb_swarm_expand(_p(xd), P, dims, _p(bd), d, R, precision, _p(out))
    ref = oswarm.expand(x, dims, base, R)
    if precision == "fp32":
        ref = ref.astype(np.float32)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fitness_matches_oracle(precision):
    import torch
    g = np.random.default_rng(2)
    P, R, n = 45, 37, 19                    # R > 32: lanes take several realisations
    theta = g.uniform(-20, 20, (P * R, n))
    theta[:R] = 0.7                         # a synchronised particle: r = 1
    dt = torch.float64 if precision == "fp64" else torch.float32
    th = _dev(theta, dt)
    fit = torch.empty(P, dtype=torch.float64, device="cuda")
    sdeb.sdeb_swarm_fitness(_p(th), P, R, n, precision, 0.35, _p(fit))
    ref = oswarm.fitness(th.cpu().double().numpy(), P, R, 0.35)
    np.testing.assert_allclose(fit.cpu().numpy(), ref, rtol=0, atol=1e-14)
    assert abs(fit[0].item() - 0.65 ** 2) < 1e-14


def test_update_is_bit_exact_over_chained_generations():
    import torch
    g = np.random.default_rng(3)
    P, D = 1500, 3                          # more particles than threads in the block
    lo, hi = [-2.0, 0.0, -10.0], [2.0, 1.0, 10.0]
    st = oswarm.new_state(g.uniform(lo, hi, (P, D)), g.uniform(-1, 1, (P, D)))
    x, v = _dev(st["x"]), _dev(st["v"])
    pbest, pbest_fit = _dev(st["pbest"]), _dev(st["pbest_fit"])
    gbest = torch.zeros(1, dtype=torch.int32, device="cuda")
    for gen in range(12):
        fit = g.uniform(0.0, 1.0, P)
        fit[g.integers(0, P, 20)] = np.nan
        fit[100] = fit[900] = -1.0 - gen          # a tie for the global best: lowest index
        b = oswarm.update(st, fit, lo, hi, 1.2, 2.0, 2.0, 99, gen)    # aggressive: clamps fire
        fd = _dev(fit)
        sdeb.sdeb_swarm_update(_p(x), _p(v), _p(pbest), _p(pbest_fit), _p(fd), P, lo, hi, 1.2, 2.0, 2.0, 99, gen,
                               _p(gbest))
        assert int(gbest.item()) == b == 100
        np.testing.assert_array_equal(x.cpu().numpy(), st["x"])
        np.testing.assert_array_equal(v.cpu().numpy(), st["v"])
        np.testing.assert_array_equal(pbest.cpu().numpy(), st["pbest"])
        np.testing.assert_array_equal(pbest_fit.cpu().numpy(), st["pbest_fit"])
    assert np.any(st["x"] == np.asarray(hi)) and np.any(np.abs(st["v"]) == np.asarray(hi) - np.asarray(lo))


def _search_problem(precision, n=8, R=6, steps=300, dt=0.02):
    p, x0 = inputs.kuramoto(n, R, seed=7)
    base = p[0].copy()
    base[1] = 0.05
    base[2:] = np.linspace(-0.5, 0.5, n)
    pb = sdeb.Problem.make("kuramoto", n, 1, dt, steps, steps, 3, precision)
    opb = oracle.make_problem("kuramoto", n, n, n + 2, dt, steps, steps, 3)
    return pb, opb, base, x0


def test_search_fp64_matches_oracle():
    from paper_1908_03869_gb300.swarm import SwarmSearch
    P, G = 12, 6
    pb, opb, base, x0 = _search_problem("fp64")
    g = np.random.default_rng(4)
    x_init = np.column_stack([g.uniform(0.0, 3.0, P), g.uniform(0.0, 0.5, P)])
    v_init = g.uniform(-0.2, 0.2, (P, 2))
    lo, hi = [0.0, 0.0], [4.0, 0.5]
    hist = oswarm.search(opb, base, x0, [0, 1], lo, hi, x_init, v_init, G, W, C1, C2, 21, 0.8, nthreads=4)
    with SwarmSearch(pb, base, x0, [0, 1], lo, hi, P, W, C1, C2, r_target=0.8, swarm_seed=21) as s:
        s.reset(x_init, v_init)
        for gen in range(G):
            s.step()
            h = hist[gen]
            assert int(s.gbest.item()) == h["gbest"], gen
            np.testing.assert_allclose(s.fit.cpu().numpy(), h["fit"], rtol=0, atol=1e-12)
            np.testing.assert_array_equal(s.x.cpu().numpy(), h["x"])
            np.testing.assert_array_equal(s.v.cpu().numpy(), h["v"])
            np.testing.assert_array_equal(s.pbest.cpu().numpy(), h["pbest"])
            np.testing.assert_allclose(s.pbest_fit.cpu().numpy(), h["pbest_fit"], rtol=0, atol=1e-12)


def test_search_fp32_properties():
    from paper_1908_03869_gb300.swarm import SwarmSearch
    P, G, R = 64, 10, 8
    pb, opb, base, x0 = _search_problem("fp32", R=R)
    g = np.random.default_rng(5)
    lo, hi = [0.0], [6.0]
    x0 = x0.astype(np.float32).astype(np.float64)
    base = base.astype(np.float32).astype(np.float64)
    with SwarmSearch(pb, base, x0, [0], lo, hi, P, W, C1, C2, r_target=0.9, swarm_seed=5) as s:
        s.reset(g.uniform(0.0, 1.0, (P, 1)), np.zeros((P, 1)))
        prev = np.full(P, np.inf)
        first = None
        for gen in range(G):
            s.step()
            pf = s.pbest_fit.cpu().numpy()
            assert np.all(pf <= prev)
            b = int(s.gbest.item())
            assert b == int(np.flatnonzero(pf == pf.min())[0])
            xs = s.x.cpu().numpy()
            assert np.all(xs >= 0.0) and np.all(xs <= 6.0)
            first = pf.min() if first is None else first
            prev = pf
        pos, fbest = s.best()
        b = int(s.gbest.item())
    assert fbest < first
    # the best position was scored by particle b, on orbits b R .. b R + R - 1
    params = oswarm.expand(np.float32(pos)[None, :].astype(np.float64), [0], base, R)
    _, fin = oracle.integrate(opb, params, x0, orbit_begin=b * R, frames=False)
    ref = oswarm.fitness(fin, 1, R, 0.9)[0]
    assert abs(ref - fbest) < 1e-4


def test_single_particle_single_realisation():
    """P = R = D = 1: the particle is its own global best; its cognitive and
    social pulls coincide."""
    from paper_1908_03869_gb300.swarm import SwarmSearch
    pb, opb, base, x0 = _search_problem("fp64", R=1, steps=100)
    hist = oswarm.search(opb, base, x0, [0], [0.0], [4.0], [[1.5]], [[0.3]], 4, W, C1, C2, 8, 0.5)
    with SwarmSearch(pb, base, x0, [0], [0.0], [4.0], 1, W, C1, C2, r_target=0.5, swarm_seed=8) as s:
        s.reset([[1.5]], [[0.3]])
        for gen in range(4):
            s.step()
            assert int(s.gbest.item()) == 0
            np.testing.assert_array_equal(s.x.cpu().numpy(), hist[gen]["x"])
            np.testing.assert_array_equal(s.v.cpu().numpy(), hist[gen]["v"])
