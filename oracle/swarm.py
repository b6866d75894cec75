"""Particle swarm search over model parameters, plain numpy: the
population-based parameter optimisation the paper builds its integrator for
(Sec. 1.2: an EA or a particle swarm integrates the model over every
parameter set of its population each generation, with several realisations
per set to average out the noise).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import this module.  It uses the
oracle's own integrator, Philox and order parameter and nothing of the CUDA
library.

The swarm is the inertia-weight particle swarm optimiser (Kennedy and
Eberhart 1995; the inertia weight w of Shi and Eberhart 1998), minimising a
fitness.  One generation g, after the fitness f_i of every particle i:
  1. personal bests: where f_i < pbest_f_i, pbest_i = x_i and pbest_f_i = f_i
     (a NaN fitness never improves);
  2. global best b: the least pbest_f, the lowest index among equals;
  3. for every particle i and dimension j, with r1, r2 uniform in (0, 1):
       v_ij = w v_ij + c1 r1 (pbest_ij - x_ij) + c2 r2 (pbest_bj - x_ij),
       v_ij clamped to [-vmax_j, vmax_j] with vmax_j = hi_j - lo_j,
       x_ij = x_ij + v_ij clamped to [lo_j, hi_j].
r1 and r2 are the first two words of Philox4x32-10 (key = the swarm seed)
at counter (g, j, i, 2), each mapped to (w + 1/2) 2^-32 -- the generator and
the uniform map of the noise (Sec. 2.1.2), on counter stream 2.

The fitness of a parameter set is the Kuramoto order parameter of Eq. 7 at
the end of the horizon, averaged over its R realisations:
f = (mean_q r(theta_q(T)) - r_target)^2.  Particle i's realisation q is orbit
i R + q; its parameter row is the base row with column dims[j] set to x_ij.
"""
import numpy as np

from . import integrate as _integrate
from . import order_param as _order_param
from . import philox_fill as _philox_fill
from . import uniform as _uniform


def expand(x, dims, base, realisations):
    """Per-orbit parameter rows [P * R][d] of the particles x [P][D]."""
    x = np.asarray(x, dtype=np.float64)
    base = np.asarray(base, dtype=np.float64)
    rows = np.empty((x.shape[0] * realisations, base.size))
    for i in range(x.shape[0]):
        row = base.copy()
        for j, c in enumerate(dims):
            row[c] = x[i, j]
        for q in range(realisations):
            rows[i * realisations + q] = row
    return rows


def fitness(theta, particles, realisations, r_target):
    """(mean over each particle's realisations of r(T) - r_target)^2."""
    theta = np.asarray(theta, dtype=np.float64)
    fit = np.empty(particles)
    for i in range(particles):
        acc = 0.0
        for q in range(realisations):
            acc += _order_param(theta[i * realisations + q])[0]
        fit[i] = (acc / realisations - r_target) ** 2
    return fit


def uniforms(seed, generation, particles, dims):
    """r1, r2 [P][D] of generation g: Philox words 0 and 1 at (g, j, i, 2)."""
    words = _philox_fill(seed, generation, 1, 0, dims, 0, particles, stream=2)[0]   # [D][P][4]
    r1 = np.empty((particles, dims))
    r2 = np.empty((particles, dims))
    for i in range(particles):
        for j in range(dims):
            r1[i, j] = _uniform(words[j, i, 0])
            r2[i, j] = _uniform(words[j, i, 1])
    return r1, r2


def update(state, fit, lo, hi, w, c1, c2, seed, generation):
    """One generation's update of state = dict(x, v, pbest, pbest_fit) in
    place, after the fitness `fit`; returns the global best index."""
    x, v, pbest, pbest_fit = state["x"], state["v"], state["pbest"], state["pbest_fit"]
    particles, dims = x.shape
    for i in range(particles):
        if fit[i] < pbest_fit[i]:
            pbest[i] = x[i]
            pbest_fit[i] = fit[i]
    b = 0
    for i in range(1, particles):
        if pbest_fit[i] < pbest_fit[b]:
            b = i
    r1, r2 = uniforms(seed, generation, particles, dims)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    vmax = hi - lo
    for i in range(particles):
        for j in range(dims):
            a = w * v[i, j]
            cog = (c1 * r1[i, j]) * (pbest[i, j] - x[i, j])
            soc = (c2 * r2[i, j]) * (pbest[b, j] - x[i, j])
            vn = min(max((a + cog) + soc, -vmax[j]), vmax[j])
            v[i, j] = vn
            x[i, j] = min(max(x[i, j] + vn, lo[j]), hi[j])
    return b


def new_state(x_init, v_init):
    x = np.array(x_init, dtype=np.float64)
    return {"x": x, "v": np.array(v_init, dtype=np.float64), "pbest": x.copy(),
            "pbest_fit": np.full(x.shape[0], np.inf)}


def search(pb, base, x0, dims, lo, hi, x_init, v_init, generations, w, c1, c2, swarm_seed, r_target,
           nthreads=1):
    """The whole search: every generation integrates the P R orbits of
    problem pb (the oracle problem; realisation q of every particle starts at
    x0[q]), takes their fitness and updates the swarm.  Returns the list of
    per-generation records (fit, x, v, pbest, pbest_fit, gbest) after each
    update."""
    state = new_state(x_init, v_init)
    particles = state["x"].shape[0]
    realisations = np.asarray(x0).shape[0]
    x0_all = np.tile(np.asarray(x0, dtype=np.float64), (particles, 1))
    history = []
    for g in range(generations):
        params = expand(state["x"], dims, base, realisations)
        _, fin = _integrate(pb, params, x0_all, frames=False, nthreads=nthreads)
        fit = fitness(fin, particles, realisations, r_target)
        b = update(state, fit, lo, hi, w, c1, c2, swarm_seed, g)
        history.append({"fit": fit, "x": state["x"].copy(), "v": state["v"].copy(),
                        "pbest": state["pbest"].copy(), "pbest_fit": state["pbest_fit"].copy(), "gbest": b})
    return history
