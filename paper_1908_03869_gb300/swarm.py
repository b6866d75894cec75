"""Particle swarm search over a model's parameters, every generation on the
GPU: the population-based parameter optimisation the paper builds the
integrator for (Sec. 1.2).

A generation, all on one CUDA stream with nothing read back in between:
sdeb_swarm_expand writes the per-orbit parameter rows of the P particles'
R realisations, the context integrates the P R orbits from the same R
initial states (realisation q of every particle starts at x0[q]; the noise
of orbit i R + q is its own Philox stream), sdeb_swarm_fitness takes the
order parameter of Eq. 7 at the end of the horizon, and sdeb_swarm_update
moves the swarm.  Argument marshalling only: all compute runs in
libsdeb.so.
"""
import ctypes

import torch

from . import (SDEB_FP64, Problem, sdeb_swarm_expand, sdeb_swarm_fitness, sdeb_swarm_update)
from .integrator import Integrator

# Inertia and acceleration coefficients of the constricted swarm (Clerc and
# Kennedy's chi = 0.7298 with phi = 4.1, in inertia-weight form).
DEFAULT_W, DEFAULT_C1, DEFAULT_C2 = 0.7298, 1.49618, 1.49618


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class SwarmSearch:
    """problem: a Problem for one particle's realisations' shape (model, n,
    dt, steps, precision, seed; its orbits field is replaced by P R and its
    frames are switched off).  base: [d] parameter row; dims: the searched
    columns; lo, hi: their bounds; x0: [R][n] initial states."""

    def __init__(self, problem, base, x0, dims, lo, hi, particles, w=DEFAULT_W, c1=DEFAULT_C1, c2=DEFAULT_C2,
                 r_target=0.5, swarm_seed=1):
        from . import SDEB_FLAG_NO_FRAMES
        self.R = int(x0.shape[0])
        self.P = int(particles)
        self.dims = [int(c) for c in dims]
        self.lo, self.hi = [float(t) for t in lo], [float(t) for t in hi]
        self.w, self.c1, self.c2 = float(w), float(c1), float(c2)
        self.r_target = float(r_target)
        self.swarm_seed = int(swarm_seed)
        pb = Problem.from_buffer_copy(problem)
        pb.orbits = self.P * self.R
        pb.flags |= SDEB_FLAG_NO_FRAMES
        self.pb = pb
        self.precision = "fp64" if pb.precision == SDEB_FP64 else "fp32"
        dt = torch.float64 if pb.precision == SDEB_FP64 else torch.float32
        dev = torch.device("cuda")
        self.base = torch.as_tensor(base, dtype=dt).to(dev).contiguous()
        self.x0_all = torch.as_tensor(x0, dtype=dt).to(dev).repeat(self.P, 1).contiguous()
        self.params = torch.empty((pb.orbits, pb.d), dtype=dt, device=dev)
        self.final = torch.empty((pb.orbits, pb.n), dtype=dt, device=dev)
        D = len(self.dims)
        f64 = dict(dtype=torch.float64, device=dev)
        self.x = torch.zeros((self.P, D), **f64)
        self.v = torch.zeros((self.P, D), **f64)
        self.pbest = torch.zeros((self.P, D), **f64)
        self.pbest_fit = torch.full((self.P,), float("inf"), **f64)
        self.fit = torch.zeros((self.P,), **f64)
        self.gbest = torch.zeros((1,), dtype=torch.int32, device=dev)
        self.generation = 0
        self.it = Integrator(pb)

    def close(self):
        self.it.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self, x_init, v_init):
        """Start a search from positions x_init and velocities v_init [P][D]."""
        self.x.copy_(torch.as_tensor(x_init, dtype=torch.float64))
        self.v.copy_(torch.as_tensor(v_init, dtype=torch.float64))
        self.pbest.copy_(self.x)
        self.pbest_fit.fill_(float("inf"))
        self.generation = 0

    def step(self, stream=None):
        """One generation (asynchronous on `stream`, default the current one)."""
        s = stream if stream is not None else torch.cuda.current_stream()
        sdeb_swarm_expand(_ptr(self.x), self.P, self.dims, _ptr(self.base), self.pb.d, self.R, self.precision,
                          _ptr(self.params), s)
        self.it.set_params(self.params, self.x0_all, stream=s)
        self.it.integrate(stream=s)
        self.it.final(stream=s, out=self.final)
        sdeb_swarm_fitness(_ptr(self.final), self.P, self.R, self.pb.n, self.precision, self.r_target,
                           _ptr(self.fit), s)
        sdeb_swarm_update(_ptr(self.x), _ptr(self.v), _ptr(self.pbest), _ptr(self.pbest_fit), _ptr(self.fit),
                          self.P, self.lo, self.hi, self.w, self.c1, self.c2, self.swarm_seed, self.generation,
                          _ptr(self.gbest), s)
        self.generation += 1

    def best(self):
        """(position [D], fitness) of the global best (synchronises)."""
        b = int(self.gbest.item())
        return self.pbest[b].cpu().numpy(), float(self.pbest_fit[b].item())
