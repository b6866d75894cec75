"""Shared helpers of the GPU parity tests: run one problem through the C ABI
(via the tensor wrapper) and through the CPU oracle on identical inputs."""
import os

import numpy as np

import oracle
import paper_1908_03869_gb300 as sdeb

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def max_rel_err(x, ref):
    """Reading of "max relative error": max |x - ref| / max(|ref|, 1)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert x.shape == ref.shape, (x.shape, ref.shape)
    if x.size == 0:
        return 0.0
    return float(np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)))


def np_dtype(precision):
    return np.float64 if precision == "fp64" else np.float32


def run_gpu(model, n, params, x0, dt, steps, stride, seed=0, precision="fp64", orbit_offset=0,
            shared=False, no_frames=False, ranges=None, ckpt_every=0, milstein=False, layout=None, rk4=False,
            implicit=None):
    """Returns (frames or None, final) as numpy arrays in the context precision."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    orbits = x0.shape[0]
    pb = sdeb.Problem.make(model, n, orbits, dt, steps, stride, seed, precision, orbit_offset=orbit_offset,
                           shared_params=shared, no_frames=no_frames, ckpt_every=ckpt_every, milstein=milstein,
                           rk4=rk4, implicit=implicit)
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    with Integrator(pb) as it:
        if layout is not None:
            it.set_layout(*layout)
        it.set_params(torch.as_tensor(params, dtype=dt_t).cuda(), torch.as_tensor(x0, dtype=dt_t).cuda())
        if ranges is None:
            it.integrate()
        else:
            for kb, ke in ranges:
                it.integrate_range(kb, ke)
        fr = None if no_frames else it.frames().cpu().numpy()
        fin = it.final().cpu().numpy()
        torch.cuda.synchronize()
    return fr, fin


def run_oracle(model, n, params, x0, dt, steps, stride, seed=0, orbit_offset=0, shared=False,
               mean_field=False, orbits=None, milstein=False, rk4=False, implicit=None):
    """Oracle on the same inputs (cast to float64).  orbits: optional index
    subset (global orbit index = orbit_offset + index)."""
    m, d = sdeb.model_shape(model, n)
    pb = oracle.make_problem(model, n, m, d, dt, steps, stride, seed, shared_params=shared,
                             mean_field=mean_field, milstein=milstein, rk4=rk4, implicit=implicit)
    params = np.asarray(params, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64)
    if orbits is None:
        return oracle.integrate(pb, params, x0, orbit_begin=orbit_offset, nthreads=NTHREADS)
    frs, fins = [], []
    for o in orbits:
        p = params if shared else params[o:o + 1]
        fr, fin = oracle.integrate(pb, p, x0[o:o + 1], orbit_begin=orbit_offset + int(o), nthreads=1)
        frs.append(fr)
        fins.append(fin)
    return np.concatenate(frs, axis=1), np.concatenate(fins, axis=0)
