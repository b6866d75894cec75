"""Tensor-level wrapper over one sdeb context.

Argument marshalling only: shapes and dtypes are checked, pointers and the
CUDA stream handle are passed to the C ABI, and results land in torch
tensors allocated here.  All compute runs in libsdeb.so.
"""
import ctypes

import torch

from . import (SDEB_FLAG_NO_FRAMES, SDEB_FLAG_SHARED_PARAMS, SDEB_FP64, Problem, sdeb_autotune, sdeb_create,
               sdeb_destroy, sdeb_get_layout, sdeb_grad, sdeb_integrate, sdeb_integrate_range, sdeb_orbit_flags,
               sdeb_read_final, sdeb_read_orbits, sdeb_set_layout, sdeb_set_params)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Integrator:
    """Owns one sdeb context.  ``Integrator(Problem.make(...))``."""

    def __init__(self, problem: Problem):
        self.pb = problem
        self.dtype = torch.float64 if problem.precision == SDEB_FP64 else torch.float32
        self.shared = bool(problem.flags & SDEB_FLAG_SHARED_PARAMS)
        self.has_frames = not (problem.flags & SDEB_FLAG_NO_FRAMES)
        self.nframes = problem.steps // problem.stride + 1 if self.has_frames else 0
        self.ctx = sdeb_create(problem)

    def close(self):
        if self.ctx is not None:
            sdeb_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        if stream is None:
            return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        return getattr(stream, "cuda_stream", stream)

    def set_params(self, params: torch.Tensor, x0: torch.Tensor, stream=None):
        pb = self.pb
        want_p = (pb.d,) if self.shared else (pb.orbits, pb.d)
        if tuple(params.shape) != want_p or tuple(x0.shape) != (pb.orbits, pb.n):
            raise ValueError("params %s / x0 %s, expected %s / %s" % (tuple(params.shape), tuple(x0.shape),
                                                                     want_p, (pb.orbits, pb.n)))
        if params.dtype != self.dtype or x0.dtype != self.dtype:
            raise TypeError("params and x0 must be %s" % self.dtype)
        if params.is_cuda != x0.is_cuda:
            raise ValueError("params and x0 must both be host or both be device tensors")
        params, x0 = params.contiguous(), x0.contiguous()
        self._keep = (params, x0)  # device copies are stream-ordered: keep the sources alive
        sdeb_set_params(self.ctx, _ptr(params), _ptr(x0), params.is_cuda, self._stream(stream))

    def set_layout(self, lanes_per_orbit, units_per_lane):
        sdeb_set_layout(self.ctx, lanes_per_orbit, units_per_lane)

    def layout(self):
        return sdeb_get_layout(self.ctx)

    def autotune(self, trial_steps=0, stream=None):
        """Pick the fastest lane-group layout (after set_params, before integrating)."""
        sdeb_autotune(self.ctx, trial_steps, self._stream(stream))
        return self.layout()

    def integrate(self, stream=None):
        sdeb_integrate(self.ctx, self._stream(stream))

    def integrate_range(self, k_begin, k_end, stream=None):
        sdeb_integrate_range(self.ctx, k_begin, k_end, self._stream(stream))

    def frames(self, begin=0, count=None, device="cuda", stream=None, out=None):
        count = self.nframes - begin if count is None else count
        shape = (count, self.pb.orbits, self.pb.n)
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=device,
                              pin_memory=(device == "cpu" and torch.cuda.is_available()))
        sdeb_read_orbits(self.ctx, _ptr(out), out.numel() * out.element_size(), begin, count, out.is_cuda,
                         self._stream(stream))
        return out

    def final(self, device="cuda", stream=None, out=None):
        if out is None:
            out = torch.empty((self.pb.orbits, self.pb.n), dtype=self.dtype, device=device)
        sdeb_read_final(self.ctx, _ptr(out), out.numel() * out.element_size(), out.is_cuda, self._stream(stream))
        return out

    def flags(self, stream=None):
        out = torch.zeros(self.pb.orbits, dtype=torch.uint8)
        sdeb_orbit_flags(self.ctx, _ptr(out), self._stream(stream))
        return out

    def grad(self, dL_dxK: torch.Tensor, want_dx0=True, stream=None):
        pb = self.pb
        dL_dxK = dL_dxK.to(self.dtype).contiguous()
        dp = torch.empty((pb.d,) if self.shared else (pb.orbits, pb.d), dtype=self.dtype, device=dL_dxK.device)
        dx0 = torch.empty((pb.orbits, pb.n), dtype=self.dtype, device=dL_dxK.device) if want_dx0 else None
        sdeb_grad(self.ctx, _ptr(dL_dxK), _ptr(dp), _ptr(dx0) if dx0 is not None else None, self._stream(stream))
        return dp, dx0
