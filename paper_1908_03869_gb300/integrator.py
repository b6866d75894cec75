"""Tensor-level wrapper over one sdeb context.

Argument marshalling only: shapes and dtypes are checked, pointers and the
CUDA stream handle are passed to the C ABI, and results land in torch
tensors allocated here.  All compute runs in libsdeb.so.
"""
import ctypes

import torch

from . import (SDEB_FLAG_NO_FRAMES, SDEB_FLAG_SHARED_PARAMS, SDEB_FP64, SDEB_MEM_DEVICE, SDEB_MEM_HOST,
               SDEB_MEM_HOST_ASYNC, Problem, sdeb_autotune, sdeb_create,
               sdeb_destroy, sdeb_frame_moments, sdeb_get_layout, sdeb_grad, sdeb_integrate, sdeb_integrate_range, sdeb_orbit_flags,
               sdeb_read_final, sdeb_read_orbits, sdeb_set_adjoint_records, sdeb_set_layout, sdeb_set_params)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _mem(t, async_host):
    """SDEB_MEM_* of tensor t: device, or host waited for / only enqueued."""
    if t.is_cuda:
        return SDEB_MEM_DEVICE
    return SDEB_MEM_HOST_ASYNC if async_host else SDEB_MEM_HOST


class Integrator:
    """Owns one sdeb context.  ``Integrator(Problem.make(...))``."""

    def __init__(self, problem: Problem, user_source=None):
        """user_source: CUDA C++ of a user-defined model (problem.model =
        SDEB_USER), compiled at run time (sdeb_create_user)."""
        self.pb = problem
        self.dtype = torch.float64 if problem.precision == SDEB_FP64 else torch.float32
        self.shared = bool(problem.flags & SDEB_FLAG_SHARED_PARAMS)
        self.has_frames = not (problem.flags & SDEB_FLAG_NO_FRAMES)
        self.nframes = problem.steps // problem.stride + 1 if self.has_frames else 0
        self.ctx = None
        if user_source is not None:
            from . import sdeb_create_user
            self.ctx = sdeb_create_user(problem, user_source)
        else:
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

    def set_params(self, params: torch.Tensor, x0: torch.Tensor, stream=None, async_host=False):
        """async_host: host tensors are only enqueued for copying on the
        stream (page-locked ones overlap other streams); they must stay
        unchanged until the stream has passed the copy."""
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
        sdeb_set_params(self.ctx, _ptr(params), _ptr(x0), _mem(params, async_host), self._stream(stream))

    def set_layout(self, lanes_per_orbit, units_per_lane):
        sdeb_set_layout(self.ctx, lanes_per_orbit, units_per_lane)

    def layout(self):
        return sdeb_get_layout(self.ctx)

    def set_adjoint_records(self, mode):
        """Where grad()'s replay keeps its step records: SDEB_RECORDS_AUTO,
        _GLOBAL or _SHARED."""
        sdeb_set_adjoint_records(self.ctx, mode)

    def autotune(self, trial_steps=0, stream=None):
        """Pick the fastest lane-group layout (after set_params, before integrating)."""
        sdeb_autotune(self.ctx, trial_steps, self._stream(stream))
        return self.layout()

    def integrate(self, stream=None):
        sdeb_integrate(self.ctx, self._stream(stream))

    def integrate_range(self, k_begin, k_end, stream=None):
        sdeb_integrate_range(self.ctx, k_begin, k_end, self._stream(stream))

    def frames(self, begin=0, count=None, device="cuda", stream=None, out=None, async_host=False):
        """async_host: a host `out` is only enqueued on the stream;
        synchronise before reading it."""
        count = self.nframes - begin if count is None else count
        shape = (count, self.pb.orbits, self.pb.n)
        if out is None:
            out = torch.empty(shape, dtype=self.dtype, device=device,
                              pin_memory=(device == "cpu" and torch.cuda.is_available()))
        sdeb_read_orbits(self.ctx, _ptr(out), out.numel() * out.element_size(), begin, count,
                         _mem(out, async_host), self._stream(stream))
        return out

    def final(self, device="cuda", stream=None, out=None, async_host=False):
        if out is None:
            out = torch.empty((self.pb.orbits, self.pb.n), dtype=self.dtype, device=device)
        sdeb_read_final(self.ctx, _ptr(out), out.numel() * out.element_size(), _mem(out, async_host),
                        self._stream(stream))
        return out

    def moments(self, begin=0, count=None, state=True, order_param=False, device="cuda", stream=None):
        """FP64 ensemble moments of frames [begin, begin + count) over the
        orbits (sdeb_frame_moments): (mom [count][n][2] or None, rmom
        [count][2] or None), each pair (mean, population variance); rmom is
        that of the order parameter of Eq. 7 (phase models)."""
        count = self.nframes - begin if count is None else count
        mom = torch.empty((count, self.pb.n, 2), dtype=torch.float64, device=device) if state else None
        rmom = torch.empty((count, 2), dtype=torch.float64, device=device) if order_param else None
        kind = mom if mom is not None else rmom
        sdeb_frame_moments(self.ctx, begin, count, _ptr(mom) if mom is not None else None,
                           mom.numel() * 8 if mom is not None else 0, _ptr(rmom) if rmom is not None else None,
                           rmom.numel() * 8 if rmom is not None else 0, _mem(kind, False), self._stream(stream))
        return mom, rmom

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


class BatchIntegrator:
    """Owns one batch context (sdeb_create_batch): heterogeneous Kuramoto
    instances integrated by one persistent, graph-launched kernel."""

    def __init__(self, problems):
        from . import sdeb_create_batch
        self.pbs = list(problems)
        self.dtype = torch.float64 if self.pbs[0].precision == SDEB_FP64 else torch.float32
        self.ctx = sdeb_create_batch(self.pbs)

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

    def set_params(self, params_list, x0_list, stream=None, device="cuda"):
        """params_list[i]: [orbits_i][d_i] (or [d_i] if shared); x0_list[i]: [orbits_i][n_i]."""
        p = torch.cat([torch.as_tensor(q, dtype=self.dtype).reshape(-1) for q in params_list]).to(device)
        x = torch.cat([torch.as_tensor(q, dtype=self.dtype).reshape(-1) for q in x0_list]).to(device)
        self._keep = (p, x)
        sdeb_set_params(self.ctx, _ptr(p), _ptr(x), p.is_cuda, self._stream(stream))

    def autotune(self, stream=None):
        sdeb_autotune(self.ctx, 0, self._stream(stream))
        return self.info()

    def info(self):
        from . import sdeb_batch_info
        return sdeb_batch_info(self.ctx)

    def set_schedule(self, chain_fraction):
        from . import sdeb_batch_set_schedule
        sdeb_batch_set_schedule(self.ctx, chain_fraction)

    def layout(self, i):
        from . import sdeb_batch_layout
        return sdeb_batch_layout(self.ctx, i)

    def integrate(self, stream=None):
        sdeb_integrate(self.ctx, self._stream(stream))

    def _read(self, i, what, shape, device, stream):
        from . import sdeb_batch_read
        out = torch.empty(shape, dtype=self.dtype, device=device)
        sdeb_batch_read(self.ctx, i, what, _ptr(out), out.numel() * out.element_size(), out.is_cuda,
                        self._stream(stream))
        return out

    def frames(self, i, device="cuda", stream=None):
        pb = self.pbs[i]
        return self._read(i, 0, (pb.steps // pb.stride + 1, pb.orbits, pb.n), device, stream)

    def final(self, i, device="cuda", stream=None):
        pb = self.pbs[i]
        return self._read(i, 1, (pb.orbits, pb.n), device, stream)

    def flags(self, stream=None):
        out = torch.zeros(sum(pb.orbits for pb in self.pbs), dtype=torch.uint8)
        sdeb_orbit_flags(self.ctx, _ptr(out), self._stream(stream))
        return out
