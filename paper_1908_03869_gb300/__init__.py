"""Many-orbit Euler-Maruyama integration of Ito SDEs on GB300 (sm_103a).

Thin ctypes binding of the C ABI in include/sdeb.h: every ``sdeb_*``
function here has the C entry point's name and arguments and only marshals
them; all work runs in the CUDA library ``_build/libsdeb.so``.  A missing
library is an error (there is no CPU fallback).  PyTorch is used only for
device memory and streams (``torch.Tensor.data_ptr()`` / ``cuda_stream``).

Build the library with ``paper_1908_03869_gb300.build.build()`` (or
``__graft_entry__.build()``).
"""
import ctypes
import os

from . import build as _build

__all__ = [
    "SdebError", "Problem", "lib", "library_path",
    "SDEB_OK", "SDEB_EINVAL", "SDEB_ENOMEM", "SDEB_ECUDA", "SDEB_ETIMEOUT", "SDEB_ESTATE",
    "SDEB_EUNSUPPORTED", "SDEB_ENONFINITE", "SDEB_EBOUNDS", "sdeb_check_status", "sdeb_check_selftest",
    "SDEB_KURAMOTO", "SDEB_KURAMOTO_PAPER", "SDEB_FHN_NET", "SDEB_OU", "SDEB_GBM", "SDEB_LINEAR_ODE",
    "SDEB_USER", "SDEB_USER_MAX_N", "SDEB_USER_MAX_M", "sdeb_create_user",
    "SDEB_FP32_KAHAN", "SDEB_FP64", "SDEB_FLAG_SHARED_PARAMS", "SDEB_FLAG_NO_FRAMES", "SDEB_FLAG_MILSTEIN",
    "SDEB_FLAG_RK4", "SDEB_FLAG_IMPLICIT_EULER", "SDEB_FLAG_IMPLICIT_MIDPOINT",
    "sdeb_create", "sdeb_destroy", "sdeb_set_params", "sdeb_integrate", "sdeb_integrate_range",
    "sdeb_read_orbits", "sdeb_read_final", "sdeb_frame_moments", "sdeb_grad", "sdeb_orbit_flags", "sdeb_frames_device_ptr",
    "sdeb_last_error", "sdeb_status_string", "sdeb_philox_fill", "sdeb_normals_fill", "sdeb_order_param",
    "sdeb_integrate_noalloc", "sdeb_pipe_rate", "sdeb_set_layout", "sdeb_get_layout", "sdeb_get_checkpoint_interval",
    "sdeb_set_adjoint_records", "SDEB_RECORDS_AUTO", "SDEB_RECORDS_GLOBAL", "SDEB_RECORDS_SHARED", "sdeb_autotune", "sdeb_create_batch", "sdeb_batch_read",
    "sdeb_batch_info", "sdeb_batch_layout", "sdeb_batch_set_schedule", "sdeb_batch_plan", "model_shape",
    "sdeb_swarm_expand", "sdeb_swarm_fitness", "sdeb_swarm_update", "SDEB_SWARM_MAX_DIMS", "PIPES",
    "SDEB_MEM_HOST", "SDEB_MEM_DEVICE", "SDEB_MEM_HOST_ASYNC",
    "EXPORTED_SYMBOLS",
]

SDEB_OK, SDEB_EINVAL, SDEB_ENOMEM, SDEB_ECUDA, SDEB_ETIMEOUT, SDEB_ESTATE, SDEB_EUNSUPPORTED, SDEB_ENONFINITE, \
    SDEB_EBOUNDS = range(9)
SDEB_KURAMOTO, SDEB_KURAMOTO_PAPER, SDEB_FHN_NET, SDEB_OU, SDEB_GBM, SDEB_LINEAR_ODE, SDEB_USER = range(1, 8)
SDEB_USER_MAX_N = SDEB_USER_MAX_M = 64
SDEB_FP32_KAHAN, SDEB_FP64 = 0, 1
SDEB_FLAG_SHARED_PARAMS, SDEB_FLAG_NO_FRAMES, SDEB_FLAG_MILSTEIN, SDEB_FLAG_RK4 = 1, 2, 4, 8
SDEB_FLAG_IMPLICIT_EULER, SDEB_FLAG_IMPLICIT_MIDPOINT = 16, 32
SDEB_SWARM_MAX_DIMS = 16
SDEB_MEM_HOST, SDEB_MEM_DEVICE, SDEB_MEM_HOST_ASYNC = 0, 1, 2
SDEB_RECORDS_AUTO, SDEB_RECORDS_GLOBAL, SDEB_RECORDS_SHARED = 0, 1, 2
IMPLICIT_FLAGS = {None: 0, "euler": SDEB_FLAG_IMPLICIT_EULER, "midpoint": SDEB_FLAG_IMPLICIT_MIDPOINT}

MODEL_IDS = {
    "kuramoto": SDEB_KURAMOTO, "kuramoto_paper": SDEB_KURAMOTO_PAPER, "fhn_net": SDEB_FHN_NET,
    "ou": SDEB_OU, "gbm": SDEB_GBM, "linear_ode": SDEB_LINEAR_ODE, "user": SDEB_USER,
}
PRECISIONS = {"fp32": SDEB_FP32_KAHAN, "fp64": SDEB_FP64}


def model_shape(model, n):
    """(m, d) of a model for n states (the rule sdeb_create enforces)."""
    model = MODEL_IDS.get(model, model)
    return {
        SDEB_KURAMOTO: (n, n + 2), SDEB_KURAMOTO_PAPER: (n, 2 * n + 1), SDEB_FHN_NET: (n // 2, 6),
        SDEB_OU: (n, 2), SDEB_GBM: (n, 2), SDEB_LINEAR_ODE: (0, 1),
    }[model]


class Problem(ctypes.Structure):
    """sdeb_problem (include/sdeb.h)."""
    _fields_ = [
        ("model", ctypes.c_int32), ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("d", ctypes.c_int32),
        ("orbits", ctypes.c_int64), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
        ("steps", ctypes.c_int64), ("stride", ctypes.c_int64), ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("ckpt_every", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32), ("orbit_offset", ctypes.c_int64),
    ]

    @classmethod
    def make(cls, model, n, orbits, dt, steps, stride=1, seed=0, precision="fp32", t0=0.0, ckpt_every=0,
             shared_params=False, no_frames=False, orbit_offset=0, m=None, d=None, milstein=False, rk4=False,
             implicit=None):
        """implicit: None, "euler" or "midpoint" (the implicit ODE schemes)."""
        mid = MODEL_IDS.get(model, model)
        if mid == SDEB_USER:
            if m is None or d is None:
                raise ValueError("a user-defined model needs m and d")
            m0, d0 = m, d
        else:
            m0, d0 = model_shape(mid, n) if mid in MODEL_IDS.values() else (0, 0)
        flags = (SDEB_FLAG_SHARED_PARAMS if shared_params else 0) | (SDEB_FLAG_NO_FRAMES if no_frames else 0) | \
            (SDEB_FLAG_MILSTEIN if milstein else 0) | (SDEB_FLAG_RK4 if rk4 else 0) | IMPLICIT_FLAGS[implicit]
        return cls(mid, n, m0 if m is None else m, d0 if d is None else d, orbits, t0, dt, steps, stride,
                   seed & 0xFFFFFFFFFFFFFFFF, PRECISIONS.get(precision, precision), ckpt_every, flags, 0,
                   orbit_offset)


class SdebError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (status %d: %s)" % (message, status, _STATUS_NAMES.get(status, "?")))
        self.status = status


_STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ESTATE",
                 6: "EUNSUPPORTED", 7: "ENONFINITE", 8: "EBOUNDS"}

_P = ctypes.c_void_p
_ST = ctypes.c_int
_SIGS = {
    "sdeb_create": (_ST, [ctypes.POINTER(Problem), ctypes.POINTER(_P)]),
    "sdeb_destroy": (None, [_P]),
    "sdeb_set_params": (_ST, [_P, _P, _P, ctypes.c_int32, _P]),
    "sdeb_integrate": (_ST, [_P, _P]),
    "sdeb_integrate_range": (_ST, [_P, ctypes.c_int64, ctypes.c_int64, _P]),
    "sdeb_read_orbits": (_ST, [_P, _P, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _P]),
    "sdeb_read_final": (_ST, [_P, _P, ctypes.c_size_t, ctypes.c_int32, _P]),
    "sdeb_frame_moments": (_ST, [_P, ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_size_t, _P, ctypes.c_size_t,
                                 ctypes.c_int32, _P]),
    "sdeb_grad": (_ST, [_P, _P, _P, _P, _P]),
    "sdeb_orbit_flags": (_ST, [_P, _P, _P]),
    "sdeb_frames_device_ptr": (_ST, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]),
    "sdeb_last_error": (ctypes.c_char_p, [_P]),
    "sdeb_status_string": (ctypes.c_char_p, [_ST]),
    "sdeb_philox_fill": (_ST, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64,
                               ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint32, _P, _P]),
    "sdeb_normals_fill": (_ST, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64,
                                ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "sdeb_order_param": (_ST, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "sdeb_integrate_noalloc": (_ST, [ctypes.POINTER(Problem), _P, _P, _P, _P, _P]),
    "sdeb_pipe_rate": (_ST, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P]),
    "sdeb_check_status": (_ST, [ctypes.POINTER(ctypes.c_uint64)]),
    "sdeb_check_selftest": (_ST, [_P]),
    "sdeb_set_layout": (_ST, [_P, ctypes.c_int32, ctypes.c_int32]),
    "sdeb_get_layout": (_ST, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "sdeb_get_checkpoint_interval": (_ST, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "sdeb_set_adjoint_records": (_ST, [_P, ctypes.c_int32]),
    "sdeb_autotune": (_ST, [_P, ctypes.c_int64, _P]),
    "sdeb_create_batch": (_ST, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "sdeb_create_user": (_ST, [_P, ctypes.c_char_p, ctypes.POINTER(_P)]),
    "sdeb_batch_read": (_ST, [_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, ctypes.c_int32, _P]),
    "sdeb_batch_info": (_ST, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32)]),
    "sdeb_batch_set_schedule": (_ST, [_P, ctypes.c_double]),
    "sdeb_batch_layout": (_ST, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "sdeb_batch_plan": (_ST, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P,
                              _P, ctypes.POINTER(ctypes.c_int32)]),
    "sdeb_swarm_expand": (_ST, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, _P, _P]),
    "sdeb_swarm_fitness": (_ST, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                 _P, _P]),
    "sdeb_swarm_update": (_ST, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, _P, _P]),
}
EXPORTED_SYMBOLS = tuple(_SIGS)

_lib = None


def library_path():
    """libsdeb.so, or the bounds-checked libsdeb_checked.so when the
    environment variable SDEB_LIBRARY is "checked"."""
    return _build.CHECKED_LIB_PATH if os.environ.get("SDEB_LIBRARY") == "checked" else _build.LIB_PATH


def lib():
    """Load libsdeb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError("CUDA library %s is missing; run paper_1908_03869_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != SDEB_OK:
        msg = lib().sdeb_last_error(ctx)
        raise SdebError(status, msg.decode() if msg else "")


def _stream(stream):
    """Accept None, an int handle, or a torch.cuda.Stream."""
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def sdeb_create(problem):
    ctx = _P()
    _check(lib().sdeb_create(ctypes.byref(problem), ctypes.byref(ctx)))
    return ctx


def sdeb_destroy(ctx):
    lib().sdeb_destroy(ctx)


def sdeb_set_params(ctx, params, x0, on_device, stream=None):
    _check(lib().sdeb_set_params(ctx, params, x0, int(on_device), _stream(stream)), ctx)


def sdeb_integrate(ctx, stream=None):
    _check(lib().sdeb_integrate(ctx, _stream(stream)), ctx)


def sdeb_integrate_range(ctx, k_begin, k_end, stream=None):
    _check(lib().sdeb_integrate_range(ctx, k_begin, k_end, _stream(stream)), ctx)


def sdeb_read_orbits(ctx, dst, dst_bytes, frame_begin, frame_count, dst_on_device, stream=None):
    _check(lib().sdeb_read_orbits(ctx, dst, dst_bytes, frame_begin, frame_count, int(dst_on_device),
                                  _stream(stream)), ctx)


def sdeb_read_final(ctx, dst, dst_bytes, dst_on_device, stream=None):
    _check(lib().sdeb_read_final(ctx, dst, dst_bytes, int(dst_on_device), _stream(stream)), ctx)


def sdeb_frame_moments(ctx, frame_begin, frame_count, mom, mom_bytes, rmom, rmom_bytes, dst_on_device, stream=None):
    _check(lib().sdeb_frame_moments(ctx, frame_begin, frame_count, mom, mom_bytes, rmom, rmom_bytes,
                                    int(dst_on_device), _stream(stream)), ctx)


def sdeb_grad(ctx, dL_dxK, dL_dp, dL_dx0=None, stream=None):
    _check(lib().sdeb_grad(ctx, dL_dxK, dL_dp, dL_dx0, _stream(stream)), ctx)


def sdeb_orbit_flags(ctx, dst, stream=None):
    _check(lib().sdeb_orbit_flags(ctx, dst, _stream(stream)), ctx)


def sdeb_frames_device_ptr(ctx):
    p, b = _P(), ctypes.c_size_t()
    _check(lib().sdeb_frames_device_ptr(ctx, ctypes.byref(p), ctypes.byref(b)), ctx)
    return p.value, b.value


def sdeb_set_layout(ctx, lanes_per_orbit, units_per_lane):
    _check(lib().sdeb_set_layout(ctx, lanes_per_orbit, units_per_lane), ctx)


def sdeb_autotune(ctx, trial_steps=0, stream=None):
    _check(lib().sdeb_autotune(ctx, trial_steps, _stream(stream)), ctx)


def sdeb_create_user(problem, source):
    """Context for a user-defined model (problem.model = SDEB_USER): `source`
    defines sdeb_drift and sdeb_diffusion in CUDA C++ (include/sdeb.h)."""
    ctx = _P()
    _check(lib().sdeb_create_user(ctypes.byref(problem), source.encode() if isinstance(source, str) else source,
                                  ctypes.byref(ctx)))
    return ctx


def sdeb_create_batch(problems):
    """problems: a sequence of Problem (or a ctypes array of them)."""
    arr = (Problem * len(problems))(*problems) if not isinstance(problems, ctypes.Array) else problems
    ctx = _P()
    _check(lib().sdeb_create_batch(ctypes.cast(arr, _P), len(arr), ctypes.byref(ctx)))
    return ctx


def sdeb_batch_read(ctx, instance, what, dst, dst_bytes, dst_on_device, stream=None):
    _check(lib().sdeb_batch_read(ctx, instance, what, dst, dst_bytes, int(dst_on_device), _stream(stream)), ctx)


def sdeb_batch_info(ctx):
    t, tm, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sdeb_batch_info(ctx, ctypes.byref(t), ctypes.byref(tm), ctypes.byref(g)), ctx)
    return {"tasks": t.value, "team_items": tm.value, "grid": g.value}


def sdeb_batch_set_schedule(ctx, chain_fraction):
    _check(lib().sdeb_batch_set_schedule(ctx, float(chain_fraction)), ctx)


def sdeb_batch_plan(problems, chain_fraction, num_sms):
    """Host-only schedule of a batch (no GPU needed).  Returns a dict of numpy
    arrays: lanes and units_per_lane per instance; task, slot and lane0 per
    orbit of every instance in order; and the task count."""
    import numpy as np
    arr = (Problem * len(problems))(*problems) if not isinstance(problems, ctypes.Array) else problems
    total = sum(int(p.orbits) for p in arr)
    lanes = np.zeros(len(arr), np.int32)
    upl = np.zeros(len(arr), np.int32)
    task = np.full(total, -1, np.int32)
    slot = np.full(total, -1, np.int32)
    lane0 = np.full(total, -1, np.int32)
    nt = ctypes.c_int32()
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(lib().sdeb_batch_plan(ctypes.cast(arr, _P), len(arr), float(chain_fraction), int(num_sms), ptr(lanes),
                                 ptr(upl), total, ptr(task), ptr(slot), ptr(lane0), ctypes.byref(nt)))
    return {"lanes": lanes, "units_per_lane": upl, "task": task, "slot": slot, "lane0": lane0, "tasks": nt.value}


def sdeb_batch_layout(ctx, instance):
    g, p = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sdeb_batch_layout(ctx, instance, ctypes.byref(g), ctypes.byref(p)), ctx)
    return g.value, p.value


def sdeb_get_layout(ctx):
    g, p = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sdeb_get_layout(ctx, ctypes.byref(g), ctypes.byref(p)), ctx)
    return g.value, p.value


def sdeb_set_adjoint_records(ctx, mode):
    _check(lib().sdeb_set_adjoint_records(ctx, mode), ctx)


def sdeb_get_checkpoint_interval(ctx):
    v = ctypes.c_int64()
    _check(lib().sdeb_get_checkpoint_interval(ctx, ctypes.byref(v)), ctx)
    return v.value


def sdeb_last_error(ctx=None):
    s = lib().sdeb_last_error(ctx)
    return s.decode() if s else ""


def sdeb_status_string(status):
    return lib().sdeb_status_string(status).decode()


def sdeb_philox_fill(seed, k0, nk, b0, nb, o0, no, stream_id, out, stream=None):
    _check(lib().sdeb_philox_fill(seed, k0, nk, b0, nb, o0, no, stream_id, out, _stream(stream)))


def sdeb_normals_fill(seed, k0, nk, o0, no, m, precision, out, stream=None):
    _check(lib().sdeb_normals_fill(seed, k0, nk, o0, no, m, precision, out, _stream(stream)))


def sdeb_order_param(theta, orbits, n, precision, r, dr=None, stream=None):
    _check(lib().sdeb_order_param(theta, orbits, n, precision, r, dr, _stream(stream)))


def sdeb_swarm_expand(x, particles, dims, base, d, realisations, precision, params_out, stream=None):
    """dims: a sequence of parameter columns (copied to a host int32 array)."""
    cols = (ctypes.c_int32 * len(dims))(*dims)
    _check(lib().sdeb_swarm_expand(x, particles, len(dims), cols, base, d, realisations,
                                   PRECISIONS.get(precision, precision), params_out, _stream(stream)))


def sdeb_swarm_fitness(theta, particles, realisations, n, precision, r_target, fit, stream=None):
    _check(lib().sdeb_swarm_fitness(theta, particles, realisations, n, PRECISIONS.get(precision, precision),
                                    float(r_target), fit, _stream(stream)))


def sdeb_swarm_update(x, v, pbest, pbest_fit, fit, particles, lo, hi, w, c1, c2, seed, generation, gbest,
                      stream=None):
    """lo, hi: sequences of the D bounds (copied to host float64 arrays)."""
    lo_a = (ctypes.c_double * len(lo))(*[float(t) for t in lo])
    hi_a = (ctypes.c_double * len(hi))(*[float(t) for t in hi])
    if len(lo) != len(hi):
        raise ValueError("lo and hi need one bound per dimension")
    _check(lib().sdeb_swarm_update(x, v, pbest, pbest_fit, fit, particles, len(lo), lo_a, hi_a, float(w), float(c1),
                                   float(c2), seed & 0xFFFFFFFFFFFFFFFF, generation, gbest, _stream(stream)))


def sdeb_check_status():
    """(status, word) of the checked build's bounds-check status word (read
    and cleared); status SDEB_EBOUNDS when a check failed, SDEB_EUNSUPPORTED
    in the unchecked library."""
    w = ctypes.c_uint64()
    st = lib().sdeb_check_status(ctypes.byref(w))
    return st, w.value


def sdeb_check_selftest(stream=None):
    _check(lib().sdeb_check_selftest(_stream(stream)))


PIPES = {"sfu_sin": 0, "sfu_lg2": 1, "sfu_sqrt": 2, "fp64_fma": 3, "fp32_fma": 4}


def sdeb_pipe_rate(pipe, iters=1024, stream=None):
    """Measured results per SM per clock of one pipe (a name of PIPES or its number)."""
    out = ctypes.c_double()
    _check(lib().sdeb_pipe_rate(PIPES.get(pipe, pipe), iters, ctypes.byref(out), _stream(stream)))
    return out.value


def sdeb_integrate_noalloc(problem, params, x0, x_final, frames=None, stream=None):
    """Allocation-free forward integration (see include/sdeb.h)."""
    _check(lib().sdeb_integrate_noalloc(ctypes.byref(problem), params, x0, x_final, frames, _stream(stream)))
