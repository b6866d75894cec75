"""ctypes binding of the plain CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It never
imports the CUDA library's package, and the CUDA library never imports it.

Model names map to the oracle's own numeric ids; callers pass names.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MODELS = {
    "kuramoto": 1,
    "kuramoto_paper": 2,
    "fhn_net": 3,
    "ou": 4,
    "gbm": 5,
    "linear_ode": 6,
}


class Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("n", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("t0", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("steps", ctypes.c_int64),
        ("stride", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("shared_params", ctypes.c_int32),
        ("mean_field", ctypes.c_int32),
        ("milstein", ctypes.c_int32),
        ("rk4", ctypes.c_int32),
        ("implicit", ctypes.c_int32),
    ]


_lib = None
_P = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_philox4x32_10.argtypes = [_P, _P, _P]
        L.oracle_philox_block.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, _P]
        L.oracle_philox_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                         ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint32,
                                         ctypes.c_int64, ctypes.c_uint32, _P]
        L.oracle_normals_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                          ctypes.c_uint32, ctypes.c_int64, ctypes.c_int32, _P]
        L.oracle_uniform.argtypes = [ctypes.c_uint32]
        L.oracle_uniform.restype = ctypes.c_double
        L.oracle_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _P]
        L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_int32, _P]
        L.oracle_drift.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P]
        L.oracle_diffusion.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P]
        L.oracle_diffusion_diag_derivative.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P]
        L.oracle_drift_jacobian.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P]
        L.oracle_check_problem.argtypes = [ctypes.POINTER(Problem)]
        L.oracle_integrate.argtypes = [ctypes.POINTER(Problem), _P, _P, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                       ctypes.c_int32]
        L.oracle_adjoint.argtypes = [ctypes.POINTER(Problem), _P, _P, ctypes.c_int64,
                                     ctypes.c_int64, _P, _P, _P]
        L.oracle_order_param.argtypes = [ctypes.c_int32, _P, _P, _P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


IMPLICIT = {None: 0, "euler": 1, "midpoint": 2}


def make_problem(model, n, m, d, dt, steps, stride=1, seed=0, t0=0.0,
                 shared_params=False, mean_field=False, milstein=False, rk4=False, implicit=None):
    return Problem(MODELS[model] if isinstance(model, str) else int(model), n, m, d, float(t0),
                   float(dt), int(steps), int(stride), int(seed) & 0xFFFFFFFFFFFFFFFF,
                   int(bool(shared_params)), int(bool(mean_field)), int(bool(milstein)), int(bool(rk4)),
                   IMPLICIT[implicit])


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_fill(seed, k0, nk, b0, nb, o0, no, stream=0):
    out = np.zeros((nk, nb, no, 4), dtype=np.uint32)
    lib().oracle_philox_fill(seed, k0, nk, b0, nb, o0, no, stream, _ptr(out))
    return out


def normals_fill(seed, k0, nk, o0, no, m):
    out = np.zeros((nk, no, m), dtype=np.float64)
    lib().oracle_normals_fill(seed, k0, nk, o0, no, m, _ptr(out))
    return out


def uniform(w):
    return lib().oracle_uniform(int(w))


def box_muller(w_first, w_second):
    out = np.zeros(2)
    lib().oracle_box_muller(int(w_first), int(w_second), _ptr(out))
    return out


def drift(pb, x, p, t=0.0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    f = np.zeros(pb.n, dtype=np.float64)
    assert lib().oracle_drift(ctypes.byref(pb), t, _ptr(x), _ptr(p), _ptr(f)) == 0
    return f


def diffusion(pb, x, p, t=0.0):
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    g = np.zeros((pb.n, max(pb.m, 1)), dtype=np.float64)
    assert lib().oracle_diffusion(ctypes.byref(pb), t, _ptr(x), _ptr(p), _ptr(g)) == 0
    return g[:, :pb.m]


def diffusion_diag_derivative(pb, x, p, t=0.0):
    """d g_jj / d x_j for j < m (diagonal noise; see oracle.h)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    dg = np.zeros(max(pb.m, 1), dtype=np.float64)
    assert lib().oracle_diffusion_diag_derivative(ctypes.byref(pb), t, _ptr(x), _ptr(p), _ptr(dg)) == 0
    return dg[:pb.m]


def drift_jacobian(pb, x, p, t=0.0):
    """J[i][j] = d f_i / d x_j."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(p, dtype=np.float64)
    J = np.zeros((pb.n, pb.n), dtype=np.float64)
    assert lib().oracle_drift_jacobian(ctypes.byref(pb), t, _ptr(x), _ptr(p), _ptr(J)) == 0
    return J


def integrate(pb, params, x0, orbit_begin=0, k_begin=0, k_end=None, frames=True, nthreads=1):
    """Returns (frames [F][count][n] or None, x_final [count][n])."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    count = x0.shape[0]
    assert x0.shape == (count, pb.n)
    if pb.shared_params:
        assert params.shape == (pb.d,)
    else:
        assert params.shape == (count, pb.d)
    if k_end is None:
        k_end = pb.steps
    F = pb.steps // pb.stride + 1 if pb.stride >= 1 else 0
    fr = np.full((F, count, pb.n), np.nan) if frames and F > 0 else None
    xout = np.zeros_like(x0)
    rc = lib().oracle_integrate(ctypes.byref(pb), _ptr(params), _ptr(x0), orbit_begin, count,
                                k_begin, k_end, _ptr(fr), _ptr(xout), nthreads)
    if rc != 0:
        raise ValueError("oracle_integrate rejected the problem")
    return fr, xout


def adjoint(pb, params, x0, dL_dxK, orbit_begin=0):
    """Returns (dL/dp [count][d], dL/dx0 [count][n])."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    params = np.ascontiguousarray(params, dtype=np.float64)
    g = np.ascontiguousarray(dL_dxK, dtype=np.float64)
    count = x0.shape[0]
    dp = np.zeros((count, pb.d))
    dx0 = np.zeros((count, pb.n))
    rc = lib().oracle_adjoint(ctypes.byref(pb), _ptr(params), _ptr(x0), orbit_begin, count,
                              _ptr(g), _ptr(dp), _ptr(dx0))
    if rc != 0:
        raise ValueError("oracle_adjoint rejected the problem")
    return dp, dx0


def order_param(theta):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    r = np.zeros(1)
    dr = np.zeros(th.shape[-1])
    lib().oracle_order_param(th.shape[-1], _ptr(th), _ptr(r), _ptr(dr))
    return float(r[0]), dr


def frame_moments(frames, order_parameter=False):
    """Ensemble moments of frames [F][orbits][n] over the orbits, FP64, by
    definition (two passes): mom [F][n][2] = (mean, population variance
    mean((x - mean)^2)) of every state component; with order_parameter, also
    rmom [F][2] = (mean, population variance) of r = |(1/n) sum_j
    exp(i x_j)|, the order parameter of Eq. 7 (Sec. 2.3: the statistics of
    r over realisations that the paper's accuracy experiment reports)."""
    fr = np.asarray(frames, dtype=np.float64)
    mean = fr.mean(axis=1)
    var = ((fr - mean[:, None, :]) ** 2).mean(axis=1)
    mom = np.stack([mean, var], axis=-1)
    if not order_parameter:
        return mom, None
    r = np.abs(np.exp(1j * fr).mean(axis=2))            # [F][orbits]
    rmean = r.mean(axis=1)
    rvar = ((r - rmean[:, None]) ** 2).mean(axis=1)
    return mom, np.stack([rmean, rvar], axis=-1)
