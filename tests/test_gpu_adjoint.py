"""GPU parity of the discrete adjoint (sdeb_grad) and the order parameter.

* Per-orbit gradients dL/dp and dL/dx0 against the FP64 oracle adjoint
  (dense Jacobians, all states stored) on the same inputs and the same
  dL/dX^K: FP64 to 1e-10 and FP32 to 1e-3, relative to the largest gradient
  component of the orbit; ragged segments (steps not a multiple of
  ckpt_every), both parameter layouts, several lane-group layouts.
* The adjoint workload (n = 32, 16384 orbits sharing one parameter vector,
  dt = 0.01, 2000 steps, checkpoints every 100, loss = mean order parameter
  at T = 20): the FP64 adjoint against central finite differences of the
  FP64 forward with common random numbers (T = 5 and T = 20).  FP32 against
  FP64: the orbit-mean gradient to 1e-3 at T = 5; at T = 20 the mean is
  carried by the ~1 % of orbits whose pathwise gradients explode (orbits
  near the synchronisation transition, where the FP32 and FP64 trajectories
  themselves part), so there the check is per orbit: the median orbit agrees
  to 1e-4 and fewer than 5 % of orbits differ by more than 1e-3.
* Per orbit on the adjoint workload at T = 5, against central finite
  differences of the FP64 forward (common random numbers): the FP64 adjoint
  of every orbit within 1e-6, the FP32 adjoint within 1e-3 except on
  orbits whose gradient is sensitive to FP32 rounding (within 45 times the
  move one FP32 ulp of x0 gives the FP64 gradient; at most 0.1 % of them;
  measured: 6 of 16384).
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import np_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    scale = np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


def _gpu_grad(model, n, p, x0, dt, steps, ckpt, seed, precision, dL_dxK, shared=False):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    dt_t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make(model, n, x0.shape[0], dt, steps, 1, seed, precision, ckpt_every=ckpt,
                           no_frames=True, shared_params=shared)
    with Integrator(pb) as it:
        it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
        it.integrate()
        xK = it.final().cpu().numpy()
        dp, dx0 = it.grad(torch.tensor(dL_dxK, dtype=dt_t).cuda())
        torch.cuda.synchronize()
        return xK, dp.cpu().numpy(), dx0.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("model,n,ckpt", [("kuramoto", 3, 37), ("kuramoto", 8, 50), ("kuramoto", 32, 64),
                                          ("kuramoto", 20, 300), ("kuramoto_paper", 12, 41),
                                          ("kuramoto", 128, 100)])
def test_adjoint_matches_oracle(precision, model, n, ckpt):
    orbits, dt, steps, seed = 9, 0.01, 300, 4
    if model == "kuramoto":
        p, x0 = inputs.kuramoto(n, orbits, seed=n)
    else:
        p, x0 = inputs.kuramoto_paper_speed(n, orbits, seed=n)
        p[:, 0] = 2.0
        p[:, n + 1:] = 0.3
    p, x0 = p.astype(np_dtype(precision)).astype(np.float64), x0.astype(np_dtype(precision)).astype(np.float64)
    c = np.random.Generator(np.random.PCG64(n)).standard_normal((orbits, n))
    _, dp, dx0 = _gpu_grad(model, n, p, x0, dt, steps, ckpt, seed, precision, c)
    m, d = sdeb.model_shape(model, n)
    pb = oracle.make_problem(model, n, m, d, dt, steps, 1, seed)
    rdp, rdx0 = oracle.adjoint(pb, p, x0, c)
    tol = 1e-10 if precision == "fp64" else 1e-3
    assert _rel(dp, rdp) < tol
    assert _rel(dx0, rdx0) < tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_with_a_shortened_checkpoint_interval(precision):
    """Many orbits of n = 128 with ckpt_every = 97: the context keeps
    checkpoints every 8 steps (an interval that does not divide the 302
    steps: a ragged last segment); at the default layout (16 lanes of 8
    units) the FP32 records fit shared memory, the FP64 ones go through the
    global buffer.  Sampled orbits' gradients against the oracle adjoint."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits, dt, steps, ckpt, seed = 128, 8192, 0.01, 302, 97, 6
    p, x0 = inputs.kuramoto(n, orbits, seed=7)
    p, x0 = p.astype(np_dtype(precision)).astype(np.float64), x0.astype(np_dtype(precision)).astype(np.float64)
    c = np.random.Generator(np.random.PCG64(3)).standard_normal((orbits, n))
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make("kuramoto", n, orbits, dt, steps, 1, seed, precision, ckpt_every=ckpt, no_frames=True)
    with Integrator(pb) as it:
        interval = sdeb.sdeb_get_checkpoint_interval(it.ctx)
        it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
        it.integrate()
        dp, dx0 = it.grad(torch.tensor(c, dtype=dt_t).cuda())
        dp, dx0 = dp.cpu().numpy(), dx0.cpu().numpy()
    print("checkpoint interval", interval)
    assert interval == 8 and steps % interval != 0
    m, d = sdeb.model_shape("kuramoto", n)
    opb = oracle.make_problem("kuramoto", n, m, d, dt, steps, 1, seed)
    tol = 1e-10 if precision == "fp64" else 1e-3
    for o in (0, 4095, 8191):
        rdp, rdx0 = oracle.adjoint(opb, p[o:o + 1], x0[o:o + 1], c[o:o + 1], orbit_begin=o)
        assert _rel(dp[o:o + 1], rdp) < tol, o
        assert _rel(dx0[o:o + 1], rdx0) < tol, o


def _loss_and_grads(precision, p, x0, W, steps=None, want_grad=True, shared=True):
    import torch
    from paper_1908_03869_gb300.autograd import integrate_final, order_parameter
    from paper_1908_03869_gb300.integrator import Integrator

    dt_t = torch.float64 if precision == "fp64" else torch.float32
    n, orbits = x0.shape[1], x0.shape[0]
    pb = sdeb.Problem.make("kuramoto", n, orbits, W["dt"], steps or W["steps"], 1, W["seed"], precision,
                           ckpt_every=W["ckpt_every"], no_frames=True, shared_params=shared)
    with Integrator(pb) as it:
        pt = torch.tensor(p, dtype=dt_t, device="cuda", requires_grad=want_grad)
        xt = torch.tensor(x0, dtype=dt_t, device="cuda")
        loss = order_parameter(integrate_final(it, pt, xt)).mean()
        if want_grad:
            loss.backward()
            return float(loss.detach()), pt.grad.cpu().numpy().astype(np.float64)
        return float(loss), None


@pytest.mark.parametrize("steps", [500, 2000])
def test_adjoint_workload_fp64_vs_central_fd(steps):
    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    p, x0 = inputs.kuramoto(32, W["orbits"], seed=1, shared=True)
    _, g64 = _loss_and_grads("fp64", p, x0, W, steps)
    scale = np.abs(g64).max()
    # Orbits near the synchronisation transition have pathwise derivatives
    # ~1e4 times the typical one at T = 20, so the loss is linear in p only
    # over a small range: the differences use h = 1e-6, 1e-7 and 1e-8
    # (times max(|p_q|, 1)) and the adjoint must match the best of them.
    for q in [0, 1, 2, 7, 33]:           # K, sigma and three omegas
        errs = []
        for rel_h in (1e-6, 1e-7, 1e-8):
            h = rel_h * max(abs(p[q]), 1.0)
            pp, pm = p.copy(), p.copy()
            pp[q] += h
            pm[q] -= h
            Lp, _ = _loss_and_grads("fp64", pp, x0, W, steps, want_grad=False)
            Lm, _ = _loss_and_grads("fp64", pm, x0, W, steps, want_grad=False)
            fd = (Lp - Lm) / (2 * h)
            errs.append(abs(g64[q] - fd) / max(abs(fd), 1e-2 * scale))
        assert min(errs) < 1e-3, (q, g64[q], errs)


def test_adjoint_workload_fp32_vs_fp64():
    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    orbits = W["orbits"]
    p, x0 = inputs.kuramoto(32, orbits, seed=1, shared=True)
    p, x0 = p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64)
    # T = 5: the orbit mean of the shared-parameter gradient
    L64, g64 = _loss_and_grads("fp64", p, x0, W, 500)
    L32, g32 = _loss_and_grads("fp32", p, x0, W, 500)
    assert abs(L32 - L64) < 1e-5
    assert np.abs(g32 - g64).max() < 1e-3 * np.abs(g64).max()
    # T = 20: per-orbit gradients
    pt = np.tile(p, (orbits, 1))
    _, G64 = _loss_and_grads("fp64", pt, x0, W, shared=False)
    _, G32 = _loss_and_grads("fp32", pt, x0, W, shared=False)
    rel = np.abs(G32 - G64).max(axis=1) / np.abs(G64).max(axis=1)
    assert np.median(rel) < 1e-4, np.median(rel)
    assert (rel > 1e-3).mean() < 0.05, (rel > 1e-3).mean()


def _per_orbit_r(precision, p, x0, W, steps):
    """r_o(T) of every orbit (FP64 host array) for per-orbit parameters p."""
    import torch
    from paper_1908_03869_gb300.autograd import order_parameter
    from paper_1908_03869_gb300.integrator import Integrator

    dt_t = torch.float64 if precision == "fp64" else torch.float32
    n, orbits = x0.shape[1], x0.shape[0]
    pb = sdeb.Problem.make("kuramoto", n, orbits, W["dt"], steps, 1, W["seed"], precision, no_frames=True)
    with Integrator(pb) as it:
        it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
        it.integrate()
        r = order_parameter(it.final())
        return r.cpu().numpy().astype(np.float64)


def test_adjoint_workload_fp32_per_orbit_vs_central_fd():
    """Per-orbit pathwise gradients on the adjoint workload at T = 5 (500
    steps) for K, sigma and three omegas, against central finite differences
    of the FP64 forward with common random numbers (h = 1e-5, 1e-6, 1e-7
    times max(|p_q|, 1), the best of them):
      * the FP64 adjoint of every orbit within 1e-6 (relative to the orbit's
        largest checked component);
      * the FP32 adjoint of every orbit within 1e-3, except orbits whose
        gradient the dynamics make sensitive to FP32 rounding: there the FP32
        gradient, which carries a rounding in every one of its 500 steps,
        may differ by up to 45 times (twice the square root of the step
        count) the move one FP32 ulp of x0 gives the FP64 gradient; at most
        0.1 % of the orbits."""
    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    orbits, steps, n = W["orbits"], 500, 32
    p, x0 = inputs.kuramoto(n, orbits, seed=1, shared=True)
    p, x0 = p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64)
    pt = np.tile(p, (orbits, 1))
    qs = [0, 1, 2, 7, 33]                 # K, sigma and three omegas
    G = {}
    for prec in ("fp32", "fp64"):
        _, g = _loss_and_grads(prec, pt, x0, W, steps, shared=False)
        G[prec] = g[:, qs] * orbits       # d r_o / d p_o: the loss is the orbit mean
    sign = np.where(np.sin(np.arange(n) * 7.1) >= 0, 1.0, -1.0)
    _, g = _loss_and_grads("fp64", pt, x0 * (1 + 2.0 ** -24 * sign), W, steps, shared=False)
    G["fp64_ulp"] = g[:, qs] * orbits

    def rel(a, b):
        return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)

    rel64, rel32 = np.full(orbits, np.inf), np.full(orbits, np.inf)
    for rel_h in (1e-5, 1e-6, 1e-7):
        fd = np.empty((orbits, len(qs)))
        for j, q in enumerate(qs):
            h = rel_h * max(abs(p[q]), 1.0)
            pp, pm = pt.copy(), pt.copy()
            pp[:, q] += h
            pm[:, q] -= h
            fd[:, j] = (_per_orbit_r("fp64", pp, x0, W, steps) - _per_orbit_r("fp64", pm, x0, W, steps)) / (2 * h)
        rel64 = np.minimum(rel64, rel(G["fp64"], fd))
        rel32 = np.minimum(rel32, rel(G["fp32"], fd))
    sens = rel(G["fp64_ulp"], G["fp64"])
    beyond = np.flatnonzero(rel32 >= 1e-3)
    print("adjoint vs fd per orbit: fp64 max %.1e; fp32 median %.1e, max %.1e, %d orbits beyond 1e-3 "
          "(one-ulp gradient sensitivity of those: %s)" % (rel64.max(), np.median(rel32), rel32.max(), beyond.size,
                                                          ["%.1e" % v for v in sens[beyond]]))
    assert rel64.max() < 1e-6, (int(np.argmax(rel64)), rel64.max())
    assert beyond.size <= orbits // 1000
    for o in beyond:
        assert rel32[o] < 45 * sens[o], (int(o), rel32[o], sens[o])


def test_adjoint_workload_sampled_orbits_vs_oracle():
    """Per-orbit FP64 gradients of the order-parameter loss against the oracle,
    whose dL/dX^K comes from its own final state."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    W = inputs.WORKLOADS["kuramoto_adjoint_n32"]
    n, orbits = 32, W["orbits"]
    p, x0 = inputs.kuramoto(n, orbits, seed=1, shared=True)
    sample = [0, 1, 777, 4095, 16383]
    pb = sdeb.Problem.make("kuramoto", n, orbits, W["dt"], W["steps"], 1, W["seed"], "fp64",
                           ckpt_every=W["ckpt_every"], no_frames=True)   # per-orbit gradients
    pfull = np.tile(p, (orbits, 1))
    with Integrator(pb) as it:
        it.set_params(torch.tensor(pfull).cuda(), torch.tensor(x0).cuda())
        it.integrate()
        xK = it.final()
        r = torch.empty(orbits, dtype=torch.float64, device="cuda")
        dr = torch.empty_like(xK)
        sdeb.sdeb_order_param(ctypes.c_void_p(xK.data_ptr()), orbits, n, sdeb.SDEB_FP64,
                              ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(dr.data_ptr()))
        dp, dx0 = it.grad(dr / orbits)
        dp, dx0, xK = dp.cpu().numpy(), dx0.cpu().numpy(), xK.cpu().numpy()
    opb = oracle.make_problem("kuramoto", n, n, n + 2, W["dt"], W["steps"], 1, W["seed"])
    for o in sample:
        _, oxK = oracle.integrate(opb, pfull[o:o + 1], x0[o:o + 1], orbit_begin=o, frames=False)
        _, odr = oracle.order_param(oxK[0])
        rdp, rdx0 = oracle.adjoint(opb, pfull[o:o + 1], x0[o:o + 1], (odr / orbits)[None, :], orbit_begin=o)
        assert _rel(dp[o:o + 1], rdp) < 1e-8, o
        assert _rel(dx0[o:o + 1], rdx0) < 1e-8, o


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_order_param_kernel(precision):
    import torch
    th = np.random.Generator(np.random.PCG64(2)).uniform(-50, 50, (300, 37)).astype(np_dtype(precision))
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(th, dtype=dt_t, device="cuda")
    r = torch.empty(300, dtype=dt_t, device="cuda")
    dr = torch.empty_like(t)
    sdeb.sdeb_order_param(ctypes.c_void_p(t.data_ptr()), 300, 37, sdeb.PRECISIONS[precision],
                          ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(dr.data_ptr()))
    r, dr = r.cpu().numpy(), dr.cpu().numpy()
    tol = 1e-13 if precision == "fp64" else 2e-5
    for o in range(300):
        rr, rdr = oracle.order_param(th[o].astype(np.float64))
        assert abs(r[o] - rr) < tol
        assert np.abs(dr[o] - rdr).max() < tol * 10


def test_autotune_on_a_checkpointed_context_keeps_the_gradient_consistent():
    """sdeb_autotune on a context with checkpoints times forward + adjoint;
    it leaves the checkpoints intact (checkpoint 0 is x0), and the gradient
    after tuning equals the gradient of a fresh context set to the chosen
    layout, bit for bit, and the FP64 oracle adjoint to 1e-3 (FP32)."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits, dt, steps, ckpt, seed = 32, 512, 0.01, 250, 100, 3
    p, x0 = inputs.kuramoto(n, orbits, seed=4)
    p, x0 = p.astype(np.float32), x0.astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(8))
    dL = rng.standard_normal((orbits, n)).astype(np.float32)
    pb = sdeb.Problem.make("kuramoto", n, orbits, dt, steps, 1, seed, "fp32", ckpt_every=ckpt, no_frames=True)
    res = []
    for tuned in (True, False):
        with Integrator(pb) as it:
            it.set_params(torch.tensor(p).cuda(), torch.tensor(x0).cuda())
            if tuned:
                lay = it.autotune()
            else:
                it.set_layout(*lay)
            it.integrate()
            dp, dx0 = it.grad(torch.tensor(dL).cuda())
            res.append((it.final().cpu().numpy(), dp.cpu().numpy(), dx0.cpu().numpy()))
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)
    m, d = sdeb.model_shape("kuramoto", n)
    opb = oracle.make_problem("kuramoto", n, m, d, dt, steps, 1, seed)
    dp_o, dx0_o = oracle.adjoint(opb, p.astype(np.float64), x0.astype(np.float64), dL.astype(np.float64))
    assert _rel(res[0][1], dp_o) < 1e-3
    assert _rel(res[0][2], dx0_o) < 1e-3


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_adjoint_records_in_shared_and_global_memory_agree(precision):
    """The replay's step records kept in shared memory or in the global
    buffer (sdeb_set_adjoint_records) give the same bits, at layouts whose
    records fit shared memory at the 8-step interval; SHARED where they do
    not fit (FP64 with 8 units per lane) is EUNSUPPORTED.  A context asked
    for checkpoints at most 6 steps apart keeps them every 6 steps.  The
    gradients against the oracle adjoint (ragged last segment: 250 steps)."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits, dt, steps, seed = 32, 300, 0.01, 250, 5
    p, x0 = inputs.kuramoto(n, orbits, seed=11)
    p, x0 = p.astype(np_dtype(precision)).astype(np.float64), x0.astype(np_dtype(precision)).astype(np.float64)
    c = np.random.Generator(np.random.PCG64(12)).standard_normal((orbits, n))
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    m, d = sdeb.model_shape("kuramoto", n)
    opb = oracle.make_problem("kuramoto", n, m, d, dt, steps, 1, seed)
    tol = 1e-10 if precision == "fp64" else 1e-3
    samples = (0, 151, 299)
    ref = [oracle.adjoint(opb, p[o:o + 1], x0[o:o + 1], c[o:o + 1], orbit_begin=o) for o in samples]
    for ckpt in (100, 6):
        for lay in ((8, 4), (4, 8)):
            # a block's records: interval x (3 P + 2) elements x 128 threads, shared memory up to 112 KB
            elem = 8 if precision == "fp64" else 4
            fits = min(ckpt, 8) * (3 * lay[1] + 2) * 128 * elem <= 112 * 1024
            res = {}
            for mode in (sdeb.SDEB_RECORDS_AUTO, sdeb.SDEB_RECORDS_GLOBAL, sdeb.SDEB_RECORDS_SHARED):
                pb = sdeb.Problem.make("kuramoto", n, orbits, dt, steps, 1, seed, precision, ckpt_every=ckpt,
                                       no_frames=True)
                with Integrator(pb) as it:
                    assert sdeb.sdeb_get_checkpoint_interval(it.ctx) == min(ckpt, 8)
                    it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
                    it.set_layout(*lay)
                    it.set_adjoint_records(mode)
                    it.integrate()
                    dL = torch.tensor(c, dtype=dt_t).cuda()
                    if mode == sdeb.SDEB_RECORDS_SHARED and not fits:
                        with pytest.raises(sdeb.SdebError) as e:
                            it.grad(dL)
                        assert e.value.status == sdeb.SDEB_EUNSUPPORTED
                        continue
                    dp, dx0 = it.grad(dL)
                    res[mode] = (dp.cpu().numpy(), dx0.cpu().numpy())
            for mode, (dp, dx0) in res.items():
                np.testing.assert_array_equal(dp, res[sdeb.SDEB_RECORDS_GLOBAL][0], err_msg=str((ckpt, lay, mode)))
                np.testing.assert_array_equal(dx0, res[sdeb.SDEB_RECORDS_GLOBAL][1], err_msg=str((ckpt, lay, mode)))
            dp, dx0 = res[sdeb.SDEB_RECORDS_AUTO]
            for o, (rdp, rdx0) in zip(samples, ref):
                assert _rel(dp[o:o + 1], rdp) < tol, (ckpt, lay, o)
                assert _rel(dx0[o:o + 1], rdx0) < tol, (ckpt, lay, o)
    with pytest.raises(sdeb.SdebError) as e:
        pb = sdeb.Problem.make("kuramoto", n, orbits, dt, steps, 1, seed, precision, ckpt_every=10, no_frames=True)
        with Integrator(pb) as it:
            it.set_adjoint_records(7)
    assert e.value.status == sdeb.SDEB_EINVAL
