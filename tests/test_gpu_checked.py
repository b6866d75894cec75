"""The bounds-checked build on the GPU: every kernel of the library runs on
small cases with libsdeb_checked.so (forward kernels of every model and
step scheme and several lane layouts, frames, checkpoints and resume, the
adjoint with its own and with a shortened checkpoint interval, a batch under
schedules that use every layout, a user model compiled at run time, the
allocation-free path, the moment reduction, a particle-swarm generation and
the stand-alone kernels), and the device status word stays clear.  The
reporting path itself is exercised by sdeb_check_selftest, which records a
synthetic failure without any other memory access.  Runs in a child process
that loads the checked library (SDEB_LIBRARY=checked)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    import ctypes
    import numpy as np
    import torch
    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import build, inputs
    build.build(checked=True)
    assert sdeb.library_path().endswith("libsdeb_checked.so")
    sdeb.lib()
    from paper_1908_03869_gb300.integrator import Integrator, BatchIntegrator
    from paper_1908_03869_gb300.swarm import SwarmSearch
    from helpers import run_gpu

    def status(tag):
        st, w = sdeb.sdeb_check_status()
        print("STATUS", tag, st, hex(w), flush=True)

    def model_inputs(model, n, orbits, seed):
        if model == "kuramoto":
            return inputs.kuramoto(n, orbits, seed=seed)
        if model == "kuramoto_paper":
            return inputs.kuramoto_paper_speed(n, orbits, seed=seed)
        if model == "fhn_net":
            return inputs.fhn(n // 2, orbits, seed=seed)
        if model in ("ou", "gbm"):
            return inputs.scalar_model(n, orbits, [0.5, 0.3], 0.5, 1.5, seed=seed)
        return inputs.scalar_model(n, orbits, [0.7], -1, 1, seed=seed)

    cases = [("kuramoto", 3), ("kuramoto", 8), ("kuramoto", 32), ("kuramoto", 100), ("kuramoto", 256),
             ("kuramoto_paper", 12), ("fhn_net", 64), ("ou", 5), ("gbm", 4), ("linear_ode", 6)]
    for prec in ("fp32", "fp64"):
        t = np.float32 if prec == "fp32" else np.float64
        for model, n in cases:
            p, x0 = model_inputs(model, n, 97, 3)
            run_gpu(model, n, p.astype(t), x0.astype(t), 0.01, 130, 7, precision=prec,
                    ckpt_every=25 if model.startswith("kuramoto") else 0, ranges=[(0, 61), (61, 130)])
        for kw in (dict(rk4=True), dict(implicit="euler"), dict(implicit="midpoint")):
            for model, n in (("kuramoto", 32), ("fhn_net", 32), ("gbm", 3)):
                p, x0 = model_inputs(model, n, 50, 4)
                run_gpu(model, n, p.astype(t), x0.astype(t), 0.01, 40, 10, precision=prec, **kw)
        p, x0 = model_inputs("gbm", 4, 50, 5)
        run_gpu("gbm", 4, p.astype(t), x0.astype(t), 0.01, 40, 10, precision=prec, milstein=True)
        for layout in ((16, 4), (8, 4), (4, 16)):
            p, x0 = model_inputs("kuramoto", 32, 70, 6)
            run_gpu("kuramoto", 32, p.astype(t), x0.astype(t), 0.01, 40, 10, precision=prec, layout=layout)
    status("forward")

    dtt = {{"fp32": torch.float32, "fp64": torch.float64}}
    for prec, (n, orbits, ckpt) in (("fp32", (32, 500, 25)), ("fp64", (32, 500, 25)), ("fp32", (128, 8192, 97))):
        p, x0 = inputs.kuramoto(n, orbits, seed=7)
        pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 302, 1, 2, prec, ckpt_every=ckpt, no_frames=True)
        with Integrator(pb) as it:
            it.set_params(torch.tensor(p, dtype=dtt[prec]).cuda(), torch.tensor(x0, dtype=dtt[prec]).cuda())
            if orbits == 500:
                it.autotune()
            it.integrate()
            it.grad(torch.ones((orbits, n), dtype=dtt[prec]).cuda())
            torch.cuda.synchronize()
            print("interval", sdeb.sdeb_get_checkpoint_interval(it.ctx))
    status("adjoint")

    insts = inputs.batched_instances(40, seed=9, k_low=50, k_high=600)
    pbs = [sdeb.Problem.make("kuramoto", d["n"], 1, d["dt"], d["steps"], 7 + (i % 3) * 20, 0, "fp32",
                             orbit_offset=i, no_frames=(i % 11 == 5)) for i, d in enumerate(insts)]
    ps = [d["params"][None, :].astype(np.float32) for d in insts]
    xs = [d["x0"][None, :].astype(np.float32) for d in insts]
    with BatchIntegrator(pbs) as b:
        kinds = set()
        for frac in (1e9, 1.0, 0.1, 1e-2, 1e-3, 1e-9):
            b.set_params(ps, xs)
            b.set_schedule(frac)
            kinds |= {{b.layout(i) for i in range(len(pbs))}}
            b.integrate()
            torch.cuda.synchronize()
        b.set_params(ps, xs)
        b.autotune()
        b.integrate()
        torch.cuda.synchronize()
        print("batch layouts", sorted(kinds))
    status("batch")

    src = '''
    __device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {{
        for (int i = 0; i < SDEB_N; ++i) f[i] = p[0] * x[i];
    }}
    __device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {{
        for (int i = 0; i < SDEB_N * SDEB_M; ++i) g[i] = 0;
        for (int i = 0; i < SDEB_N; ++i) g[i * SDEB_M + i] = p[1] * x[i];
    }}
    '''
    p, x0 = model_inputs("gbm", 4, 60, 8)
    for prec in ("fp32", "fp64"):
        pb = sdeb.Problem.make("user", 4, 60, 0.01, 90, 10, 1, prec, m=4, d=2)
        with Integrator(pb, user_source=src) as it:
            it.set_params(torch.tensor(p, dtype=dtt[prec]).cuda(), torch.tensor(x0, dtype=dtt[prec]).cuda())
            it.integrate()
            it.frames()
            torch.cuda.synchronize()
    status("user model")

    for prec in ("fp32", "fp64"):
        p, x0 = inputs.kuramoto(32, 300, seed=10)
        pt, xt = torch.tensor(p, dtype=dtt[prec]).cuda(), torch.tensor(x0, dtype=dtt[prec]).cuda()
        pb = sdeb.Problem.make("kuramoto", 32, 300, 0.01, 100, 10, 1, prec)
        xf, fr = torch.empty_like(xt), torch.empty((11, 300, 32), dtype=dtt[prec], device="cuda")
        sdeb.sdeb_integrate_noalloc(pb, ctypes.c_void_p(pt.data_ptr()), ctypes.c_void_p(xt.data_ptr()),
                                    ctypes.c_void_p(xf.data_ptr()), ctypes.c_void_p(fr.data_ptr()))
        with Integrator(pb) as it:
            it.set_params(pt, xt)
            it.integrate()
            it.moments(order_param=True)
            it.moments(begin=3, count=5, order_param=True, device="cpu")
        torch.cuda.synchronize()
    status("noalloc and moments")

    p, x0 = inputs.kuramoto(16, 8, seed=11)
    pb = sdeb.Problem.make("kuramoto", 16, 1, 0.01, 100, 100, 0, "fp32")
    with SwarmSearch(pb, p[0].copy(), x0, [0, 1], [0.0, 0.0], [4.0, 0.5], 40, r_target=0.8, swarm_seed=3) as s:
        g = torch.Generator().manual_seed(1)
        s.reset(torch.rand((40, 2), generator=g, dtype=torch.float64) * torch.tensor([4.0, 0.5]),
                torch.zeros((40, 2), dtype=torch.float64))
        s.step()
        s.step()
        torch.cuda.synchronize()
    th = torch.rand((33, 9), device="cuda")
    r, dr = torch.empty(33, device="cuda"), torch.empty_like(th)
    sdeb.sdeb_order_param(ctypes.c_void_p(th.data_ptr()), 33, 9, 0, ctypes.c_void_p(r.data_ptr()),
                          ctypes.c_void_p(dr.data_ptr()))
    out = torch.empty((3, 5, 7, 4), dtype=torch.int32, device="cuda")
    sdeb.sdeb_philox_fill(0, 0, 3, 0, 5, 0, 7, 0, ctypes.c_void_p(out.data_ptr()))
    z = torch.empty((3, 7, 6), dtype=torch.float64, device="cuda")
    sdeb.sdeb_normals_fill(0, 0, 3, 0, 7, 6, 1, ctypes.c_void_p(z.data_ptr()))
    torch.cuda.synchronize()
    status("swarm and stand-alone kernels")

    sdeb.sdeb_check_selftest()
    status("selftest")
    status("after selftest")
""")


def test_checked_build_runs_every_kernel_with_a_clear_status_word():
    import paper_1908_03869_gb300 as sdeb
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, SDEB_LIBRARY="checked"),
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    lines = [l.split() for l in r.stdout.splitlines() if l.startswith("STATUS")]
    print(r.stdout)
    by_tag = {" ".join(l[1:-2]): (int(l[-2]), l[-1]) for l in lines}
    for tag in ("forward", "adjoint", "batch", "user model", "noalloc and moments", "swarm and stand-alone kernels",
                "after selftest"):
        assert by_tag[tag] == (sdeb.SDEB_OK, "0x0"), (tag, by_tag[tag])
    st, word = by_tag["selftest"]
    assert st == sdeb.SDEB_EBOUNDS
    assert int(word, 16) == (0xFFFF << 48) | 12345
    assert "batch layouts" in r.stdout and "(128, 2)" in r.stdout and "(64, 2)" in r.stdout
