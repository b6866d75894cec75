"""Failure detection with host-side fault injection (SDEB_FAULT), no GPU
fault: an allocation of a context's buffers that fails comes back as
SDEB_ENOMEM naming the buffer, with nothing left allocated, and the next
context is created normally; a forward launch that fails comes back as
SDEB_ECUDA with the step counter unchanged, and integrating the same range
again gives the bits of a run without the fault.  Each case runs in a child
process so the injection plan is read afresh."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    import paper_1908_03869_gb300 as sdeb
    from paper_1908_03869_gb300 import inputs
    from paper_1908_03869_gb300.integrator import Integrator

    n, orbits = 16, 300
    p, x0 = inputs.kuramoto(n, orbits, seed=3)
    pt, xt = torch.tensor(p).cuda(), torch.tensor(x0).cuda()
    pb = sdeb.Problem.make("kuramoto", n, orbits, 0.01, 200, 20, 1, "fp64")
    mode = sys.argv[1]
    if mode == "alloc":
        try:
            sdeb.sdeb_create(pb)
            print("UNEXPECTED create succeeded")
        except sdeb.SdebError as e:
            print("STATUS", e.status, sdeb.sdeb_last_error())
        with Integrator(pb) as it:              # the following allocations succeed
            it.set_params(pt, xt)
            it.integrate()
            print("RECOVERED", float(it.final().abs().sum()))
    elif mode == "launch_tuned":
        with Integrator(pb) as it:
            it.set_params(pt, xt)
            it.autotune(trial_steps=16)          # trial launches are not counted
            it.integrate_range(0, 100)           # launch 0
            try:
                it.integrate_range(100, 200)     # launch 1: injected failure
                print("UNEXPECTED launch succeeded")
            except sdeb.SdebError as e:
                print("STATUS", e.status, sdeb.sdeb_last_error(it.ctx))
            it.integrate_range(100, 200)         # the counter stayed at 100
            got = it.final().cpu().numpy()
            lay = it.layout()
        with Integrator(pb) as ref:
            ref.set_layout(*lay)
            ref.set_params(pt, xt)
            ref.integrate()                      # launch 3
            print("SAME", bool(np.array_equal(got, ref.final().cpu().numpy())))
    else:
        with Integrator(pb) as ref:
            ref.set_params(pt, xt)
            ref.integrate()                      # launch 0
            want = ref.final().cpu().numpy()
        with Integrator(pb) as it:
            it.set_params(pt, xt)
            it.integrate_range(0, 100)           # launch 1
            try:
                it.integrate_range(100, 200)     # launch 2: injected failure
                print("UNEXPECTED launch succeeded")
            except sdeb.SdebError as e:
                print("STATUS", e.status, sdeb.sdeb_last_error(it.ctx))
            it.integrate_range(100, 200)         # the counter stayed at 100
            got = it.final().cpu().numpy()
            print("SAME", bool(np.array_equal(got, want)))
""")


def _child(mode, fault):
    env = dict(os.environ, SDEB_FAULT=fault)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT), mode], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_injected_allocation_failure_is_enomem_and_recoverable():
    import paper_1908_03869_gb300 as sdeb
    out = _child("alloc", "alloc:2")                  # parameters, state, then the frames (FP64: no compensation)
    assert "UNEXPECTED" not in out, out
    status_line = [l for l in out.splitlines() if l.startswith("STATUS")][0]
    assert int(status_line.split()[1]) == sdeb.SDEB_ENOMEM
    assert "frames" in status_line
    assert any(l.startswith("RECOVERED") for l in out.splitlines())


def test_injected_launch_failure_is_ecuda_and_the_range_can_be_rerun():
    import paper_1908_03869_gb300 as sdeb
    out = _child("launch", "launch:2")
    assert "UNEXPECTED" not in out, out
    status_line = [l for l in out.splitlines() if l.startswith("STATUS")][0]
    assert int(status_line.split()[1]) == sdeb.SDEB_ECUDA
    assert "forward kernel launch" in status_line
    assert "SAME True" in out


def test_injected_launch_counts_integrate_calls_not_tuner_trials():
    import paper_1908_03869_gb300 as sdeb
    out = _child("launch_tuned", "launch:1")
    assert "UNEXPECTED" not in out, out
    status_line = [l for l in out.splitlines() if l.startswith("STATUS")][0]
    assert int(status_line.split()[1]) == sdeb.SDEB_ECUDA
    assert "SAME True" in out
