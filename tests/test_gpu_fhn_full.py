"""Parity of the FitzHugh-Nagumo network workload at full size: 64 units
(n = 128, m = 64), 2^18 orbits, dt = 0.01, 10^5 steps, a frame every 1000.

FP32 runs the whole horizon (t = 1000); FP64 the first 2*10^4 steps.  On a
fixed sample of orbits, recomputed by the oracle: FP32 <= 1e-4 and
FP64 <= 1e-12 over the first 1000 steps (t <= 10), FP32 <= 1e-3 over the
whole horizon, FP64 <= 1e-10 over its 2*10^4 steps.  The excitable units
with multiplicative noise amplify rounding differences (spike timing); the
oracle alone shows it (test_oracle_sensitivity.py).  Over all orbits, FP32
and FP64 agree in the orbit mean of every state component to 1e-4 over the
common 2*10^4 steps.
"""
import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _err(x, ref):
    return (np.abs(x - ref) / np.maximum(np.abs(ref), 1.0)).max(axis=(1, 2))


def test_fhn_full_size():
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    W = inputs.WORKLOADS["fhn_64units"]
    n, orbits = W["n"], W["orbits"]
    p, x0 = inputs.fhn(n // 2, orbits, seed=1)
    p, x0 = p.astype(np.float32).astype(np.float64), x0.astype(np.float32).astype(np.float64)
    sample = [0, 4099, 123456, orbits - 1]
    idx = torch.tensor(sample, device="cuda")
    out = {}
    for prec, steps in (("fp32", W["steps"]), ("fp64", 20000)):
        dt_t = torch.float64 if prec == "fp64" else torch.float32
        pb = sdeb.Problem.make("fhn_net", n, orbits, W["dt"], steps, W["stride"], W["seed"], prec)
        with Integrator(pb) as it:
            it.set_params(torch.tensor(p, dtype=dt_t).cuda(), torch.tensor(x0, dtype=dt_t).cuda())
            it.integrate()
            assert it.flags().sum().item() == 0
            fr = it.frames()
            out[prec] = (fr[:, idx].cpu().numpy().astype(np.float64),
                         fr[:21].mean(dim=1, dtype=torch.float64).cpu().numpy())
            del fr
    e32 = _err(out["fp32"][0], run_oracle("fhn_net", n, p, x0, W["dt"], W["steps"], W["stride"], W["seed"],
                                         orbits=sample)[0])
    e64 = _err(out["fp64"][0], run_oracle("fhn_net", n, p, x0, W["dt"], 20000, W["stride"], W["seed"],
                                         orbits=sample)[0])
    assert e32[:2].max() < 1e-4, e32[:2]
    assert e64[:2].max() < 1e-12, e64[:2]
    assert e32.max() < 1e-3, e32.max()
    assert e64.max() < 1e-10, e64.max()
    mean32, mean64 = out["fp32"][1], out["fp64"][1]
    assert np.abs(mean32 - mean64).max() < 1e-4, np.abs(mean32 - mean64).max()
