"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: Kuramoto n = 8 / 32 / 128 with 2^20 / 2^18 / 2^16 orbits,
dt = 0.005, 10^4 steps, a frame every 100 steps.  The oracle recomputes a
sample of orbits (the first and last and some in between) one by one."""
import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from helpers import max_rel_err, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _sample(orbits, k=6):
    rng = np.random.Generator(np.random.PCG64(orbits))
    mid = sorted(rng.choice(np.arange(1, orbits - 1), size=k, replace=False).tolist())
    return [0] + mid + [orbits - 1]


@pytest.mark.parametrize("n,orbits", [(8, 1 << 20), (32, 1 << 18), (128, 1 << 16)])
def test_full_size_fp32(n, orbits):
    sample = _sample(orbits)
    got_fr, got_fin, rfr, rfin, _ = _run_full_sampled(n, orbits, "fp32", sample)
    assert max_rel_err(got_fr, rfr) < 1e-4
    assert max_rel_err(got_fin, rfin) < 1e-4


def test_full_size_fp64_n8():
    sample = _sample(1 << 20)
    got_fr, got_fin, rfr, rfin, _ = _run_full_sampled(8, 1 << 20, "fp64", sample)
    assert max_rel_err(got_fr, rfr) < 1e-12
    assert max_rel_err(got_fin, rfin) < 1e-12


def _run_full_sampled(n, orbits, precision, sample):
    """The sampled orbits keep their global index (Philox key): the oracle is
    run per orbit with orbit_begin = that index."""
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    W = inputs.WORKLOADS["kuramoto_n%d" % n]
    p, x0 = inputs.kuramoto(n, orbits, seed=1)
    dt_t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make("kuramoto", n, orbits, W["dt"], W["steps"], W["stride"], W["seed"], precision)
    with Integrator(pb) as it:
        pt = torch.tensor(p, dtype=dt_t).cuda()
        xt = torch.tensor(x0, dtype=dt_t).cuda()
        it.set_params(pt, xt)
        it.integrate()
        idx = torch.tensor(sample, device="cuda")
        got_fr = it.frames()[:, idx].cpu().numpy()
        got_fin = it.final()[idx].cpu().numpy()
        assert it.flags().sum().item() == 0
        p_s = pt.cpu().numpy().astype(np.float64)
        x_s = xt.cpu().numpy().astype(np.float64)
    rfr, rfin = run_oracle("kuramoto", n, p_s, x_s, W["dt"], W["steps"], W["stride"], W["seed"],
                           mean_field=True, orbits=sample)
    return got_fr, got_fin, rfr, rfin, sample
