"""The paper's accuracy protocol (Sec. 2.3.1) on the GPU: N = 100, 64
realisations, K = 0.02 and 0.2, 400 s, the paper's five time steps
dt = 2^(l-5) / 5, l = 1..5, in FP64 (as the paper) and FP32.

* The coherence statistics <r(t)> and sigma(r(t)) every 50 s agree with
  the FP64 oracle's on the same realisations to 0.01 (dt = 0.05).
* The paper's findings hold at every dt: below K_c, <r> stays at the
  finite-size level; above it, <r> > 0.9 from t = 100 s on and
  <r(t_MAX)> > 0.93 with sigma < 0.05; <r(t_MAX)> and sigma(r(t_MAX))
  change by less than 0.04 and 0.03 across the dt sweep."""
import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build
from paper_1908_03869_gb300 import inputs

from test_oracle_paper_accuracy import coherence_stats

pytestmark = pytest.mark.gpu
DTS = [2.0 ** (l - 5) / 5 for l in range(1, 6)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def gpu_coherence_stats(K, dt, precision, n=100, orbits=64, seed=1):
    import torch
    from paper_1908_03869_gb300.integrator import Integrator

    p, x0 = inputs.kuramoto_paper_accuracy(K, orbits=orbits, n=n, seed=seed)
    steps, stride = int(round(400 / dt)), int(round(50 / dt))
    t = torch.float64 if precision == "fp64" else torch.float32
    pb = sdeb.Problem.make("kuramoto_paper", n, orbits, dt, steps, stride, 0, precision)
    with Integrator(pb) as it:
        it.set_params(torch.tensor(p, dtype=t).cuda(), torch.tensor(x0, dtype=t).cuda())
        it.integrate()
        fr = it.frames().double().cpu().numpy()
    r = np.abs(np.exp(1j * fr).mean(axis=2))
    return r.mean(axis=1), r.std(axis=1)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_accuracy_protocol(precision):
    stats = {(K, dt): gpu_coherence_stats(K, dt, precision) for K in (0.02, 0.2) for dt in DTS}
    for K in (0.02, 0.2):
        ref_mean, ref_sd = coherence_stats(K, 0.05)
        mean, sd = stats[(K, 0.05)]
        assert np.abs(mean - ref_mean).max() < 0.01, (K, mean, ref_mean)
        assert np.abs(sd - ref_sd).max() < 0.01, (K, sd, ref_sd)
    for dt in DTS:
        mean_lo, _ = stats[(0.02, dt)]
        mean_hi, sd_hi = stats[(0.2, dt)]
        assert (mean_lo < 0.2).all() and 0.05 < mean_lo[-1] < 0.15, dt
        assert (mean_hi[2:] > 0.9).all() and mean_hi[-1] > 0.93 and sd_hi[-1] < 0.05, dt
    for K in (0.02, 0.2):
        ends = np.array([stats[(K, dt)][0][-1] for dt in DTS])
        sds = np.array([stats[(K, dt)][1][-1] for dt in DTS])
        assert ends.max() - ends.min() < 0.04, (K, ends)
        assert sds.max() - sds.min() < 0.03, (K, sds)
