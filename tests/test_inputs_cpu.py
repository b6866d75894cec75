"""The seeded input generators (paper_1908_03869_gb300/inputs.py) draw the
workloads' stated distributions: Kuramoto omega ~ N(0, 1), K ~ U(0, 4),
sigma ~ U(0.1, 0.5), theta(0) ~ U(0, 2 pi); the paper's speed protocol
(Sec. 2.2.1: K = 1, omega ~ U(0.01, 0.03), p ~ U(0.001, 0.003),
theta(0) ~ U(-pi, pi)) and accuracy protocol (Sec. 2.3.1: omega ~ U(0.2, 0.4),
whose density 5 at the centre gives K_c = 2 / (5 pi)); the FitzHugh-Nagumo
parameter ranges; the batch's n ~ U{2..256}, steps log-uniform on
[10^3, 10^5] and dt in {0.001, 0.01} with equal odds; and the workload
table's sizes.  Same seed, same arrays."""
import math

import numpy as np
from scipy import stats

from paper_1908_03869_gb300 import inputs


def test_kuramoto_distributions_and_determinism():
    p, x0 = inputs.kuramoto(32, 20000, seed=5)
    assert p.shape == (20000, 34) and x0.shape == (20000, 32)
    assert p[:, 0].min() >= 0.0 and p[:, 0].max() < 4.0
    assert p[:, 1].min() >= 0.1 and p[:, 1].max() < 0.5
    assert stats.kstest(p[:, 0] / 4.0, "uniform").pvalue > 1e-3
    om = p[:, 2:].ravel()
    assert abs(om.mean()) < 0.01 and abs(om.std() - 1.0) < 0.01
    assert stats.kstest(om[:50000], "norm").pvalue > 1e-3
    assert x0.min() >= 0.0 and x0.max() < 2 * math.pi
    p2, x2 = inputs.kuramoto(32, 20000, seed=5)
    np.testing.assert_array_equal(p, p2)
    np.testing.assert_array_equal(x0, x2)
    ps, _ = inputs.kuramoto(32, 10, seed=5, shared=True)
    assert ps.shape == (34,)


def test_paper_protocol_distributions():
    p, x0 = inputs.kuramoto_paper_speed(15, 4000, seed=2)
    assert p.shape == (4000, 31)
    assert np.all(p[:, 0] == 1.0)
    assert p[:, 1:16].min() >= 0.01 and p[:, 1:16].max() <= 0.03
    assert p[:, 16:].min() >= 0.001 and p[:, 16:].max() <= 0.003
    assert x0.min() >= -math.pi and x0.max() <= math.pi
    p, x0 = inputs.kuramoto_paper_accuracy(0.2, orbits=64, n=100, seed=3)
    assert p.shape == (64, 201) and np.all(p[:, 0] == 0.2)
    om = p[:, 1:101]
    assert om.min() >= 0.2 and om.max() <= 0.4
    g0 = 1.0 / (0.4 - 0.2)                      # uniform density at its centre
    assert abs(2.0 / (math.pi * g0) - 2.0 / (5.0 * math.pi)) < 1e-15
    assert p[:, 101:].min() >= 0.01 and p[:, 101:].max() <= 0.03


def test_fhn_parameter_ranges():
    p, x0 = inputs.fhn(64, 5000, seed=4)
    assert p.shape == (5000, 6) and x0.shape == (5000, 128)
    for col, (lo, hi) in enumerate([(0.6, 0.8), (0.7, 0.9), (0.05, 0.1), (0.3, 0.6), (0.0, 0.5), (0.01, 0.1)]):
        assert p[:, col].min() >= lo and p[:, col].max() <= hi, col


def test_batched_instances_distributions():
    inst = inputs.batched_instances(count=4096, seed=0)
    n = np.array([i["n"] for i in inst])
    k = np.array([i["steps"] for i in inst])
    dt = np.array([i["dt"] for i in inst])
    assert n.min() >= 2 and n.max() <= 256
    assert stats.chisquare(np.bincount(n - 2, minlength=255)).pvalue > 1e-4
    assert k.min() >= 1000 and k.max() <= 100000
    u = (np.log(k) - math.log(1e3)) / (math.log(1e5) - math.log(1e3))
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    assert set(np.unique(dt)) == {0.001, 0.01}
    assert abs((dt == 0.001).mean() - 0.5) < 0.03
    for i in inst[:50]:
        assert i["params"].shape == (i["n"] + 2,) and i["x0"].shape == (i["n"],)


def test_workload_table_sizes():
    W = inputs.WORKLOADS
    assert (W["kuramoto_n4_fp64"]["n"], W["kuramoto_n4_fp64"]["orbits"], W["kuramoto_n4_fp64"]["steps"],
            W["kuramoto_n4_fp64"]["stride"], W["kuramoto_n4_fp64"]["dt"]) == (4, 1024, 1000, 10, 0.01)
    for name, n, orbits in (("kuramoto_n8", 8, 1 << 20), ("kuramoto_n32", 32, 1 << 18),
                            ("kuramoto_n128", 128, 1 << 16)):
        w = W[name]
        assert (w["n"], w["orbits"], w["dt"], w["steps"], w["stride"]) == (n, orbits, 0.005, 10000, 100)
    a = W["kuramoto_adjoint_n32"]
    assert (a["n"], a["orbits"], a["dt"], a["steps"], a["ckpt_every"]) == (32, 16384, 0.01, 2000, 100)
    f = W["fhn_64units"]
    assert (f["n"], f["orbits"], f["dt"], f["steps"]) == (128, 1 << 18, 0.01, 100000)
    assert W["batched_4096"]["count"] == 4096
