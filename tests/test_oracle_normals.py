"""Pins for the oracle's uniform map and Box-Muller transform (Eq. 3).

Special cases reduce to closed forms (angle 0, pi/2, pi; the extreme
uniforms), and the bulk stream is checked against the standard normal
distribution (moments, Kolmogorov-Smirnov via scipy, chi-square radius,
pair independence).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def test_uniform_endpoints_and_spacing():
    assert oracle.uniform(0) == 2.0 ** -33
    assert oracle.uniform(2**32 - 1) == 1.0 - 2.0 ** -33
    assert oracle.uniform(2**31) == 0.5 + 2.0 ** -33
    for w in [0, 1, 12345, 2**31 - 1, 2**32 - 2, 2**32 - 1]:
        u = oracle.uniform(w)
        assert 0.0 < u < 1.0
        assert u == (w + 0.5) / 2.0**32


def test_box_muller_special_angles():
    w_first = 123456789
    radius = math.sqrt(-2.0 * math.log((w_first + 0.5) / 2.0**32))
    # angle ~ 0: cos branch = radius, sin branch ~ 0
    z = oracle.box_muller(w_first, 0)
    assert z[0] == pytest.approx(radius, rel=1e-15)
    assert abs(z[1]) < 1e-8 * radius
    # angle ~ pi/2 (U2 = 1/4): cos ~ 0, sin = radius
    z = oracle.box_muller(w_first, 2**30)
    assert abs(z[0]) < 1e-8 * radius
    assert z[1] == pytest.approx(radius, rel=1e-15)
    # angle ~ pi: cos branch = -radius
    z = oracle.box_muller(w_first, 2**31)
    assert z[0] == pytest.approx(-radius, rel=1e-15)
    # angle ~ 3 pi / 2: sin branch = -radius
    z = oracle.box_muller(w_first, 3 * 2**30)
    assert z[1] == pytest.approx(-radius, rel=1e-15)


def test_box_muller_extreme_radii():
    # U1 = 2^-33: radius = sqrt(66 ln 2); U1 = 1 - 2^-33: radius ~ 2^-16
    z = oracle.box_muller(0, 0)
    assert z[0] == pytest.approx(math.sqrt(66.0 * math.log(2.0)), rel=1e-14)
    z = oracle.box_muller(2**32 - 1, 0)
    assert z[0] == pytest.approx(2.0 ** -16, rel=1e-6)
    assert np.all(np.isfinite(z))


def test_normals_distribution():
    m = 8
    z = oracle.normals_fill(3, 0, 256, 0, 512, m)   # 2^20 draws
    x = z.reshape(-1)
    nsd = 1.0 / math.sqrt(x.size)
    assert abs(x.mean()) < 6 * nsd
    assert abs(x.var() - 1.0) < 6 * math.sqrt(2.0) * nsd
    assert abs(stats.skew(x)) < 6 * math.sqrt(6.0) * nsd
    assert abs(stats.kurtosis(x)) < 6 * math.sqrt(24.0) * nsd
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # radius^2 of each Box-Muller pair is chi-square with 2 dof
    pairs = z.reshape(-1, 2)
    r2 = (pairs ** 2).sum(axis=1)
    assert stats.kstest(r2, "chi2", args=(2,)).pvalue > 1e-4
    # the two members of a pair, and neighbouring pairs, are uncorrelated
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 6 * 2 * nsd
    blocks = z.reshape(-1, 4)
    assert abs(np.corrcoef(blocks[:, 0], blocks[:, 2])[0, 1]) < 6 * 4 * nsd
    # different steps and orbits are uncorrelated
    assert abs(np.corrcoef(z[:-1, :, 0].ravel(), z[1:, :, 0].ravel())[0, 1]) < 0.02
    assert abs(np.corrcoef(z[:, :-1, 0].ravel(), z[:, 1:, 0].ravel())[0, 1]) < 0.02


def test_normals_block_structure():
    # words past m are discarded; m = 5 is a prefix of m = 8, and normal j
    # comes from block j // 4 only
    a = oracle.normals_fill(9, 17, 3, 40, 5, 5)
    b = oracle.normals_fill(9, 17, 3, 40, 5, 8)
    np.testing.assert_array_equal(a, b[:, :, :5])
    w = oracle.philox_fill(9, 17, 1, 1, 1, 40, 1)[0, 0, 0]
    np.testing.assert_array_equal(b[0, 0, 4:6], oracle.box_muller(w[0], w[1]))
    np.testing.assert_array_equal(b[0, 0, 6:8], oracle.box_muller(w[2], w[3]))
