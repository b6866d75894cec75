"""Host logic of the batch scheduler (sdeb_batch_plan: no GPU needed).

The schedule must place every orbit exactly once; a packed warp holds items
of one units-per-lane value side by side within 32 lanes, each on
ceil(n / P) lanes, with step counts within a factor 1.2 of each other;
teams hold one item on 64 or 128 lanes.  Without a chain limit nothing runs
as a team; with the tightest limit every item takes the layout of the
shortest chain for its n, 2 units per lane: a warp of its own up to n = 64,
a 64-lane team up to 128, a 128-lane team above."""
import math

import numpy as np
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build


@pytest.fixture(scope="module", autouse=True)
def _built():
    sdeb_build.build()
    sdeb.lib()


def _problems(count, seed, k_low=10, k_high=20000):
    rng = np.random.Generator(np.random.PCG64(seed))
    pbs = []
    for i in range(count):
        n = int(rng.integers(1, 257))
        steps = int(round(math.exp(rng.uniform(math.log(k_low), math.log(k_high)))))
        orbits = 3 if i % 7 == 0 else 1
        pbs.append(sdeb.Problem.make("kuramoto", n, orbits, 0.01, steps, 100, 1, "fp32", orbit_offset=10 * i))
    return pbs


def _per_orbit(pbs, key):
    return np.concatenate([np.full(pb.orbits, getattr(pb, key)) for pb in pbs])


@pytest.mark.parametrize("frac", [1e-9, 0.05, 0.25, 1.0, 1e9])
def test_every_orbit_placed_once_and_warps_packed_within_32_lanes(frac):
    pbs = _problems(300, 1)
    plan = sdeb.sdeb_batch_plan(pbs, frac, 152)
    n = _per_orbit(pbs, "n")
    steps = _per_orbit(pbs, "steps")
    inst_of = np.concatenate([np.full(pb.orbits, i) for i, pb in enumerate(pbs)])
    lanes = plan["lanes"][inst_of]
    upl = plan["units_per_lane"][inst_of]
    assert (plan["task"] >= 0).all() and (plan["task"] < plan["tasks"]).all()
    assert (lanes * upl >= n).all()
    packed = plan["slot"] <= 3
    assert np.isin(upl[packed], [8, 4, 2]).all()        # 2: an orbit alone on its warp
    assert (lanes[packed] == -(-n[packed] // upl[packed])).all()
    assert (lanes[packed] <= 32).all()
    team64 = (plan["slot"] == 4) | (plan["slot"] == 5)
    assert (lanes[team64] == 64).all() and np.isin(upl[team64], [4, 2]).all()
    team128 = plan["slot"] == 6
    assert (lanes[team128] == 128).all() and (upl[team128] == 2).all()
    groups = {}
    for g in range(len(n)):
        groups.setdefault((plan["task"][g], plan["slot"][g]), []).append(g)
    for (t, slot), members in groups.items():
        if slot >= 4:
            assert len(members) == 1                      # one item per team
            continue
        assert len({int(upl[g]) for g in members}) == 1   # one units-per-lane value per warp
        if upl[members[0]] == 2:
            assert len(members) == 1                      # a single-warp orbit has the warp to itself
        spans = sorted((int(plan["lane0"][g]), int(plan["lane0"][g] + lanes[g])) for g in members)
        assert spans[0][0] == 0 and spans[-1][1] <= 32
        for (a0, a1), (b0, _) in zip(spans, spans[1:]):
            assert a1 == b0                               # side by side, no overlap, no gap
        ks = steps[members]
        assert ks.max() <= 1.2 * ks.min() + 1e-9          # one bucket of similar step counts
    # a task holds either packed warps or teams, never both
    for t in range(plan["tasks"]):
        slots = set(plan["slot"][plan["task"] == t].tolist())
        assert slots <= {0, 1, 2, 3} or slots <= {4, 5} or slots == {6}


def test_chain_limit_extremes():
    pbs = _problems(300, 2)
    loose = sdeb.sdeb_batch_plan(pbs, 1e9, 152)
    assert (loose["slot"] <= 3).all() and (loose["lanes"] <= 32).all()
    tight = sdeb.sdeb_batch_plan(pbs, 1e-9, 152)
    for i, pb in enumerate(pbs):
        if pb.n <= 64:
            want = (-(-pb.n // 2), 2)    # a warp of its own
        else:
            want = (64, 2) if pb.n <= 128 else (128, 2)
        assert (tight["lanes"][i], tight["units_per_lane"][i]) == want, (pb.n, pb.steps)


def test_plan_is_deterministic_and_matches_orbit_order():
    pbs = _problems(120, 3)
    a = sdeb.sdeb_batch_plan(pbs, 0.3, 152)
    b = sdeb.sdeb_batch_plan(pbs, 0.3, 152)
    for k in ("lanes", "units_per_lane", "task", "slot", "lane0"):
        np.testing.assert_array_equal(a[k], b[k])
    # every task is used by some orbit
    assert len(set(a["task"].tolist())) == a["tasks"]


def test_plan_rejects_bad_arguments():
    import ctypes
    pbs = _problems(5, 4)
    for frac, sms in ((0.0, 152), (-1.0, 152), (float("inf"), 152), (0.5, 0)):
        with pytest.raises(sdeb.SdebError) as e:
            sdeb.sdeb_batch_plan(pbs, frac, sms)
        assert e.value.status == sdeb.SDEB_EINVAL
    arr = (sdeb.Problem * len(pbs))(*pbs)
    buf = (ctypes.c_int32 * 64)()
    st = sdeb.lib().sdeb_batch_plan(ctypes.cast(arr, ctypes.c_void_p), len(pbs), 0.5, 152, None, None,
                                    63, ctypes.cast(buf, ctypes.c_void_p), None, None, None)
    assert st == sdeb.SDEB_EINVAL                          # total_orbits does not match
    bad = list(pbs)
    bad[2] = sdeb.Problem.make("ou", 4, 1, 0.01, 10, 1, 1, "fp32")
    with pytest.raises(sdeb.SdebError) as e:
        sdeb.sdeb_batch_plan(bad, 0.5, 152)
    assert e.value.status == sdeb.SDEB_EUNSUPPORTED
