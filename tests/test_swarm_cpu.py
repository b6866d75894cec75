"""Argument checks of the swarm entry points (sdeb_swarm_*), without a GPU:
every refusal happens before any CUDA call."""
import ctypes

import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

P = ctypes.c_void_p(256)     # never dereferenced: each call below is refused first


@pytest.fixture(scope="module", autouse=True)
def _lib():
    sdeb_build.build()
    sdeb.lib()


def _status(fn, *args):
    with pytest.raises(sdeb.SdebError) as e:
        fn(*args)
    assert sdeb.sdeb_last_error()
    return e.value.status


def test_expand_refusals():
    ok = (P, 4, [0, 1], P, 10, 3, "fp64", P)
    for bad in ((P, 4, [0, 10], P, 10, 3, "fp64", P),          # column outside [0, d)
                (P, 4, [1, 1], P, 10, 3, "fp64", P),           # a column twice
                (P, 0, [0], P, 10, 3, "fp64", P), (P, 4, [0], P, 10, 0, "fp64", P),
                (P, 4, list(range(17)), P, 40, 3, "fp64", P),  # more than SDEB_SWARM_MAX_DIMS
                (P, 4, [0], P, 10, 3, 7, P), (None, 4, [0], P, 10, 3, "fp64", P)):
        assert _status(sdeb.sdeb_swarm_expand, *bad) == sdeb.SDEB_EINVAL, bad
    assert len(ok) == 8


def test_fitness_and_update_refusals():
    assert _status(sdeb.sdeb_swarm_fitness, P, 0, 2, 8, "fp64", 0.5, P) == sdeb.SDEB_EINVAL
    assert _status(sdeb.sdeb_swarm_fitness, None, 4, 2, 8, "fp64", 0.5, P) == sdeb.SDEB_EINVAL
    assert _status(sdeb.sdeb_swarm_fitness, P, 4, 2, 0, "fp64", 0.5, P) == sdeb.SDEB_EINVAL
    upd = sdeb.sdeb_swarm_update
    assert _status(upd, P, P, P, P, P, 4, [1.0], [0.0], 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL   # lo > hi
    assert _status(upd, P, P, P, P, P, 4, [float("nan")], [1.0], 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL
    assert _status(upd, P, P, P, P, P, 0, [0.0], [1.0], 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL
    assert _status(upd, P, P, P, P, P, 2 ** 24 + 1, [0.0], [1.0], 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL
    assert _status(upd, P, P, None, P, P, 4, [0.0], [1.0], 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL
    assert _status(upd, P, P, P, P, P, 4, [0.0] * 17, [1.0] * 17, 0.7, 1.5, 1.5, 1, 0, P) == sdeb.SDEB_EINVAL
