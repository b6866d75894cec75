"""sdeb_pipe_rate: the measured per-SM, per-clock rates the benchmark's
roofline peaks are built from.  Sanity of the measurement (positive, below
the 128 lanes an SM issues per clock, FP64 slower than FP32 on this GPU,
the special-function unit slower than the FP32 fused multiply-add), repeat
stability, and argument checks."""
import pytest

import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def test_pipe_rates_are_plausible_and_repeatable():
    r = {p: sdeb.sdeb_pipe_rate(p, 2048 if p.startswith("sfu") else 256) for p in sdeb.PIPES}
    print("pipe rates per SM per clock:", r)
    for v in r.values():
        assert 0.5 < v <= 128.5
    assert r["fp64_fma"] < r["fp32_fma"]
    assert r["sfu_sin"] < r["fp32_fma"] and r["sfu_lg2"] < r["fp32_fma"] and r["sfu_sqrt"] < r["fp32_fma"]
    again = sdeb.sdeb_pipe_rate("sfu_sin", 2048)
    assert abs(again - r["sfu_sin"]) < 0.05 * r["sfu_sin"]


def test_pipe_rate_rejects_bad_arguments():
    import ctypes
    L = sdeb.lib()
    out = ctypes.c_double()
    assert L.sdeb_pipe_rate(5, 16, ctypes.byref(out), None) == sdeb.SDEB_EINVAL
    assert L.sdeb_pipe_rate(0, 0, ctypes.byref(out), None) == sdeb.SDEB_EINVAL
    assert L.sdeb_pipe_rate(0, 16, None, None) == sdeb.SDEB_EINVAL
