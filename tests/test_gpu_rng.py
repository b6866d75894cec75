"""GPU parity of the noise: Philox words bit-exact, Box-Muller normals to rounding."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1908_03869_gb300 as sdeb
from paper_1908_03869_gb300 import build as sdeb_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sdeb_build.build()
    sdeb.lib()


def _gpu_philox(seed, k0, nk, b0, nb, o0, no, stream_id=0):
    import torch
    out = torch.empty((nk, nb, no, 4), dtype=torch.int32, device="cuda")
    sdeb.sdeb_philox_fill(seed, k0, nk, b0, nb, o0, no, stream_id, ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 0x8000000000000005, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("k0,b0,o0", [(0, 0, 0), (2**32 - 3, 7, 2**32 - 64), (123456, 1, 99999)])
def test_philox_bit_exact(seed, k0, b0, o0):
    nk, nb, no = 3, 3, 64
    got = _gpu_philox(seed, k0, nk, b0, nb, o0, no)
    want = oracle.philox_fill(seed, k0, nk, b0, nb, o0, no)
    np.testing.assert_array_equal(got, want)


def test_philox_bit_exact_large_grid_and_stream_word():
    got = _gpu_philox(42, 1000, 16, 0, 32, 5000, 256, stream_id=1)
    want = oracle.philox_fill(42, 1000, 16, 0, 32, 5000, 256, stream=1)
    np.testing.assert_array_equal(got, want)


def _gpu_normals(seed, k0, nk, o0, no, m, precision):
    import torch
    dt = torch.float64 if precision == sdeb.SDEB_FP64 else torch.float32
    out = torch.empty((nk, no, m), dtype=dt, device="cuda")
    sdeb.sdeb_normals_fill(seed, k0, nk, o0, no, m, precision, ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m", [1, 3, 4, 8, 13, 64])
def test_normals_fp64_match_oracle(m):
    got = _gpu_normals(7, 10, 20, 300, 200, m, sdeb.SDEB_FP64)
    want = oracle.normals_fill(7, 10, 20, 300, 200, m)
    # CUDA and the host libm each round log / sqrt / sin / cos within a few ulp
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14)


def _fp32_bound(want):
    """Error budget of the FP32 Box-Muller: the angle part (SFU sin / cos
    absolute error and the float rounding of 2 pi a, together < 1e-6) scales
    with the pair's radius r; the radius part (SFU log2 / sqrt, with the
    series branch within 2^-4 of U1 = 1) is relative to |N|."""
    pairs = want.reshape(-1, 2)
    r = np.repeat(np.sqrt((pairs ** 2).sum(axis=1)), 2).reshape(want.shape)
    return 1e-6 * (r + np.abs(want)) + 1e-7


def test_normals_fp32_match_oracle():
    got = _gpu_normals(3, 0, 64, 0, 4096, 8, sdeb.SDEB_FP32_KAHAN)   # 2^21 normals
    want = oracle.normals_fill(3, 0, 64, 0, 4096, 8)
    excess = np.abs(got - want) / _fp32_bound(want)
    assert excess.max() < 1.0, excess.max()


def test_normals_fp32_extreme_words():
    # every step has some orbits whose radius word is within 2^-10 of 2^32
    got = _gpu_normals(11, 0, 256, 0, 4096, 4, sdeb.SDEB_FP32_KAHAN)
    want = oracle.normals_fill(11, 0, 256, 0, 4096, 4)
    words = oracle.philox_fill(11, 0, 256, 0, 1, 0, 4096)[:, 0, :, 0]
    near_one = words >= 2**32 - 2**22
    assert near_one.sum() > 100
    excess = np.abs(got - want) / _fp32_bound(want)
    assert excess[near_one].max() < 1.0
    assert excess.max() < 1.0
    assert np.all(np.isfinite(got))
