"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11).

The oracle is checked against two independent library implementations of the
same published generator: cuRAND's host-side PHILOX4_32_10 generator (which
runs on the CPU) and Triton's ``tl.philox`` run by Triton's CPU interpreter.
Neither shares code with the oracle.
"""
import ctypes
import ctypes.util
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

MASK32 = 0xFFFFFFFF


def _curand_host_words(seed, nwords):
    name = ctypes.util.find_library("curand")
    candidates = [name] if name else []
    candidates += ["libcurand.so", "/usr/local/cuda/lib64/libcurand.so"]
    lib = None
    for c in candidates:
        try:
            lib = ctypes.CDLL(c)
            break
        except OSError:
            continue
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    out = np.zeros(nwords, dtype=np.uint32)
    assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host generator emits, for its first blocks, Philox4x32-10 of
    # counter (0, 0, i, 0) under key (seed lo32, seed hi32).
    nblocks = 256
    words = _curand_host_words(seed, 4 * nblocks).reshape(nblocks, 4)
    key = [seed & MASK32, (seed >> 32) & MASK32]
    for i in range(nblocks):
        got = oracle.philox([0, 0, i, 0], key)
        np.testing.assert_array_equal(got, words[i], err_msg="block %d" % i)


_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        c0 = tl.load(c_ptr + offs * 4 + 0)
        c1 = tl.load(c_ptr + offs * 4 + 1)
        c2 = tl.load(c_ptr + offs * 4 + 2)
        c3 = tl.load(c_ptr + offs * 4 + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + offs * 4 + 0, a)
        tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c)
        tl.store(out_ptr + offs * 4 + 3, d)

    spec = json.loads(sys.argv[1])
    res = {}
    for seed, ctrs in spec:
        c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32)).contiguous()
        out = torch.zeros_like(c)
        k[(1,)](c, out, seed, N=len(ctrs))
        res[str(seed)] = out.numpy().view(np.uint32).tolist()
    print(json.dumps(res))
    """
)


def test_philox_matches_triton_interpreter():
    pytest.importorskip("triton")
    import json

    rng = np.random.Generator(np.random.PCG64(7))
    spec = []
    for seed in [0, 3, 0xDEADBEEF12345678]:
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [MASK32, MASK32, MASK32, MASK32]
        spec.append([seed, ctrs.tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, json.dumps(spec)],
                          capture_output=True, text=True, timeout=600, env=env)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    res = json.loads(proc.stdout.strip().splitlines()[-1])
    for seed, ctrs in spec:
        want = np.array(res[str(seed)], dtype=np.uint32).reshape(-1, 4)
        key = [seed & MASK32, (seed >> 32) & MASK32]
        for i, c in enumerate(ctrs):
            np.testing.assert_array_equal(oracle.philox(c, key), want[i])


def test_counter_layout_of_wiener_blocks():
    # Reading of Sec. 2.1.2: counter = (step k, noise block b, orbit o, stream).
    seed = 0x0102030405060708
    key = [seed & MASK32, seed >> 32]
    grid = oracle.philox_fill(seed, 5, 3, 2, 2, 1000, 4, stream=0)
    for k in range(3):
        for b in range(2):
            for o in range(4):
                np.testing.assert_array_equal(grid[k, b, o], oracle.philox([5 + k, 2 + b, 1000 + o, 0], key))
    other = oracle.philox_fill(seed, 5, 1, 2, 1, 1000, 1, stream=1)
    assert not np.array_equal(other[0, 0, 0], grid[0, 0, 0])


def test_philox_words_are_uniform():
    # 2^20 words: byte histogram and top-bit balance (chi-square at a loose level).
    w = oracle.philox_fill(11, 0, 64, 0, 16, 0, 256).reshape(-1)
    counts = np.bincount((w & 0xFF).astype(np.int64), minlength=256)
    expected = w.size / 256.0
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 400.0  # 255 dof; mean 255, sd ~22.6
    assert abs((w >> 31).mean() - 0.5) < 0.005
