"""Pins of the oracle's Philox-4x32-10 and uniform mapping.

External pin: cuRAND's host-side Philox4_32_10 generator (a CPU
implementation shipped with CUDA, run as a black box).  Its output group g
is Philox-4x32-10 of counter (g div 2^16, 0, g mod 2^16, 0) under key
(seed_lo, seed_hi); the oracle must reproduce every word bit for bit.  The
path kernels use counter (step, instance, path_lo, path_hi), so for one
instance and fewer than 2^32 paths every draw they make sits in the pinned
(word 0, word 2) plane.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from oracle import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    for path in ("/usr/local/cuda/lib64/libcurand.so",):
        try:
            return ctypes.CDLL(path)
        except OSError:
            pass
    return None


def _curand_host_stream(seed: int, n_groups: int) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_groups, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [42, 0x123456789ABCDEF0, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host_generator(seed):
    n_groups = (1 << 16) * 3 + 1000
    ref = _curand_host_stream(seed, n_groups)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    rng = np.random.default_rng(1)
    groups = np.concatenate([np.arange(2048), rng.integers(0, n_groups, 3000),
                             [65535, 65536, 65537, 131072, n_groups - 1]])
    for g in groups:
        g = int(g)
        got = oracle.philox((g >> 16, 0, g & 0xFFFF, 0), key)
        assert got == [int(v) for v in ref[g]], (seed, g)


def test_philox_uses_every_counter_and_key_word():
    base = oracle.philox((5, 6, 7, 8), (9, 10))
    for pos in range(4):
        ctr = [5, 6, 7, 8]
        ctr[pos] ^= 1
        out = oracle.philox(ctr, (9, 10))
        assert all(a != b for a, b in zip(out, base)), pos
    for pos in range(2):
        key = [9, 10]
        key[pos] ^= 1
        out = oracle.philox((5, 6, 7, 8), key)
        assert all(a != b for a, b in zip(out, base)), pos


def test_philox_bit_balance():
    # Each output bit is one with probability 1/2 (binomial 5-sigma band).
    words = np.array([oracle.philox((k, 3, p, 0), (42, 0)) for k in range(64) for p in range(64)],
                     dtype=np.uint64)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 128)
    frac = bits.mean(axis=0)
    nsamp = bits.shape[0]
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / np.sqrt(nsamp))


def test_unit_uniform_mapping_is_exact_in_fp32():
    # u = ((w >> 9) + 0.5) 2^-23: odd multiples of 2^-24, so FP32 holds them exactly.
    w = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFFFF, 0xFFFFFE00], dtype=np.uint64)
    u = ((w >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert u.min() == 2.0 ** -24 and u.max() == 1 - 2.0 ** -24
