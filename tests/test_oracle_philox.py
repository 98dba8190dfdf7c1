"""Pins of the oracle's Philox-4x32-10 and uniform mapping.

External pin: cuRAND's host-side Philox4_32_10 generator (a CPU
implementation shipped with CUDA, run as a black box).  Its output group G
(counting from the generator offset divided by 4) is Philox-4x32-10 of the
counter (G div 2^16 mod 2^32, G div 2^48, G mod 2^16, 0) under key
(seed_lo, seed_hi); the oracle must reproduce every word bit for bit.  With
offsets beyond 2^50 words this reaches counter word 1 (the batched launch's
instance word), including the carry out of word 0.  Word 3 (path_hi) is
pinned on the GPU through cuRAND's device API (tests/test_gpu_philox.py).
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


def _curand_host_stream(seed: int, n_groups: int, offset: int = 0) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
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


@pytest.mark.parametrize("seed", [42, 0xFEDCBA9876543210])
@pytest.mark.parametrize("first_group", [(1 << 48) + (5 << 16) + 7,          # word 1 = 1
                                         (3 << 48) + (0xFFFFFFFF << 16) + 0xFFF0,  # carry word 0 -> 1
                                         (0x3FFF << 48) + (0x89ABCDEF << 16)])      # word 1 = 2^14 - 1
def test_philox_counter_word_1_matches_curand_offset_stream(seed, first_group):
    n_groups = 64
    ref = _curand_host_stream(seed, n_groups, offset=4 * first_group)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    words1 = set()
    for g in range(n_groups):
        G = first_group + g
        ctr = ((G >> 16) & 0xFFFFFFFF, G >> 48, G & 0xFFFF, 0)
        words1.add(ctr[1])
        assert oracle.philox(ctr, key) == [int(v) for v in ref[g]], (seed, hex(G))
    assert min(words1) > 0


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
