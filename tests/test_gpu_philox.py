"""Bit-exact checks of the integer Philox-4x32-10 stream on the GPU.

* cuRAND's device-side Philox4_32_10 (curand_init(seed, subsequence, offset)
  followed by curand4, run as a black box) produces Philox-4x32-10 of the
  counter (offset/4 mod 2^32, offset/4 div 2^32, subsequence mod 2^32,
  subsequence div 2^32) under key (seed_lo, seed_hi).  The oracle must
  reproduce every word on counters whose four words are all non-zero: this
  pins counter words 1 and 3 (instance and path_hi of the path kernels),
  which cuRAND's host generator cannot reach beyond word 1.
* The library's device generator (lll_philox_words, the function every path
  kernel draws from) must equal the oracle word for word on the same and on
  random counters.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import oracle as ora

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


@pytest.fixture(scope="module")
def curand_words(lll):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not available to build the cuRAND helper")
    d = tempfile.mkdtemp(prefix="curand_words_")
    so = os.path.join(d, "libcurand_words.so")
    src = os.path.join(HERE, "gpu_helpers", "curand_device_words.cu")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    lib.curand_device_words.restype = ctypes.c_int
    lib.curand_device_words.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p]

    def run(seed, sub, off):
        sub = np.ascontiguousarray(sub, dtype=np.uint64)
        off = np.ascontiguousarray(off, dtype=np.uint64)
        out = np.zeros((len(sub), 4), dtype=np.uint32)
        rc = lib.curand_device_words(ctypes.c_ulonglong(seed), sub.ctypes.data, off.ctypes.data, len(sub),
                                     out.ctypes.data)
        assert rc == 0, rc
        return out

    yield run
    shutil.rmtree(d, ignore_errors=True)


def _counters(rng, count):
    c = rng.integers(1, 2 ** 32, size=(count, 4), dtype=np.uint64).astype(np.uint32)
    c[:4] = [[0xFFFFFFFF, 1, 0, 1], [0, 0xFFFFFFFF, 1, 0xFFFFFFFF], [7, 3, 5, 2], [1, 1, 1, 1]]
    return c


@pytest.mark.parametrize("seed", [42, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_oracle_matches_curand_device_generator_on_all_four_counter_words(curand_words, seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    ctr = _counters(rng, 256)
    sub = ctr[:, 2].astype(np.uint64) | (ctr[:, 3].astype(np.uint64) << np.uint64(32))
    off4 = ctr[:, 0].astype(np.uint64) | (ctr[:, 1].astype(np.uint64) << np.uint64(32))
    ok = off4 < np.uint64(1 << 62)  # offsets are 64-bit words: offset/4 < 2^62
    ctr, sub, off4 = ctr[ok], sub[ok], off4[ok]
    assert np.all(ctr[4:, 1] > 0) and np.all(ctr[4:, 3] > 0)
    ref = curand_words(seed, sub, off4 * np.uint64(4))
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for c, r in zip(ctr, ref):
        assert ora.philox(tuple(int(v) for v in c), key) == [int(v) for v in r], c


@pytest.mark.parametrize("seed", [42, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_library_device_words_equal_oracle_bit_for_bit(lll, seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    ctr = _counters(rng, 4096)
    # the path kernels' own counters: (step, instance, path_lo, path_hi)
    ctr[4:36] = [[k, q, p & 0xFFFFFFFF, p >> 32] for k, q, p in
                 zip(range(32), range(255, 255 - 32, -1), [(1 << 32) + 3 * i for i in range(32)])]
    got = lll.lll_philox_words(ctr, seed)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for c, g in zip(ctr, got):
        assert ora.philox(tuple(int(v) for v in c), key) == [int(v) for v in g], c
