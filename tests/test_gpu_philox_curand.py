"""The oracle's Philox4x32-10 against cuRAND's (an independent implementation of Salmon et al.'s generator), word
for word at many keys and counters: random ones and the counters ProbeSim draws (walk k, step s: (k, s, 0, 0);
randomized PROBE: (k, 2^24 | i << 8 | j, x, 0)).  The GPU path's walks equal the oracle's bit for bit, so this
also pins the library's own generator."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import core

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                           "-fPIC", os.path.join(HERE, "curand_philox.cu"), "-o", out, "-lcudart"])
    L = C.CDLL(out)
    L.curand_philox_blocks.restype = C.c_int
    L.curand_philox_blocks.argtypes = [C.c_void_p] * 4 + [C.c_int]
    return L


def _curand(L, ctr, key):
    ctr = np.asarray(ctr, np.uint64)
    key = np.asarray(key, np.uint64)
    seed = key[:, 0] | (key[:, 1] << np.uint64(32))
    sub = ctr[:, 2] | (ctr[:, 3] << np.uint64(32))
    off = (ctr[:, 0] | (ctr[:, 1] << np.uint64(32))) * np.uint64(4)
    seed, sub, off = (np.ascontiguousarray(a, np.uint64) for a in (seed, sub, off))
    out = np.zeros((ctr.shape[0], 4), np.uint32)
    rc = L.curand_philox_blocks(seed.ctypes.data, sub.ctypes.data, off.ctypes.data, out.ctypes.data, ctr.shape[0])
    assert rc == 0
    return out


def _oracle(ctr, key):
    return np.array([core.philox(c, k) for c, k in zip(ctr, key)], np.uint32)


def test_random_counters_and_keys(curand_lib):
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, (20000, 4), dtype=np.uint64)
    ctr[:, 0] &= np.uint64(0x3FFFFFFF)  # the offset argument holds 4 x (low 64 counter bits) in 64 bits
    ctr[:, 1] &= np.uint64(0x0FFFFFFF)
    key = rng.integers(0, 2 ** 32, (20000, 2), dtype=np.uint64)
    assert np.array_equal(_curand(curand_lib, ctr, key), _oracle(ctr, key))


def test_probesim_counters(curand_lib):
    rng = np.random.default_rng(2)
    rows, keys = [], []
    for k in range(0, 60000, 997):           # walk k, step s
        for s in range(0, 64, 7):
            rows.append((k, s, 0, 0))
            keys.append((3, int(rng.integers(0, 2 ** 32))))
    for k in range(0, 4000, 131):            # randomized PROBE: walk k, prefix i, level j, candidate x
        for i in (2, 5, 17):
            for j in range(0, i - 1, 3):
                rows.append((k, (1 << 24) | (i << 8) | j, int(rng.integers(0, 2 ** 31)), 0))
                keys.append((7, int(rng.integers(0, 2 ** 32))))
    ctr = np.array(rows, np.uint64)
    key = np.array(keys, np.uint64)
    assert np.array_equal(_curand(curand_lib, ctr, key), _oracle(ctr, key))
