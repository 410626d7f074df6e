"""The oracle's Philox4x32-10 against cuRAND's device Philox4_32_10.

cuRAND is NVIDIA's implementation of the same published generator (Salmon et
al., SC'11), written independently of this repository; it runs here as a
library through the small helper tests/curand_philox.cu (the mapping of a
counter and key onto curand_init/skipahead is stated there).  Agreement on
the published known-answer vectors and on counters of the method's own
layout (id, step, stream, step high word) pins the oracle's generator, and
through the bit-exact pairing and Bernoulli tests, the GPU path's.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from tests.test_oracle_philox import kat_vectors

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    build = os.path.join(HERE, "_build")
    os.makedirs(build, exist_ok=True)
    so = os.path.join(build, "libcurand_philox.so")
    src = os.path.join(HERE, "curand_philox.cu")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                               "-Xcompiler", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    L = ctypes.CDLL(so)
    L.curand_philox_blocks.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    L.curand_philox_blocks.restype = ctypes.c_int
    return L


def _curand(L, ctrs, keys):
    c = np.ascontiguousarray(ctrs, dtype=np.uint32)
    k = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.zeros_like(c)
    rc = L.curand_philox_blocks(c.ctypes.data, k.ctypes.data, out.ctypes.data, c.shape[0])
    assert rc == 0, f"CUDA error {rc}"
    return out


def test_curand_known_answer_vectors(curand_lib):
    rows = kat_vectors()
    got = _curand(curand_lib, [r[0] for r in rows], [r[1] for r in rows])
    for g, (_, _, want) in zip(got, rows):
        assert [int(x) for x in g] == want


def test_oracle_equals_curand_on_the_method_counters(curand_lib):
    rng = np.random.default_rng(7)
    n = 4000
    ids = rng.integers(0, 2**32, n, dtype=np.uint64)
    ids[:8] = [0, 1, 2, 3, 2**32 - 1, 2**31, 12345, 4]
    step = rng.integers(0, 2**33, n, dtype=np.uint64)
    stream = rng.integers(1, 8, n, dtype=np.uint64)
    seed = rng.integers(0, 2**64 - 1, n, dtype=np.uint64)
    ctr = np.stack([ids, step & 0xFFFFFFFF, stream, step >> 32], axis=1).astype(np.uint32)
    key = np.stack([seed & 0xFFFFFFFF, seed >> 32], axis=1).astype(np.uint32)
    got = _curand(curand_lib, ctr, key)
    want = np.array([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)], dtype=np.uint32)
    assert np.array_equal(got, want)
