"""The surrogate epilogue's SiLU forms (csrc/act_math.cuh) against the exact
SiLU in FP64 and against CUDA's expf-based SiLU, on a dense grid of z = 2 h:

  * silu2_fma (2^y by range reduction and a minimax polynomial, Newton
    reciprocal, FMA pipe only): relative error below 1e-4 for |z| < 80 (the
    polynomial's 7.5e-5 plus the reciprocal's 6.5e-6 and the clamp's 5e-6),
    i.e. within 1e-4 plus CUDA expf's own bound (2 ulp) of CUDA's SiLU; beyond
    |z| = 80 the value is z (z > 0, relative 1e-5) or 0 to within 1e-6
    absolute (z < 0); NaN propagates;
  * silu2_mufu (tanh.approx.f32): absolute error below |h| 2^-10 (the
    hardware tanh's absolute bound, scaled by h in y = h + h tanh h).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def act_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    build = os.path.join(HERE, "_build")
    os.makedirs(build, exist_ok=True)
    so = os.path.join(build, "libact_math.so")
    src = os.path.join(HERE, "act_math_eval.cu")
    dep = os.path.join(os.path.dirname(HERE), "paper_2206_02937_gb300", "csrc", "act_math.cuh")
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(dep)):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                               "-Xcompiler", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    L = ctypes.CDLL(so)
    L.act_math_eval.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.act_math_eval.restype = ctypes.c_int
    return L


def _eval(L, h):
    h = np.ascontiguousarray(h, dtype=np.float32)
    outs = [np.empty_like(h) for _ in range(3)]
    rc = L.act_math_eval(h.ctypes.data, h.size, *(o.ctypes.data for o in outs))
    assert rc == 0
    return outs


def _grid():
    z = np.concatenate([np.linspace(-100.0, 100.0, 1_000_001), np.geomspace(1e-30, 100.0, 100_001),
                        -np.geomspace(1e-30, 100.0, 100_001), [0.0]])
    return (z / 2).astype(np.float32)


def test_silu_fma_relative_error(act_lib):
    h = _grid()
    fma, _, via_expf = _eval(act_lib, h)
    z = 2.0 * h.astype(np.float64)
    exact = z / (1.0 + np.exp(-z))
    inner = np.abs(z) < 80
    rel = np.abs(fma[inner] - exact[inner]) / np.maximum(np.abs(exact[inner]), 1e-300)
    print("silu2_fma: max relative error", rel.max(), "median", np.median(rel))
    assert rel.max() <= 1e-4, rel.max()
    # against CUDA's own expf-based SiLU: within 1e-4 plus 2 ulp of expf and
    # the rounding of 1 + expf, z / (...)
    ref = via_expf[inner].astype(np.float64)
    tol = 1e-4 * np.abs(ref) + 4 * np.spacing(np.abs(via_expf[inner])).astype(np.float64)
    assert np.all(np.abs(fma[inner] - ref) <= tol + 1e-30)
    hi, lo = z >= 80, z <= -80
    assert np.all(np.abs(fma[hi] / z[hi] - 1) <= 1e-5)
    assert np.all(np.abs(fma[lo]) <= 1e-6)


def test_silu_fma_special_values(act_lib):
    h = np.array([0.0, -0.0, np.inf, np.nan, 1e30, -1e30, 1e-37, -1e-37], np.float32)
    fma, mufu, _ = _eval(act_lib, h)
    assert fma[0] == 0.0 and fma[1] == 0.0
    assert fma[2] == np.inf
    assert np.isnan(fma[3]) and np.isnan(mufu[3])
    assert abs(fma[4] / 2e30 - 1) <= 1e-5
    assert abs(fma[5]) <= 1e-6
    assert abs(fma[6] / 1e-37 - 1) <= 1e-4 and abs(fma[7] / -1e-37 - 1) <= 1e-4


def test_silu_mufu_error(act_lib):
    h = _grid()
    _, mufu, _ = _eval(act_lib, h)
    z = 2.0 * h.astype(np.float64)
    exact = z / (1.0 + np.exp(-z))
    err = np.abs(mufu - exact)
    bound = np.abs(h.astype(np.float64)) * 2.0 ** -10 + 1e-38
    print("silu2_mufu: max error / bound", (err / bound).max())
    assert np.all(err <= bound)
