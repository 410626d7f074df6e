"""The FP64 Newton-Raphson helpers of the collision update (device_math.cuh:
rcp_nr, rsqrt_nr, sqrt_nr: an FP32 hardware seed refined by one Newton step,
stated within 5e-14 relative) against CUDA's correctly rounded FP64 reciprocal and
square root, over [1e-30, 1e30] where the refinement applies and beyond it,
where the helpers fall back to the full-precision operators."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = 5e-14   # relative, inside [1e-30, 1e30]


@pytest.fixture(scope="module")
def nr_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    build = os.path.join(HERE, "_build")
    os.makedirs(build, exist_ok=True)
    so = os.path.join(build, "libnr_helpers.so")
    src = os.path.join(HERE, "nr_helpers.cu")
    dep = os.path.join(os.path.dirname(HERE), "paper_2206_02937_gb300", "csrc", "device_math.cuh")
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(src), os.path.getmtime(dep)):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                               "-Xcompiler", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    L = ctypes.CDLL(so)
    L.nr_helpers_eval.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    L.nr_helpers_eval.restype = ctypes.c_int
    return L


def _eval(L, d):
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros((d.size, 6))
    assert L.nr_helpers_eval(d.ctypes.data, d.size, out.ctypes.data) == 0
    return out


def test_refined_range(nr_lib):
    rng = np.random.default_rng(3)
    d = 10.0 ** rng.uniform(-29.9, 29.9, 200000)
    d = np.concatenate([d, [1.0, 2.0, 0.5, 3.0, 1e-29, 9.9e29], rng.uniform(0.5, 4.0, 50000)])
    o = _eval(nr_lib, d)
    rel = lambda a, b: np.abs(a - b) / np.abs(b)  # noqa: E731
    assert rel(o[:, 0], o[:, 1]).max() <= BOUND
    assert rel(o[:, 2], o[:, 3]).max() <= BOUND
    assert rel(o[:, 4], o[:, 5]).max() <= BOUND
    # negative arguments of the reciprocal
    on = _eval(nr_lib, -d[:1000])
    assert rel(on[:, 0], on[:, 1]).max() <= BOUND


def test_outside_refined_range_falls_back_exactly(nr_lib):
    d = np.array([1e-31, 1e-100, 1e31, 1e200, 4.9e-324, 1.7e308])
    o = _eval(nr_lib, d)
    assert np.array_equal(o[:, 0], o[:, 1])
    assert np.array_equal(o[:, 4], o[:, 5])
    # 1/sqrt(d) against the correctly rounded reciprocal of the rounded root:
    # within one rounding of each
    assert np.all(np.abs(o[:, 2] - o[:, 3]) <= 3e-16 * np.abs(o[:, 3]))
