"""The batch kernel's own FP64 helpers, compiled for the host from the
kernels' header and checked against NumPy: exp_series (range reduction by
ln 2 and the Taylor series of e^r to degree 10) over the arguments the flux
factors use, and pow_uint (repeated squaring) for the geometric tables."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("devmath") / "libdevmath.so")
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-std=c++17",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-o", out,
                    os.path.join(HERE, "device_math_host.cu")], check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.exp_series_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    L.pow_uint_host.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return L


def test_exp_series_relative_error(lib):
    """Relative error below 1e-12 over [-130, 130] (the pulse exponents are
    -z^2/2 >= -40.5 and Lambda/2 - S G with Lambda <= 120), including the
    points where the reduction switches n."""
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-130.0, 130.0, 200001), rng.uniform(-130, 130, 100000),
                        np.arange(-187, 188) * np.log(2.0) / 2.0, [0.0, -0.0, 1e-300, -1e-300]])
    y = np.empty_like(x)
    lib.exp_series_host(x.ctypes.data, y.ctypes.data, x.size)
    rel = np.abs(y / np.exp(x) - 1.0)
    assert rel.max() < 1e-12, (rel.max(), x[np.argmax(rel)])


def test_pow_uint_tables(lib):
    """t_lo and t_hi factors: q^e for q = exp(-beta), beta = B / N over the
    workloads' range, e up to 255.  Every squaring doubles the relative
    error carried so far, so the bound is about e u = 255 x 1.1e-16 = 2.8e-14
    (far below the FP32 rounding of the factors)."""
    rng = np.random.default_rng(1)
    beta = rng.uniform(0.0, 20.0, 4000) / rng.choice([500, 2000, 16000], 4000)
    e = rng.integers(0, 256, 4000).astype(np.int32)
    q = np.exp(-beta)
    y = np.empty_like(q)
    lib.pow_uint_host(q.ctypes.data, e.ctypes.data, y.ctypes.data, q.size)
    ref = np.power(q, e.astype(np.float64))
    assert np.max(np.abs(y / ref - 1.0)) < 4e-14
