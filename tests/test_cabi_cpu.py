"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every symbol include/spl.h declares, the struct layouts agree,
and host-side validation rejects bad input before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2509_20500_gb300 import build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    build.build()
    from paper_2509_20500_gb300 import spl
    spl.lib()
    return spl


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "spl.h")).read()
    return sorted(set(re.findall(r"SPL_API\s+[\w\s\*]*?\b(spl_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(S):
    decl = declared_symbols()
    assert len(decl) >= 20
    L = S.lib()
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(S.EXPORTED) == decl


def test_struct_layouts(S, tmp_path):
    """The binding's structures have the sizes the C header gives them (a
    small C program compiled against include/spl.h prints them)."""
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "spl.h"\nint main(void) { printf("%zu %zu %zu %zu\\n", '
                   'sizeof(spl_pixel_t), sizeof(spl_report_t), sizeof(spl_batch_opts_t), sizeof(spl_run_plan_t)); '
                   'return 0; }\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(S.spl_pixel_t), ctypes.sizeof(S.spl_report_t), ctypes.sizeof(S.spl_batch_opts_t),
                     ctypes.sizeof(S.spl_run_plan_t)]
    assert ctypes.sizeof(S.spl_pixel_t) == 56 == W.PIXEL_DTYPE.itemsize
    assert ctypes.sizeof(S.spl_report_t) == 24 == S.REPORT_DTYPE.itemsize
    assert ctypes.sizeof(S.spl_batch_opts_t) == 40


def test_strerror_and_version(S):
    L = S.lib()
    assert L.spl_strerror(0) == b"ok"
    assert b"converge" in L.spl_strerror(4)
    assert b"sm_103a" in L.spl_version()


BAD = [dict(sigma=0.0), dict(sigma=-1.0), dict(t_r=0.0), dict(t_d=-1.0), dict(S=-0.1), dict(B=-0.1),
       dict(S=0.0, B=0.0), dict(tau=100.0), dict(tau=-0.5), dict(n_bins=1), dict(t_d=float("nan")),
       dict(S=float("inf")), dict(S=100.0, B=30.0), dict(shift_override=-2)]


@pytest.mark.parametrize("bad", BAD)
def test_build_rejects_invalid_pixel_without_gpu(S, bad):
    kw = dict(n_bins=100, t_d=75.0, tau=30.0, sigma=0.5, S=0.5, B=0.5)
    kw.update(bad)
    px = W.pixel(**kw)
    out = ctypes.c_void_p()
    st = S.lib().spl_build(S.pixels_to_c(px), S.SPL_FUSED, None, ctypes.byref(out))
    assert st == S.SPL_EINVAL and not out.value


def test_null_arguments_rejected(S):
    L = S.lib()
    out = ctypes.c_void_p()
    assert L.spl_build(None, 0, None, ctypes.byref(out)) == S.SPL_EINVAL
    assert L.spl_build(S.pixels_to_c(W.single()), 7, None, ctypes.byref(out)) == S.SPL_EINVAL
    assert L.spl_stationary(None, 1e-6, 10, None, None, None) == S.SPL_EINVAL
    assert L.spl_matrix(None, None) == S.SPL_EINVAL
    assert L.spl_batch_stationary(None, 3, 1e-6, 10, None, None, None, None, None) == S.SPL_EINVAL
    assert L.spl_batch_stationary(S.pixels_to_c(W.single()), 1, -1.0, 10, None, None, None, None, None) \
        == S.SPL_EINVAL
    L.spl_free(None)


@pytest.mark.parametrize("bad", BAD[:-2] + [dict(S=16.5), dict(B=17.0), dict(n_bins=16385)])
def test_mc_rejects_invalid_input_without_gpu(S, bad):
    """spl_mc_histograms validates every pixel and its limits (at most 64
    photons per source and cycle, 16384 bins) before touching the GPU."""
    kw = dict(n_bins=100, t_d=75.0, tau=30.0, sigma=0.5, S=0.5, B=0.5)
    kw.update(bad)
    L = S.lib()
    fake = ctypes.c_void_p(256)   # never dereferenced: validation fails first
    assert L.spl_mc_histograms(S.pixels_to_c(W.pixel(**kw)), 1, 4, 100, 1, fake, None) == S.SPL_EINVAL


def test_mc_rejects_bad_counts_without_gpu(S):
    L = S.lib()
    px = S.pixels_to_c(W.single())
    fake = ctypes.c_void_p(256)
    assert L.spl_mc_histograms(px, 1, 0, 100, 1, fake, None) == S.SPL_EINVAL
    assert L.spl_mc_histograms(px, 1, 4, 0, 1, fake, None) == S.SPL_EINVAL
    assert L.spl_mc_histograms(px, 0, 4, 100, 1, fake, None) == S.SPL_EINVAL
    assert L.spl_mc_histograms(px, 1, 4, 100, 1, None, None) == S.SPL_EINVAL
    assert L.spl_mc_histograms(None, 1, 4, 100, 1, fake, None) == S.SPL_EINVAL


def test_oracle_and_library_share_nothing():
    """The oracle sources and the CUDA sources include none of each other's
    files, and neither Python side imports the other."""
    csrc = os.path.join(ROOT, "paper_2509_20500_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    otxt = open(os.path.join(ROOT, "oracle", "spl_oracle.c")).read()
    assert "spl.h" not in otxt and "spl_device" not in otxt
    for f in ("spl.py", "build.py", "workloads.py", "__init__.py"):
        txt = open(os.path.join(ROOT, "paper_2509_20500_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f
    ow = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2509_20500_gb300" not in ow
