"""The batch solver's allocation-free entry point.

spl_batch_stationary_noalloc serves callers that may not allocate device
memory (allocation-free real-time pipelines, plug-ins whose host application
owns the GPU memory budget).  Its scratch is a fixed device array inside the
library, shared by every call.  Here it is called three times in a row through the
C ABI (with and without reports, two different batches) and each result is
checked against the allocating entry point, spl_batch_stationary, with the
parity tolerance of the other GPU tests (1e-6 in L1 per pixel); the driver's
free device memory must not change across a call.  This file is collected last so that a run stopping
at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2509_20500_gb300 import workloads as W

torch = pytest.importorskip("torch")

L1_TOL = 1e-6


def _call(L, spl, arr, n, out, offsets, reps):
    return L.spl_batch_stationary_noalloc(arr, n, 1e-6, 1000, None, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(offsets.data_ptr()), reps,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_20500_gb300 import build, spl
    build.build()
    L = spl.lib()
    # ragged sizes up to the entry point's limit, and two different batches
    batches = [np.concatenate([W.array_pixels(300, seed=41, n_bins=2000),
                               W.random_small(40, seed=42, n_min=2, n_max=3072)]),
               W.array_pixels(500, seed=43, n_bins=1500)]
    cases = []
    for px in batches:
        ref, off, ref_reps = spl.batch_stationary(px, tol=1e-6, max_iter=1000)
        cases.append({"n": len(px), "off": off, "ref": ref.cpu().numpy().astype(np.float64),
                      "iters": ref_reps["iters"], "arr": spl.pixels_to_c(px),
                      "offsets": torch.from_numpy(off).cuda(),
                      "out": torch.full((int(off[-1]),), -1.0, dtype=torch.float32, device="cuda")})
    torch.cuda.synchronize()

    def check(c):
        o = c["out"].cpu().numpy().astype(np.float64)
        off, r = c["off"], c["ref"]
        for k in range(c["n"]):
            assert np.abs(o[off[k]:off[k + 1]] - r[off[k]:off[k + 1]]).sum() < L1_TOL, k
        return o

    # call 1, with reports: the call waits for its result (the first call on a
    # device may also reserve the library's scratch array)
    c = cases[0]
    reps = (spl.spl_report_t * c["n"])()
    assert _call(L, spl, c["arr"], c["n"], c["out"], c["offsets"], reps) == spl.SPL_OK
    first = check(c)
    np.testing.assert_array_equal(np.array([reps[k].iters for k in range(c["n"])]), c["iters"])

    # call 2, another batch without reports: asynchronous; the driver's free
    # device memory is the same before the call and after its work finished
    c = cases[1]
    free0 = torch.cuda.mem_get_info()[0]
    assert _call(L, spl, c["arr"], c["n"], c["out"], c["offsets"], None) == spl.SPL_OK
    torch.cuda.current_stream().synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    check(c)

    # call 3, the first batch again over the array that call 2 left behind:
    # the same pmfs bit for bit
    c = cases[0]
    c["out"].fill_(-1.0)
    reps = (spl.spl_report_t * c["n"])()
    assert _call(L, spl, c["arr"], c["n"], c["out"], c["offsets"], reps) == spl.SPL_OK
    np.testing.assert_array_equal(check(c), first)


def test_noalloc_rejects_sizes_beyond_its_limit():
    """Host-side checks run before any device work (no GPU needed)."""
    from paper_2509_20500_gb300 import build, spl
    build.build()
    L = spl.lib()
    big = W.pixel(3073, 75.0, 30.0, 0.5, 0.5, 0.5)
    assert L.spl_batch_stationary_noalloc(spl.pixels_to_c(big), 1, 1e-6, 100, None, ctypes.c_void_p(8),
                                          ctypes.c_void_p(8), None, None) == spl.SPL_EINVAL
    many = W.array_pixels(65537, seed=1, n_bins=100)
    assert L.spl_batch_stationary_noalloc(spl.pixels_to_c(many), len(many), 1e-6, 100, None,
                                          ctypes.c_void_p(8), ctypes.c_void_p(8), None, None) == spl.SPL_EINVAL
