"""Thin ctypes binding of libspl (include/spl.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (passed by data pointer with
the current torch stream); host buffers are NumPy arrays.  The library must
have been built (``paper_2509_20500_gb300.build.build()``); a missing library
raises ImportError rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspl.so")

SPL_OK, SPL_EINVAL, SPL_ENOMEM, SPL_ECUDA, SPL_ENOCONV, SPL_ETIMEOUT = range(6)
SPL_MATERIALIZED, SPL_FUSED = 0, 1


class spl_pixel_t(ctypes.Structure):
    _fields_ = [("t_r", ctypes.c_double), ("t_d", ctypes.c_double), ("tau", ctypes.c_double),
                ("sigma", ctypes.c_double), ("S", ctypes.c_double), ("B", ctypes.c_double),
                ("n_bins", ctypes.c_int32), ("shift_override", ctypes.c_int32)]


class spl_report_t(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("last_step_l1", ctypes.c_float),
                ("err_bound", ctypes.c_float), ("lambda2_abs", ctypes.c_float),
                ("lambda2_phase", ctypes.c_float)]


class spl_batch_opts_t(ctypes.Structure):
    _fields_ = [("warm_kind", ctypes.c_int32), ("warm_ld", ctypes.c_int32), ("min_iter", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("time_kernel", ctypes.c_int32), ("pass_kind", ctypes.c_int32),
                ("flux_kind", ctypes.c_int32), ("tune", ctypes.c_int32), ("state_level", ctypes.c_int32),
                ("cols", ctypes.c_int32)]


SPL_WARM_WEIGHTS, SPL_WARM_LOGITS, SPL_WARM_LEARNED = 0, 1, 2
SPL_PASS_DENSE, SPL_PASS_STRUCTURED, SPL_PASS_DENSE_ROWSCAN = 0, 1, 2
SPL_FLUX_POINT, SPL_FLUX_BININT = 0, 1


REPORT_DTYPE = np.dtype([("iters", np.int32), ("status", np.int32), ("last_step_l1", np.float32),
                         ("err_bound", np.float32), ("lambda2_abs", np.float32),
                         ("lambda2_phase", np.float32)])

# Symbols include/spl.h declares (checked by the CPU tests).
EXPORTED = ["spl_build", "spl_stationary", "spl_batch_stationary", "spl_batch_stationary_ex", "spl_batch_kernel_ms",
            "spl_batch_stationary_host", "spl_batch_stationary_noalloc", "spl_matrix", "spl_chain_flux", "spl_free", "spl_strerror",
            "spl_last_cuda_error", "spl_version", "spl_mlp_create", "spl_mlp_param_count", "spl_mlp_set_params",
            "spl_mlp_get_params", "spl_mlp_get_state", "spl_mlp_set_state", "spl_mlp_forward", "spl_mlp_loss_grad", "spl_mlp_train_step", "spl_mlp_logits",
            "spl_mlp_free", "spl_batch_stationary_learned",
            "spl_batch_stationary_learned_host", "spl_gemm_bf16", "spl_chain_time_pass", "spl_chain_time_step", "spl_selftest_bounded_waits", "spl_chain_run_plan",
            "spl_chain_time_build", "spl_batch_spectral", "spl_mc_histograms", "spl_mlp_time_forward", "spl_batch_tune_lookup",
            "spl_fp32_fma_peak", "spl_chains_stationary", "spl_chains_plan"]

_lib = None
_lock = threading.Lock()


class SplError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().spl_strerror(status).decode()
        if status == SPL_ECUDA:
            msg += f" ({lib().spl_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg}")


def lib():
    """Load libspl (raises ImportError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libspl is not built ({LIB_PATH} missing); run paper_2509_20500_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.spl_build.argtypes = [ctypes.POINTER(spl_pixel_t), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.spl_build.restype = ctypes.c_int
        L.spl_stationary.argtypes = [vp, f64, i32, vp, vp, ctypes.POINTER(spl_report_t)]
        L.spl_stationary.restype = ctypes.c_int
        L.spl_batch_stationary.argtypes = [ctypes.POINTER(spl_pixel_t), i32, f64, i32, vp, vp, vp,
                                           ctypes.POINTER(spl_report_t), vp]
        L.spl_batch_stationary.restype = ctypes.c_int
        L.spl_batch_stationary_ex.argtypes = [ctypes.POINTER(spl_pixel_t), i32, f64, i32, vp, vp, vp,
                                              ctypes.POINTER(spl_report_t), vp,
                                              ctypes.POINTER(spl_batch_opts_t)]
        L.spl_batch_stationary_ex.restype = ctypes.c_int
        L.spl_batch_stationary_host.argtypes = [ctypes.POINTER(spl_pixel_t), i32, f64, i32, vp, vp,
                                                ctypes.POINTER(spl_report_t), vp]
        L.spl_batch_stationary_host.restype = ctypes.c_int
        L.spl_batch_stationary_noalloc.argtypes = [ctypes.POINTER(spl_pixel_t), i32, f64, i32, vp, vp, vp,
                                                   ctypes.POINTER(spl_report_t), vp]
        L.spl_batch_stationary_noalloc.restype = ctypes.c_int
        L.spl_batch_kernel_ms.argtypes = [ctypes.POINTER(ctypes.c_float)]
        L.spl_batch_kernel_ms.restype = ctypes.c_int
        L.spl_matrix.argtypes = [vp, vp]
        L.spl_matrix.restype = ctypes.c_int
        L.spl_chain_flux.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        L.spl_chain_flux.restype = ctypes.c_int
        L.spl_free.argtypes = [vp]
        L.spl_free.restype = None
        L.spl_strerror.argtypes = [ctypes.c_int]
        L.spl_strerror.restype = ctypes.c_char_p
        L.spl_last_cuda_error.argtypes = []
        L.spl_last_cuda_error.restype = ctypes.c_char_p
        L.spl_version.argtypes = []
        L.spl_version.restype = ctypes.c_char_p
        P = ctypes.POINTER(spl_pixel_t)
        fp = ctypes.POINTER(ctypes.c_float)
        L.spl_mlp_create.argtypes = [i32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        L.spl_mlp_create.restype = ctypes.c_int
        L.spl_mlp_param_count.argtypes = []
        L.spl_mlp_param_count.restype = ctypes.c_int64
        L.spl_mlp_set_params.argtypes = [vp, vp, ctypes.c_int64]
        L.spl_mlp_set_params.restype = ctypes.c_int
        L.spl_mlp_get_params.argtypes = [vp, vp, ctypes.c_int64]
        L.spl_mlp_get_params.restype = ctypes.c_int
        L.spl_mlp_get_state.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
        L.spl_mlp_get_state.restype = ctypes.c_int
        L.spl_mlp_set_state.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32]
        L.spl_mlp_set_state.restype = ctypes.c_int
        L.spl_mlp_forward.argtypes = [vp, P, i32, vp]
        L.spl_mlp_forward.restype = ctypes.c_int
        L.spl_mlp_time_forward.argtypes = [vp, P, i32, i32, fp]
        L.spl_mlp_time_forward.restype = ctypes.c_int
        L.spl_batch_tune_lookup.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]
        L.spl_batch_tune_lookup.restype = ctypes.c_int
        L.spl_mlp_loss_grad.argtypes = [vp, P, i32, vp, fp, vp]
        L.spl_mlp_loss_grad.restype = ctypes.c_int
        L.spl_mlp_train_step.argtypes = [vp, P, i32, vp, ctypes.c_float, ctypes.c_float, fp]
        L.spl_mlp_train_step.restype = ctypes.c_int
        L.spl_mlp_logits.argtypes = [vp]
        L.spl_mlp_logits.restype = ctypes.c_void_p
        L.spl_mlp_free.argtypes = [vp]
        L.spl_mlp_free.restype = None
        L.spl_batch_stationary_learned.argtypes = [vp, P, i32, f64, i32, vp, vp, ctypes.POINTER(spl_report_t), vp,
                                                   ctypes.POINTER(spl_batch_opts_t)]
        L.spl_batch_stationary_learned.restype = ctypes.c_int
        L.spl_batch_stationary_learned_host.argtypes = [vp, P, i32, f64, i32, vp, ctypes.POINTER(spl_report_t), vp,
                                                        ctypes.POINTER(spl_batch_opts_t)]
        L.spl_batch_stationary_learned_host.restype = ctypes.c_int
        L.spl_batch_spectral.argtypes = [ctypes.POINTER(spl_pixel_t), i32, i32, vp, vp]
        L.spl_batch_spectral.restype = ctypes.c_int
        L.spl_mc_histograms.argtypes = [ctypes.POINTER(spl_pixel_t), i32, i32, ctypes.c_int64, ctypes.c_uint64, vp,
                                        vp]
        L.spl_mc_histograms.restype = ctypes.c_int
        L.spl_chain_time_build.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
        L.spl_chain_time_build.restype = ctypes.c_int
        L.spl_chain_time_pass.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
        L.spl_chain_time_pass.restype = ctypes.c_int
        L.spl_chain_time_step.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_float)]
        L.spl_chain_time_step.restype = ctypes.c_int
        L.spl_selftest_bounded_waits.argtypes = [vp]
        L.spl_selftest_bounded_waits.restype = ctypes.c_int
        L.spl_chain_run_plan.argtypes = [i32, i32, i32, ctypes.POINTER(spl_run_plan_t)]
        L.spl_chain_run_plan.restype = ctypes.c_int
        L.spl_gemm_bf16.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        L.spl_gemm_bf16.restype = ctypes.c_int
        L.spl_chains_stationary.argtypes = [vp, i32, f64, i32, vp, ctypes.POINTER(spl_report_t)]
        L.spl_chains_stationary.restype = ctypes.c_int
        L.spl_chains_plan.argtypes = [vp, i32, i32, i32, vp]
        L.spl_chains_plan.restype = ctypes.c_int
        L.spl_fp32_fma_peak.argtypes = [i32, i32, vp, ctypes.POINTER(f64), ctypes.POINTER(f64), ctypes.POINTER(i32)]
        L.spl_fp32_fma_peak.restype = ctypes.c_int
        _lib = L
        return L


def _check(st: int, where: str, allow=(SPL_OK,)):
    if st not in allow:
        raise SplError(st, where)
    return st


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def pixels_to_c(px: np.ndarray, pinned: bool = False):
    """Marshal a workloads.PIXEL_DTYPE array into a ctypes spl_pixel_t array.
    pinned=True places it in page-locked host memory (through PyTorch), so the
    library's host-to-device copies of it are asynchronous; the array keeps
    its buffer alive."""
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    n = max(1, len(px))
    if pinned:
        import torch
        buf = torch.empty(n * ctypes.sizeof(spl_pixel_t), dtype=torch.uint8, pin_memory=True)
        arr = (spl_pixel_t * n).from_address(buf.data_ptr())
        arr._pinned_buffer = buf
    else:
        arr = (spl_pixel_t * n)()
    ctypes.memmove(arr, px.ctypes.data, px.nbytes)
    return arr


def offsets_of(px: np.ndarray) -> np.ndarray:
    off = np.zeros(len(px) + 1, dtype=np.int64)
    off[1:] = np.cumsum(px["n_bins"].astype(np.int64))
    return off


def _reports_np(reps, n):
    out = np.zeros(n, dtype=REPORT_DTYPE)
    if n:
        ctypes.memmove(out.ctypes.data, reps, out.nbytes)
    return out


class Chain:
    """One built pixel chain (spl_build ... spl_free)."""

    def __init__(self, pixel: np.ndarray, mode: int = SPL_FUSED, stream=None):
        self._c = ctypes.c_void_p()
        self.n_bins = int(np.asarray(pixel)["n_bins"].reshape(-1)[0])
        arr = pixels_to_c(np.asarray(pixel).reshape(-1)[:1])
        self.mode = mode
        self._stream = _stream_ptr(stream)
        _check(lib().spl_build(arr, mode, self._stream, ctypes.byref(self._c)), "spl_build")

    def stationary(self, tol: float = 1e-6, max_iter: int = 1000, warm=None, out=None, allow_noconv=False):
        import torch
        if out is None:
            out = torch.empty(self.n_bins, dtype=torch.float32, device="cuda")
        rep = spl_report_t()
        allow = (SPL_OK, SPL_ENOCONV) if allow_noconv else (SPL_OK,)
        st = lib().spl_stationary(self._c, float(tol), int(max_iter), _dptr(warm), _dptr(out), ctypes.byref(rep))
        _check(st, "spl_stationary", allow)
        return out, _reports_np(ctypes.addressof(rep), 1)[0]

    def time_pass(self, reps: int = 20) -> float:
        """Device ms of one dense power-step pass (spl_chain_time_pass)."""
        ms = ctypes.c_float()
        _check(lib().spl_chain_time_pass(self._c, int(reps), ctypes.byref(ms)), "spl_chain_time_pass")
        return float(ms.value)

    def time_step(self, reps: int = 20) -> float:
        """Device ms of one whole power step (spl_chain_time_step)."""
        ms = ctypes.c_float()
        _check(lib().spl_chain_time_step(self._c, int(reps), ctypes.byref(ms)), "spl_chain_time_step")
        return float(ms.value)

    def time_build(self, reps: int = 10) -> float:
        """Device ms of one materialised build (spl_chain_time_build)."""
        ms = ctypes.c_float()
        _check(lib().spl_chain_time_build(self._c, int(reps), ctypes.byref(ms)), "spl_chain_time_build")
        return float(ms.value)

    def matrix(self):
        import torch
        P = torch.empty((self.n_bins, self.n_bins), dtype=torch.float32, device="cuda")
        _check(lib().spl_matrix(self._c, _dptr(P)), "spl_matrix")
        return P

    def flux(self):
        import torch
        lam = torch.empty(self.n_bins, dtype=torch.float32, device="cuda")
        F = torch.empty(self.n_bins, dtype=torch.float64, device="cuda")
        Lam = ctypes.c_double()
        sh = ctypes.c_int32()
        _check(lib().spl_chain_flux(self._c, _dptr(lam), _dptr(F), ctypes.byref(Lam), ctypes.byref(sh)),
               "spl_chain_flux")
        return lam, F, Lam.value, sh.value

    def close(self):
        if self._c:
            lib().spl_free(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ChainSet:
    """Fused chains of several pixels, solved together by
    spl_chains_stationary (one cooperative launch, one CTA group per chain)."""

    def __init__(self, px: np.ndarray, stream=None):
        px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
        self.chains = [Chain(px[k:k + 1], SPL_FUSED, stream) for k in range(len(px))]
        self.off = offsets_of(px)
        self._arr = (ctypes.c_void_p * max(1, len(self.chains)))(*[c._c.value for c in self.chains])

    def stationary(self, tol: float = 1e-6, max_iter: int = 1000, out=None, reports: bool = True):
        import torch
        n = len(self.chains)
        if out is None:
            out = torch.empty(max(1, int(self.off[-1])), dtype=torch.float32, device="cuda")
        reps = (spl_report_t * max(1, n))() if reports else None
        st = lib().spl_chains_stationary(self._arr, n, float(tol), int(max_iter), _dptr(out), reps)
        _check(st, "spl_chains_stationary", (SPL_OK, SPL_ENOCONV))
        return out, self.off, (_reports_np(ctypes.addressof(reps), n) if reports else None)

    def close(self):
        for c in self.chains:
            c.close()
        self.chains = []


def chains_stationary(px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, stream=None):
    """Builds fused chains for the pixels and solves them in one launch;
    returns (packed pmfs, offsets, reports)."""
    cs = ChainSet(px, stream)
    try:
        return cs.stationary(tol=tol, max_iter=max_iter)
    finally:
        import torch
        torch.cuda.current_stream().synchronize()
        cs.close()


def batch_stationary(px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, warm=None, out=None,
                     warm_kind: int = SPL_WARM_WEIGHTS, warm_ld: int = 0, min_iter: int = 1, threads: int = 0,
                     reports: bool = True, offsets=None, stream=None, time_kernel: bool = False, c_pixels=None,
                     pass_kind: int = SPL_PASS_DENSE, flux_kind: int = SPL_FLUX_POINT, tune: int = 0,
                     state_level: int = -1, cols: int = 0):
    """spl_batch_stationary_ex over a PIXEL_DTYPE array; returns (out, offsets, reports)."""
    import torch
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    n = len(px)
    off = offsets_of(px)
    if offsets is None:
        offsets = torch.from_numpy(off).to("cuda")
    if out is None:
        out = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
    arr = pixels_to_c(px) if c_pixels is None else c_pixels
    reps = (spl_report_t * max(1, n))() if reports else None
    opts = spl_batch_opts_t(int(warm_kind), int(warm_ld), int(min_iter), int(threads), int(bool(time_kernel)),
                            int(pass_kind), int(flux_kind), int(tune), int(state_level), int(cols))
    st = lib().spl_batch_stationary_ex(arr, n, float(tol), int(max_iter), _dptr(warm), _dptr(out), _dptr(offsets),
                                       reps, _stream_ptr(stream), ctypes.byref(opts))
    _check(st, "spl_batch_stationary", (SPL_OK, SPL_ENOCONV))
    return out, off, (_reports_np(ctypes.addressof(reps), n) if reports else None)


def batch_stationary_noalloc(px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, warm=None, out=None,
                             offsets=None, reports: bool = True, stream=None, c_pixels=None):
    """spl_batch_stationary_noalloc: the batch solver for callers that may not
    allocate device memory (its scratch is a fixed device array inside the
    library).  ``out`` and ``offsets`` are caller-owned device tensors; they
    are created here only when not given.  Returns (out, offsets, reports)."""
    import torch
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    n = len(px)
    off = offsets_of(px)
    if offsets is None:
        offsets = torch.from_numpy(off).to("cuda")
    if out is None:
        out = torch.empty(max(1, int(off[-1])), dtype=torch.float32, device="cuda")
    arr = pixels_to_c(px) if c_pixels is None else c_pixels
    reps = (spl_report_t * max(1, n))() if reports else None
    st = lib().spl_batch_stationary_noalloc(arr, n, float(tol), int(max_iter), _dptr(warm), _dptr(out),
                                            _dptr(offsets), reps, _stream_ptr(stream))
    _check(st, "spl_batch_stationary_noalloc", (SPL_OK, SPL_ENOCONV))
    return out, off, (_reports_np(ctypes.addressof(reps), n) if reports else None)


def batch_tune_lookup(n_bins_max: int, pass_kind: int = SPL_PASS_DENSE):
    """The cached measured launch configuration (threads, state level, blocks
    per SM, columns per thread) for batches of this size and pass kind on the
    current device, or None."""
    t, lv, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    st = lib().spl_batch_tune_lookup(int(n_bins_max), int(pass_kind), ctypes.byref(t), ctypes.byref(lv),
                                     ctypes.byref(b), ctypes.byref(c))
    if st == SPL_ENOCONV:
        return None
    _check(st, "spl_batch_tune_lookup")
    return int(t.value), int(lv.value), int(b.value), int(c.value)


def mc_histograms(px: np.ndarray, runs: int, cycles: int, seed: int, out=None, stream=None):
    """spl_mc_histograms: per-run registration histograms of the event Monte
    Carlo, packed as run r of pixel k at runs*off[k] + r*N_k (int32 CUDA
    tensor holding the uint32 counts).  Returns (hist, off)."""
    import torch
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    off = offsets_of(px)
    total = int(off[-1]) * int(runs)
    if out is None:
        out = torch.empty(max(1, total), dtype=torch.int32, device="cuda")
    _check(lib().spl_mc_histograms(pixels_to_c(px), len(px), int(runs), int(cycles), ctypes.c_uint64(int(seed)),
                                   _dptr(out), _stream_ptr(stream)), "spl_mc_histograms")
    return out[:total], off


def batch_spectral(px: np.ndarray, subspace_iters: int = 60, stream=None):
    """spl_batch_spectral: (|lambda_2|, |arg lambda_2|) per pixel as a [n, 2] CUDA tensor."""
    import torch
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    out = torch.empty((max(1, len(px)), 2), dtype=torch.float32, device="cuda")
    _check(lib().spl_batch_spectral(pixels_to_c(px), len(px), int(subspace_iters), _dptr(out), _stream_ptr(stream)),
           "spl_batch_spectral")
    return out[:len(px)]


class spl_run_plan_t(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("tiles", ctypes.c_int32), ("row_blocks", ctypes.c_int32),
                ("segs", ctypes.c_int32), ("chunk", ctypes.c_int32), ("vlen", ctypes.c_int32)]


def chain_run_plan(n_bins: int, sms: int, blocks_per_sm: int) -> dict:
    """spl_chain_run_plan (host arithmetic, no GPU needed)."""
    pl = spl_run_plan_t()
    _check(lib().spl_chain_run_plan(int(n_bins), int(sms), int(blocks_per_sm), ctypes.byref(pl)),
           "spl_chain_run_plan")
    return {k: int(getattr(pl, k)) for k, _ in spl_run_plan_t._fields_}


def chains_plan(n_bins, sms: int, blocks_per_sm: int) -> np.ndarray:
    """spl_chains_plan (host arithmetic, no GPU needed): partial slots per
    column tile of each chain of a lockstep multi-chain launch."""
    nb = np.ascontiguousarray(n_bins, dtype=np.int32)
    out = np.zeros(len(nb), dtype=np.int32)
    _check(lib().spl_chains_plan(nb.ctypes.data_as(ctypes.c_void_p), len(nb), int(sms), int(blocks_per_sm),
                                 out.ctypes.data_as(ctypes.c_void_p)), "spl_chains_plan")
    return out


def selftest_bounded_waits(stream=None) -> int:
    """spl_selftest_bounded_waits: the status (SPL_OK when every wait gave up
    as designed)."""
    return int(lib().spl_selftest_bounded_waits(_stream_ptr(stream)))


def fp32_fma_peak(iters: int = 800_000, reps: int = 5, stream=None) -> dict:
    """spl_fp32_fma_peak: measured FP32 FMA throughput (TFLOP/s, median and
    fastest of `reps` launches) and the SM count."""
    med, best, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().spl_fp32_fma_peak(int(iters), int(reps), _stream_ptr(stream), ctypes.byref(med), ctypes.byref(best),
                                   ctypes.byref(sms)), "spl_fp32_fma_peak")
    return {"tflops_median": med.value, "tflops_best": best.value, "sms": int(sms.value)}


def batch_kernel_ms() -> float:
    """Device time of the batch kernel of the last call made with time_kernel=True."""
    ms = ctypes.c_float()
    _check(lib().spl_batch_kernel_ms(ctypes.byref(ms)), "spl_batch_kernel_ms")
    return float(ms.value)


def batch_stationary_host(px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, warm: np.ndarray | None = None,
                          out: np.ndarray | None = None, reports: bool = True, stream=None, c_pixels=None):
    """spl_batch_stationary_host: host buffers in and out (copies inside the call)."""
    px = np.ascontiguousarray(px, dtype=workloads.PIXEL_DTYPE)
    n = len(px)
    off = offsets_of(px)
    if out is None:
        out = np.empty(int(off[-1]), dtype=np.float32)
    arr = pixels_to_c(px) if c_pixels is None else c_pixels
    reps = (spl_report_t * max(1, n))() if reports else None
    wp = None if warm is None else ctypes.c_void_p(np.ascontiguousarray(warm, dtype=np.float32).ctypes.data)
    st = lib().spl_batch_stationary_host(arr, n, float(tol), int(max_iter), wp, ctypes.c_void_p(out.ctypes.data),
                                         reps, _stream_ptr(stream))
    _check(st, "spl_batch_stationary_host", (SPL_OK, SPL_ENOCONV))
    return out, off, (_reports_np(ctypes.addressof(reps), n) if reports else None)


def gemm_bf16(A, B):
    """D = A @ B^T with the library's tcgen05 kernel (A [M,K], B [N,K] bf16 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(lib().spl_gemm_bf16(_dptr(A), _dptr(B), M, N, K, _dptr(D), _stream_ptr()), "spl_gemm_bf16")
    return D


class MLP:
    """The learned warm-start network (spl_mlp_*)."""

    N_OUT = 2000
    LD = 2048

    def __init__(self, max_batch: int, seed: int = 0, stream=None):
        self._m = ctypes.c_void_p()
        self._stream = _stream_ptr(stream)
        self.max_batch = max_batch
        _check(lib().spl_mlp_create(int(max_batch), int(seed), self._stream, ctypes.byref(self._m)), "spl_mlp_create")

    @staticmethod
    def param_count() -> int:
        return int(lib().spl_mlp_param_count())

    def get_params(self) -> np.ndarray:
        out = np.empty(self.param_count(), dtype=np.float32)
        _check(lib().spl_mlp_get_params(self._m, ctypes.c_void_p(out.ctypes.data), out.size), "spl_mlp_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().spl_mlp_set_params(self._m, ctypes.c_void_p(p.ctypes.data), p.size), "spl_mlp_set_params")

    def get_state(self):
        """AdamW state (moments packed like the parameters) and step count."""
        out = np.empty(2 * self.param_count(), dtype=np.float32)
        step = ctypes.c_int32()
        _check(lib().spl_mlp_get_state(self._m, ctypes.c_void_p(out.ctypes.data), out.size, ctypes.byref(step)),
               "spl_mlp_get_state")
        return out, int(step.value)

    def set_state(self, state: np.ndarray, step: int):
        state = np.ascontiguousarray(state, dtype=np.float32)
        _check(lib().spl_mlp_set_state(self._m, ctypes.c_void_p(state.ctypes.data), state.size, int(step)),
               "spl_mlp_set_state")

    def time_forward(self, px: np.ndarray, reps: int = 10) -> float:
        """Device ms of one forward pass (kernels only) over px."""
        ms = ctypes.c_float()
        _check(lib().spl_mlp_time_forward(self._m, pixels_to_c(px), len(px), int(reps), ctypes.byref(ms)),
               "spl_mlp_time_forward")
        return float(ms.value)

    def forward(self, px: np.ndarray, out=None):
        import torch
        n = len(px)
        if out is None:
            out = torch.empty((n, self.LD), dtype=torch.float32, device="cuda")
        _check(lib().spl_mlp_forward(self._m, pixels_to_c(px), n, _dptr(out)), "spl_mlp_forward")
        return out

    def loss_grad(self, px: np.ndarray, target, grads: bool = True):
        loss = ctypes.c_float()
        g = np.empty(self.param_count(), dtype=np.float32) if grads else None
        _check(lib().spl_mlp_loss_grad(self._m, pixels_to_c(px), len(px), _dptr(target), ctypes.byref(loss),
                                       ctypes.c_void_p(g.ctypes.data) if grads else None), "spl_mlp_loss_grad")
        return float(loss.value), g

    def train_step(self, c_px, n: int, target, lr: float, weight_decay: float = 0.0, want_loss: bool = False):
        loss = ctypes.c_float()
        _check(lib().spl_mlp_train_step(self._m, c_px, int(n), _dptr(target), float(lr), float(weight_decay),
                                        ctypes.byref(loss) if want_loss else None), "spl_mlp_train_step")
        return float(loss.value) if want_loss else None

    def batch_stationary(self, px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, out=None, offsets=None,
                         reports: bool = True, c_pixels=None, pass_kind: int = SPL_PASS_DENSE,
                         flux_kind: int = SPL_FLUX_POINT, threads: int = 0, tune: int = 0, state_level: int = -1,
                         time_kernel: bool = True):
        import torch
        n = len(px)
        off = offsets_of(px)
        if offsets is None:
            offsets = torch.from_numpy(off).to("cuda")
        if out is None:
            out = torch.empty(int(off[-1]), dtype=torch.float32, device="cuda")
        reps = (spl_report_t * max(1, n))() if reports else None
        arr = pixels_to_c(px) if c_pixels is None else c_pixels
        opts = spl_batch_opts_t(0, 0, 1, int(threads), int(bool(time_kernel)), int(pass_kind), int(flux_kind),
                                int(tune), int(state_level), 0)
        st = lib().spl_batch_stationary_learned(self._m, arr, n, float(tol), int(max_iter), _dptr(out),
                                                _dptr(offsets), reps, self._stream, ctypes.byref(opts))
        _check(st, "spl_batch_stationary_learned", (SPL_OK, SPL_ENOCONV))
        return out, off, (_reports_np(ctypes.addressof(reps), n) if reports else None)

    def batch_stationary_host(self, px: np.ndarray, tol: float = 1e-6, max_iter: int = 1000, out=None,
                              reports: bool = True, c_pixels=None, pass_kind: int = SPL_PASS_DENSE,
                              flux_kind: int = SPL_FLUX_POINT, tune: int = 0):
        """spl_batch_stationary_learned_host: pmfs into a host tensor `out`
        (pinned if allocated here), packed in caller order."""
        import torch
        n = len(px)
        off = offsets_of(px)
        if out is None:
            out = torch.empty(int(off[-1]), dtype=torch.float32).pin_memory()
        reps = (spl_report_t * max(1, n))() if reports else None
        arr = pixels_to_c(px) if c_pixels is None else c_pixels
        opts = spl_batch_opts_t(0, 0, 1, 0, 0, int(pass_kind), int(flux_kind), int(tune), -1, 0)
        st = lib().spl_batch_stationary_learned_host(self._m, arr, n, float(tol), int(max_iter),
                                                     ctypes.c_void_p(out.data_ptr()), reps, self._stream,
                                                     ctypes.byref(opts))
        _check(st, "spl_batch_stationary_learned_host", (SPL_OK, SPL_ENOCONV))
        return out, off, (_reports_np(ctypes.addressof(reps), n) if reports else None)

    def close(self):
        if self._m:
            lib().spl_mlp_free(self._m)
            self._m = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
