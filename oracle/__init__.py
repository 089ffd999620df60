"""FP64 CPU oracle for the SP-LiDAR dead-time Markov chain (arXiv 2509.20500).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The GPU library never imports this
package and this package never imports the GPU library; they share only the
seeded input generators, which hold none of the method's arithmetic.

The arithmetic lives in ``spl_oracle.c`` (plain C, FP64, compiled with gcc on
first use) and in ``mlp.py`` (NumPy FP64 reference of the warm-start network).
This module is a thin ctypes layer plus the Monte Carlo ground truth.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(quadrature, Theorem 1/2 identities, LAPACK eigenvectors, closed-form special
cases, convergence order, event Monte Carlo).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libspl_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile spl_oracle.c into a shared library (gcc, -O2, no fast-math,
    no FMA contraction so FP64 expressions round as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_lambda.argtypes = [_dp, ctypes.c_double]
        lib.oracle_lambda.restype = ctypes.c_double
        lib.oracle_F.argtypes = [_dp, ctypes.c_double]
        lib.oracle_F.restype = ctypes.c_double
        lib.oracle_Lambda.argtypes = [_dp]
        lib.oracle_Lambda.restype = ctypes.c_double
        lib.oracle_q.argtypes = [_dp, ctypes.c_int32]
        lib.oracle_q.restype = ctypes.c_double
        lib.oracle_shift_l.argtypes = [_dp, ctypes.c_int32]
        lib.oracle_shift_l.restype = ctypes.c_int64
        lib.oracle_build_seq.argtypes = [_dp, ctypes.c_int32, _dp]
        lib.oracle_build_seq.restype = None
        lib.oracle_build_binint.argtypes = [_dp, ctypes.c_int32, ctypes.c_int64, _dp]
        lib.oracle_build_binint.restype = None
        lib.oracle_build_reparam.argtypes = [_dp, ctypes.c_int32, ctypes.c_int64, _dp]
        lib.oracle_build_reparam.restype = None
        lib.oracle_normalize_rows.argtypes = [ctypes.c_int32, _dp]
        lib.oracle_normalize_rows.restype = ctypes.c_int
        lib.oracle_power.argtypes = [ctypes.c_int32, _dp, ctypes.c_double, ctypes.c_int32,
                                     _dp, _dp, _dp]
        lib.oracle_power.restype = ctypes.c_int
        lib.oracle_stationary.argtypes = [_dp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_int32, _dp]
        lib.oracle_stationary.restype = ctypes.c_int
        lib.oracle_batch_stationary.argtypes = [_dp, _i32p, ctypes.c_int32, _i64p,
                                                ctypes.c_double, ctypes.c_int32,
                                                ctypes.c_int32, _dp, _i32p]
        lib.oracle_batch_stationary.restype = ctypes.c_int
        lib.oracle_mc_deadtime.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, _i64p]
        lib.oracle_mc_deadtime.restype = ctypes.c_int64
        _u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_philox4x64.argtypes = [_u64p, _u64p, _u64p]
        lib.oracle_philox4x64.restype = None
        lib.oracle_mc_philox.argtypes = [_dp, _i32p, ctypes.c_int32, _i64p, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)]
        lib.oracle_mc_philox.restype = ctypes.c_int
        lib.oracle_mc_philox_run.argtypes = [_dp, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)]
        lib.oracle_mc_philox_run.restype = None
        _lib = lib
        return lib


def _theta(p) -> np.ndarray:
    """theta vector {t_r, t_d, tau, sigma, S, B} from a mapping or record."""
    return np.ascontiguousarray(
        [float(p["t_r"]), float(p["t_d"]), float(p["tau"]), float(p["sigma"]),
         float(p["S"]), float(p["B"])], dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def flux_lambda(p, t) -> np.ndarray:
    """Eq. 1 arrival flux lambda(t) on one period."""
    lib, th = _load(), _theta(p)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([lib.oracle_lambda(_ptr(th), float(x)) for x in t])


def flux_F(p, t) -> np.ndarray:
    """Theorem 1 cumulative flux F(t) = int_0^t lambda, t in [0, t_r]."""
    lib, th = _load(), _theta(p)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    return np.array([lib.oracle_F(_ptr(th), float(x)) for x in t])


def Lambda(p) -> float:
    """Flux of one period, F(t_r)."""
    th = _theta(p)
    return _load().oracle_Lambda(_ptr(th))


def shift_q(p) -> float:
    """q = fmod(t_d, t_r) * N / t_r in FP64 (x_d / Delta)."""
    th = _theta(p)
    return _load().oracle_q(_ptr(th), int(p["n_bins"]))


def shift_l(p) -> int:
    """Theorem 2 row shift l = ceil(x_d / Delta)."""
    th = _theta(p)
    return int(_load().oracle_shift_l(_ptr(th), int(p["n_bins"])))


def shift_exact(p) -> int:
    """Shift that makes quantise-then-shift equal shift-then-quantise:
    ceil(q + 1/2) - 1, reduced modulo N."""
    N = int(p["n_bins"])
    return int(np.ceil(shift_q(p) + 0.5) - 1) % N


def build_seq(p) -> np.ndarray:
    """Unnormalised P from Rapp's sequential per-entry form (Eq. 3-4)."""
    N = int(p["n_bins"])
    th = _theta(p)
    P = np.empty((N, N), dtype=np.float64)
    _load().oracle_build_seq(_ptr(th), N, _ptr(P))
    return P


def build_reparam(p, shift: int) -> np.ndarray:
    """Unnormalised P from the reparameterised form (Eq. 6 + row roll)."""
    N = int(p["n_bins"])
    th = _theta(p)
    P = np.empty((N, N), dtype=np.float64)
    _load().oracle_build_reparam(_ptr(th), N, int(shift), _ptr(P))
    return P


def build_binint(p, shift: int) -> np.ndarray:
    """Unnormalised P of the bin-integrated variant (exact integral of the
    detection density over each bin instead of its midpoint value)."""
    N = int(p["n_bins"])
    th = _theta(p)
    P = np.empty((N, N), dtype=np.float64)
    _load().oracle_build_binint(_ptr(th), N, int(shift), _ptr(P))
    return P


def normalize_rows(P: np.ndarray) -> np.ndarray:
    """Row-normalised copy P~ (Sec. 2.3)."""
    Q = np.ascontiguousarray(P, dtype=np.float64).copy()
    if _load().oracle_normalize_rows(Q.shape[0], _ptr(Q)) != 0:
        raise ValueError("row with zero mass")
    return Q


def power(Pt: np.ndarray, tol: float = 1e-12, max_iter: int = 100000, start=None):
    """Dense FP64 power iteration pi <- pi P~; returns (pi, iterations, last step)."""
    Pt = np.ascontiguousarray(Pt, dtype=np.float64)
    N = Pt.shape[0]
    out = np.empty(N, dtype=np.float64)
    last = ctypes.c_double(0.0)
    st = None
    if start is not None:
        st = np.ascontiguousarray(start, dtype=np.float64)
    it = _load().oracle_power(N, _ptr(Pt), float(tol), int(max_iter),
                              _ptr(st) if st is not None else None, _ptr(out),
                              ctypes.byref(last))
    return out, it, last.value


def stationary(p, tol: float = 1e-12, max_iter: int = 100000, shift=None, flux: str = "point") -> np.ndarray:
    """Stationary pmf of one pixel.  shift=None: sequential construction
    (shift-then-quantise).  shift=k: reparameterised build with row shift k.
    flux="binint" (needs a shift): the bin-integrated variant."""
    N = int(p["n_bins"])
    th = _theta(p)
    out = np.empty(N, dtype=np.float64)
    if flux == "binint":
        if shift is None:
            raise ValueError("the bin-integrated variant takes an explicit shift")
        mode, sh = 2, int(shift)
    else:
        mode, sh = (0, 0) if shift is None else (1, int(shift))
    it = _load().oracle_stationary(_ptr(th), N, mode, sh, float(tol), int(max_iter), _ptr(out))
    if it < 0:
        raise RuntimeError(f"oracle power iteration failed (status {it})")
    return out


def batch_stationary(pixels, tol: float = 1e-12, max_iter: int = 100000,
                     nthreads: int | None = None):
    """Sequential-construction stationary pmfs of many pixels over host threads.
    Returns (packed pmfs, offsets [n+1], iterations [n], threads used)."""
    n = len(pixels)
    thetas = np.ascontiguousarray(np.stack([_theta(p) for p in pixels]) if n else
                                  np.zeros((0, 6)), dtype=np.float64)
    Ns = np.ascontiguousarray([int(p["n_bins"]) for p in pixels], dtype=np.int32)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ns)
    out = np.empty(int(offsets[-1]), dtype=np.float64)
    iters = np.zeros(n, dtype=np.int32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    used = _load().oracle_batch_stationary(_ptr(thetas), _ptr(Ns, _i32p), n, _ptr(offsets, _i64p),
                                           float(tol), int(max_iter), int(nthreads),
                                           _ptr(out), _ptr(iters, _i32p))
    return out, offsets, iters, used


def mc_registrations(p, n_periods: int, rng: np.random.Generator) -> np.ndarray:
    """Event-level Monte Carlo of a free-running SPAD (Sec. 2.2): Poisson(S)
    Gaussian signal photons per period (kept inside [0, t_r)), Poisson(B)
    uniform background photons per period, non-paralysable dead time t_d.
    Returns relative timestamps X_k = T_k mod t_r of the registrations."""
    t_r, tau, sig = float(p["t_r"]), float(p["tau"]), float(p["sigma"])
    S, B, t_d = float(p["S"]), float(p["B"]), float(p["t_d"])
    ns = rng.poisson(S, n_periods)
    nb = rng.poisson(B, n_periods)
    sig_x = tau + sig * rng.standard_normal(int(ns.sum()))
    sig_per = np.repeat(np.arange(n_periods), ns)
    keep = (sig_x >= 0.0) & (sig_x < t_r)
    bg_x = rng.uniform(0.0, t_r, int(nb.sum()))
    bg_per = np.repeat(np.arange(n_periods), nb)
    T = np.concatenate([sig_per[keep] * t_r + sig_x[keep], bg_per * t_r + bg_x])
    T.sort(kind="stable")
    T = np.ascontiguousarray(T)
    idx = np.empty(T.size, dtype=np.int64)
    m = _load().oracle_mc_deadtime(_ptr(T), T.size, t_d, _ptr(idx, _i64p))
    return np.mod(T[idx[:m]], t_r)


def mc_histogram(p, n_periods: int, rng: np.random.Generator) -> np.ndarray:
    """Histogram of Monte Carlo registrations over the N bins [k Delta, (k+1) Delta)."""
    N = int(p["n_bins"])
    X = mc_registrations(p, n_periods, rng)
    k = np.minimum((X * N / float(p["t_r"])).astype(np.int64), N - 1)
    return np.bincount(k, minlength=N).astype(np.float64)


def philox4x64(counter, key) -> np.ndarray:
    """One Philox4x64-10 block (Salmon et al., SC 2011): four 64-bit words."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    _load().oracle_philox4x64(_ptr(c, u64p), _ptr(k, u64p), _ptr(out, u64p))
    return out


def mc_philox_histograms(pixels, runs: int, cycles: int, seed: int, nthreads: int | None = None):
    """Counter-based event Monte Carlo (the Monte Carlo reference of Sec. 5,
    exactly specified in spl_oracle.c): per-run registration histograms.
    Returns (hist uint32 packed [runs * N_k per pixel], offsets [n+1] of the
    bins, so run r of pixel k is hist[runs*off[k] + r*N_k : + N_k])."""
    n = len(pixels)
    thetas = np.ascontiguousarray(np.stack([_theta(p) for p in pixels]), dtype=np.float64)
    Ns = np.ascontiguousarray([int(p["n_bins"]) for p in pixels], dtype=np.int32)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ns)
    hist = np.zeros(int(offsets[-1]) * runs, dtype=np.uint32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    _load().oracle_mc_philox(_ptr(thetas), _ptr(Ns, _i32p), n, _ptr(offsets, _i64p), int(runs), int(cycles),
                             ctypes.c_uint64(int(seed)), int(nthreads), _ptr(hist, ctypes.POINTER(ctypes.c_uint32)))
    return hist, offsets


def mc_philox_run(p, k: int, r: int, cycles: int, seed: int) -> np.ndarray:
    """Histogram of run r of the pixel at position k of a launch (the key
    depends on both), from the same experiment as mc_philox_histograms."""
    th = _theta(p)
    N = int(p["n_bins"])
    h = np.zeros(N, dtype=np.uint32)
    _load().oracle_mc_philox_run(_ptr(th), N, ctypes.c_uint64(int(seed)), ctypes.c_uint64(int(k)),
                                 ctypes.c_uint64(int(r)), int(cycles), _ptr(h, ctypes.POINTER(ctypes.c_uint32)))
    return h
