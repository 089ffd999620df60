"""Seeded synthetic pixel workloads.

This module only draws pixel parameters; it holds none of the method's
arithmetic.  Both the GPU library's tests/benchmark and the CPU oracle take
their inputs from here.

A pixel is theta = (t_r, t_d, tau, sigma, S, B) with n_bins states (Eq. 1 and
Sec. 2.2 of the paper).  Times are in ns.  ``shift_override`` = -1 asks the
library for the paper's row shift l = ceil(x_d / Delta); a value >= 0 forces a
shift (used to compare against the exact shift-then-quantise construction).

Workloads (shapes follow the paper's synthetic flux settings: Gaussian pulse
plus uniform background over one 100 ns laser period):
  single     : one pixel, N=1000, t_d=75, tau=30, sigma=0.5, S=B=0.5
  highres    : 12 pixels, N=10000, t_d in {10,40,75,130}, tau=30, sigma=0.3,
               S in {0.05,0.5,5}, B=0.5
  array128   : 128x128 pixels, N=2000, tau~U[5,95], sigma~U[0.2,1],
               S,B ~ logU[0.01,5], t_d=75                       (seed 3)
  uneven     : 4096 pixels, N~U{500,...,16000}, t_d~U[20,150], tau=30,
               sigma=0.3, B=0.5, S~U{0.05,0.5,5}                  (seed 4)
  array256   : 256x256 pixels, theta as array128                 (seed 5)
  training   : 200k pixels, theta as array128                    (seed 2)
"""
from __future__ import annotations

import numpy as np

PIXEL_DTYPE = np.dtype([
    ("t_r", np.float64), ("t_d", np.float64), ("tau", np.float64),
    ("sigma", np.float64), ("S", np.float64), ("B", np.float64),
    ("n_bins", np.int32), ("shift_override", np.int32),
])

T_R = 100.0


def _empty(n: int) -> np.ndarray:
    a = np.zeros(n, dtype=PIXEL_DTYPE)
    a["t_r"] = T_R
    a["shift_override"] = -1
    return a


def pixel(n_bins: int, t_d: float, tau: float, sigma: float, S: float, B: float,
          t_r: float = T_R, shift_override: int = -1) -> np.ndarray:
    a = _empty(1)
    a["t_r"], a["t_d"], a["tau"], a["sigma"] = t_r, t_d, tau, sigma
    a["S"], a["B"], a["n_bins"], a["shift_override"] = S, B, n_bins, shift_override
    return a


def single() -> np.ndarray:
    return pixel(1000, 75.0, 30.0, 0.5, 0.5, 0.5)


def highres() -> np.ndarray:
    rows = [pixel(10000, t_d, 30.0, 0.3, S, 0.5)
            for t_d in (10.0, 40.0, 75.0, 130.0) for S in (0.05, 0.5, 5.0)]
    return np.concatenate(rows)


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def array_pixels(n: int, seed: int, n_bins: int = 2000, t_d: float = 75.0) -> np.ndarray:
    """Pixels with theta drawn as in the 128x128 array workload."""
    rng = np.random.default_rng(seed)
    a = _empty(n)
    a["tau"] = rng.uniform(5.0, 95.0, n)
    a["sigma"] = rng.uniform(0.2, 1.0, n)
    a["S"] = _log_uniform(rng, 0.01, 5.0, n)
    a["B"] = _log_uniform(rng, 0.01, 5.0, n)
    a["t_d"] = t_d
    a["n_bins"] = n_bins
    return a


def array128(seed: int = 3) -> np.ndarray:
    return array_pixels(128 * 128, seed)


def array256(seed: int = 5) -> np.ndarray:
    return array_pixels(256 * 256, seed)


def training(n: int = 200_000, seed: int = 2) -> np.ndarray:
    return array_pixels(n, seed)


UNEVEN_N = (500, 1000, 2000, 4000, 8000, 16000)


def uneven(n: int = 4096, seed: int = 4) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = _empty(n)
    a["n_bins"] = rng.choice(np.array(UNEVEN_N, dtype=np.int32), n)
    a["t_d"] = rng.uniform(20.0, 150.0, n)
    a["tau"] = 30.0
    a["sigma"] = 0.3
    a["B"] = 0.5
    a["S"] = rng.choice(np.array([0.05, 0.5, 5.0]), n)
    return a


def accuracy_grid(n_bins: int = 256, steps: int = 21, t_d: float = 75.0, tau: float = 30.0,
                  sigma: float = 0.5) -> np.ndarray:
    """S, B on an even steps x steps grid over [0, 10] (the (0, 0) point
    dropped: no photons), the other parameters fixed; row-major in S."""
    g = np.linspace(0.0, 10.0, steps)
    SB = [(S, B) for S in g for B in g if S + B > 0.0]
    a = _empty(len(SB))
    a["t_r"], a["t_d"], a["tau"], a["sigma"] = T_R, t_d, tau, sigma
    a["S"] = [x[0] for x in SB]
    a["B"] = [x[1] for x in SB]
    a["n_bins"], a["shift_override"] = n_bins, -1
    return a


def random_small(n: int, seed: int, n_min: int = 2, n_max: int = 64) -> np.ndarray:
    """Small pixels with broad parameters (incl. t_d > t_r and t_d = 0) for
    exhaustive construction checks."""
    rng = np.random.default_rng(seed)
    a = _empty(n)
    a["n_bins"] = rng.integers(n_min, n_max + 1, n)
    a["t_d"] = rng.uniform(0.0, 250.0, n)
    a["t_d"][::7] = 0.0
    a["tau"] = rng.uniform(5.0, 95.0, n)
    a["sigma"] = rng.uniform(0.5, 8.0, n)
    a["S"] = _log_uniform(rng, 0.01, 8.0, n)
    a["B"] = _log_uniform(rng, 0.01, 8.0, n)
    return a


def sample_indices(n_total: int, k: int, seed: int) -> np.ndarray:
    """k distinct pixel indices drawn by seed (sorted)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_total, size=min(k, n_total), replace=False))


def as_dicts(a: np.ndarray):
    return [{name: a[name][k].item() for name in PIXEL_DTYPE.names} for k in range(len(a))]
