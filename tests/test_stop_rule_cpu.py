"""The power iteration's stop rule, compiled for the host and replayed on
synthetic step sequences whose true error is known.

The iterate is modelled as pi_k = pi + e_k + eta_k: e_k the transient of
one or two modes (a real lambda_2, or a complex pair rho e^{+-i theta}, as
Sec. 4 finds for P~) and eta_k a rounding term of fixed L1 size (fresh
random vectors, or a two-state cycle, the FP32 fixed points the kernel
meets).  Requirements: whenever the rule stops, the true L1 error
||e_k + eta_k||_1 is below the parity tolerance 1e-6; a start already at
the noise floor stops within two 8-step blocks; a clean transient stops
within a few steps of the first one whose true error is below tol_err.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-6
TOL_ERR = 0.5 * TOL
M = 512


@pytest.fixture(scope="module")
def rule(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("stop") / "libstoprule.so")
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O2", "-std=c++17",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-o", out,
                    os.path.join(HERE, "stop_rule_host.cu")], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    f = lib.stop_rule_replay_warm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_float,
                  ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]
    lib.stop_rule_warm_floor.restype = ctypes.c_float
    warm_floor = lib.stop_rule_warm_floor()

    def replay(d, min_iter=1, tau=1.0, warm=False):
        d = np.ascontiguousarray(d, dtype=np.float64)
        err, rho, th, rel = ctypes.c_float(), ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
        k = f(d.ctypes.data, d.shape[0], d.shape[1], TOL_ERR, min_iter, float(tau),
              float(warm_floor if warm else 0.0), ctypes.byref(err), ctypes.byref(rho), ctypes.byref(th),
              ctypes.byref(rel))
        return k, dict(err=err.value, rho=rho.value, theta=th.value, reliable=rel.value)
    return replay


def _zero_sum_unit(rng, n=1):
    v = rng.standard_normal((n, M))
    v -= v.mean(axis=1, keepdims=True)
    return v / np.abs(v).sum(axis=1, keepdims=True)


def sequence(rng, K, amp, rho, theta=0.0, noise=0.0, cycle=False, amp2=0.0, mu=0.3):
    """Step vectors d_1..d_K and the true errors ||pi_k - pi||_1, k = 0..K."""
    v1, v2, v3 = _zero_sum_unit(rng, 3)
    k = np.arange(K + 1)[:, None]
    e = amp * rho ** k * (np.cos(k * theta) * v1 + np.sin(k * theta) * v2) + amp2 * mu ** k * v3
    if cycle:
        eta = noise * (-1.0) ** k * _zero_sum_unit(rng)
    else:
        eta = noise * _zero_sum_unit(rng, K + 1)
    it = e + eta
    return np.diff(it, axis=0), np.abs(it).sum(axis=1)


CLEAN = [(0.05, 0.0), (0.3, 0.0), (0.6, 0.0), (0.87, 0.0), (0.7, np.pi), (0.8, 0.4), (0.8, 1.2), (0.8, 2.5),
         (0.5, 2.0)]


@pytest.mark.parametrize("rho,theta", CLEAN)
@pytest.mark.parametrize("noise", [0.0, 1e-7])
@pytest.mark.parametrize("tau_margin", [None, 0.02])
def test_transient_from_far_start(rule, rho, theta, noise, tau_margin):
    """tau_margin None: no a priori bound (tau = 1); else an honest bound
    tau = |lambda_2| + margin, as the ergodicity coefficient gives."""
    rng = np.random.default_rng(int(rho * 100 + theta * 10 + noise * 1e9))
    d, true = sequence(rng, 200, 1.0, rho, theta, noise, amp2=0.5)
    k, st = rule(d, tau=1.0 if tau_margin is None else rho + tau_margin)
    assert k > 0, st
    assert true[k] < TOL, (k, true[k], st)
    # no more than a few steps past the first iterate within tol_err (more
    # with noise: a floor under an oscillating transient shows only after
    # the transient has decayed well below it)
    first = int(np.argmax(true < 0.5 * TOL_ERR))
    assert k <= first + (6 if noise == 0.0 else 12), (k, first, st)


@pytest.mark.parametrize("noise", [3e-8, 1e-7, 2e-7, 3.5e-7, 6e-7])
@pytest.mark.parametrize("cycle", [False, True])
def test_start_on_the_noise_floor_stops(rule, noise, cycle):
    """A warm start already within rounding noise of pi: no trustworthy
    estimate of lambda_2 is possible, and the rule must still end, within
    two 8-step blocks.  Ending as converged requires the true error below
    the tolerance; a floor whose steps exceed 1e-6 may end as not converged
    (the rule cannot certify it)."""
    rng = np.random.default_rng(int(noise * 1e9) + cycle)
    d, true = sequence(rng, 200, 0.0, 0.5, 0.0, noise, cycle=cycle)
    k, st = rule(d)
    assert k != 0 and abs(k) <= 16, (k, st)
    if k > 0:
        assert true[k] < TOL
    else:
        assert noise >= 5e-7


@pytest.mark.parametrize("noise", [3e-6, 2e-5])
def test_floor_above_tolerance_ends_as_not_converged(rule, noise):
    """An FP32 floor above the tolerance: further steps cannot help; below
    1e-5 steps it ends within two blocks as not converged, above it the
    rule keeps iterating (max_iter ends it)."""
    rng = np.random.default_rng(5)
    d, _ = sequence(rng, 64, 0.0, 0.5, 0.0, noise)
    k, st = rule(d)
    if noise < 5e-6:
        assert -16 <= k < 0, (k, st)
    else:
        assert k == 0, (k, st)


@pytest.mark.parametrize("rho,theta,amp,noise", [(0.87, 0.0, 3e-6, 1e-7), (0.87, 0.0, 6e-6, 5e-8),
                                                 (0.85, 0.5, 3e-6, 5e-8), (0.8, 0.0, 1e-5, 1e-7),
                                                 (0.87, 0.0, 2e-6, 0.0), (0.6, np.pi, 4e-6, 1e-7)])
def test_warm_start_on_a_slow_mode(rule, rho, theta, amp, noise):
    """A warm start whose whole error lies in a slow mode: its steps are
    already below the stall floors, so only the decay pattern tells it from
    noise; the rule must not stop while the error exceeds the tolerance,
    with or without an honest a priori bound on |lambda_2|."""
    for seed in range(5):
        for tau in (1.0, min(1.0, rho + 0.03)):
            rng = np.random.default_rng(seed)
            d, true = sequence(rng, 300, amp, rho, theta, noise)
            k, st = rule(d, tau=tau)
            assert k > 0, st
            assert true[k] < TOL, (seed, tau, k, true[k], st)


@pytest.mark.parametrize("rho_fast,tau", [(0.005, 0.17), (0.01, 0.45), (0.02, 0.8)])
@pytest.mark.parametrize("noise", [5e-8, 7e-8, 1.2e-7])
def test_a_priori_bound_ends_a_fast_start_on_the_floor(rule, rho_fast, tau, noise):
    """A good warm start on a fast-mixing chain: one step lands on the FP32
    floor, where no trustworthy fit is possible.  Without an a priori bound
    the rule must assume |lambda_2| = 0.9 and wait for a stall; with the
    ergodicity bound tau it stops as soon as the floor is reached, with the
    true error below the tolerance."""
    rng = np.random.default_rng(int(tau * 100 + noise * 1e9))
    d, true = sequence(rng, 60, 8e-4, rho_fast, 0.0, noise)
    k_blind, _ = rule(d)
    k, st = rule(d, tau=tau)
    assert 0 < k <= 4, (k, st)
    assert k <= k_blind
    assert true[k] < TOL


@pytest.mark.parametrize("amp_slow", [1e-7, 2e-7, 4e-7, 8e-7, 1.6e-6])
@pytest.mark.parametrize("seed", range(4))
def test_warm_start_with_a_hidden_slow_mode(rule, amp_slow, seed):
    """A warm start whose visible steps come from a fast mode (0.25) while a
    slow mode (0.55, well below the a priori bound tau = 0.9) holds a small
    error: the fits see only the fast mode.  With the warm-start floor every
    stop is within the tolerance; without it (a cold start's rule) the same
    sequences stop with a larger error."""
    rng = np.random.default_rng(seed)
    d, true = sequence(rng, 80, 2e-4, 0.25, 0.0, 5e-8, amp2=amp_slow, mu=0.55)
    k, st = rule(d, tau=0.9, warm=True)
    assert k > 0, st
    assert true[k] < TOL, (k, true[k], st)
    k_cold, _ = rule(d, tau=0.9)
    assert abs(k_cold) <= k and true[abs(k_cold)] >= true[k]


def test_warm_floor_on_a_real_chain(rule):
    """The mechanism on a real chain (Eq. 6, a background-dominated pixel like
    the array pixels where it showed): a start at pi plus a fast mode
    (|lambda| ~ 0.21) and a small part of the slow pair (|lambda_2| ~ 0.55,
    left eigenvectors from LAPACK).  A cold start's rule fits only the fast
    mode; with the warm-start floor the stop comes later and closer to pi."""
    import oracle
    from paper_2509_20500_gb300 import workloads as W
    p = W.as_dicts(W.pixel(200, 75.0, 38.0, 0.36, 0.03, 4.1))[0]
    P = oracle.normalize_rows(oracle.build_reparam(p, oracle.shift_l(p)))
    tau = 1.0 - P.min(axis=0).sum()
    pi_star = oracle.power(P, tol=1e-15)[0]
    ev, V = np.linalg.eig(P.T)
    o = np.argsort(-np.abs(ev))
    lam2 = abs(ev[o[1]])
    slow = np.real(V[:, o[1]])
    slow /= np.abs(slow).sum()
    j = o[2:][np.argmin(np.abs(np.abs(ev[o[2:]]) - 0.2))]
    fast = np.real(V[:, j])
    fast /= np.abs(fast).sum()
    for seed in range(4):
        rng = np.random.default_rng(seed)
        pi = pi_star + 3e-4 * fast + (1e-6 if seed % 2 else -1e-6) * slow
        ds, true = [], []
        for _ in range(60):
            y = pi @ P
            y = y * (1.0 + 5e-8 * rng.standard_normal(200))
            y /= y.sum()
            ds.append(y - pi)
            pi = y
            true.append(np.abs(pi - pi_star).sum())
        k_cold, st_cold = rule(np.array(ds), tau=tau)
        k_warm, st_warm = rule(np.array(ds), tau=tau, warm=True)
        assert st_cold["rho"] < 0.5 * lam2           # the fit misses the slow pair
        assert k_warm >= k_cold and true[k_warm - 1] < true[k_cold - 1]
        assert true[k_warm - 1] < 0.25 * TOL


def test_min_iter_is_respected(rule):
    rng = np.random.default_rng(0)
    d, _ = sequence(rng, 50, 0.0, 0.5, 0.0, 1e-8)
    k, _ = rule(d, min_iter=12)
    assert k >= 12


def test_exact_fixed_point_stops_at_once(rule):
    d = np.zeros((10, M))
    k, st = rule(d)
    assert k == 3 and st["err"] == 0.0


def test_lambda2_estimate_from_clean_transient(rule):
    rng = np.random.default_rng(3)
    for rho, theta in [(0.6, 0.0), (0.8, 1.2), (0.7, np.pi)]:
        d, _ = sequence(rng, 200, 1.0, rho, theta)
        k, st = rule(d)
        assert st["reliable"] == 1
        assert abs(st["rho"] - rho) < 2e-2 * rho, (rho, theta, st)
        assert abs(st["theta"] - theta) < 5e-2, (rho, theta, st)


def _column_min_bound(P):
    return 1.0 - P.min(axis=0).sum()


@pytest.mark.parametrize("seed", range(6))
def test_ergodicity_bound_on_real_chains(seed):
    """On P~ of Eq. 6 (oracle build, broad random pixels): |lambda_2| <=
    tau_1 (Dobrushin's coefficient, max over row pairs of half the L1
    distance) <= 1 - sum_j min_i P~_ij, the bound the batch kernel forms in
    closed form."""
    import oracle
    from paper_2509_20500_gb300 import workloads as W
    for p in W.as_dicts(W.random_small(4, seed=100 + seed, n_min=20, n_max=120)):
        P = oracle.normalize_rows(oracle.build_reparam(p, oracle.shift_l(p)))
        tau1 = max(0.5 * np.abs(P - P[i]).sum(axis=1).max() for i in range(P.shape[0]))
        lam = np.sort(np.abs(np.linalg.eigvals(P)))[::-1]
        assert lam[1] <= tau1 + 1e-12
        assert tau1 <= _column_min_bound(P) + 1e-12


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("noise", [0.0, 5e-8])
def test_rigorous_stop_on_real_chains(rule, seed, noise):
    """Power iteration on real chains, from the uniform vector and from warm
    starts at distances 1e-3 .. 1e-7, replayed through the rule with the
    column-minimum bound as tau: every stop has true L1 error below the
    tolerance, also with a rounding floor injected into every iterate."""
    import oracle
    from paper_2509_20500_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    for p in W.as_dicts(W.random_small(3, seed=200 + seed, n_min=30, n_max=160)):
        P = oracle.normalize_rows(oracle.build_reparam(p, oracle.shift_l(p)))
        N = P.shape[0]
        pi_star = oracle.power(P, tol=1e-15)[0]
        tau = _column_min_bound(P)
        for amp in (None, 1e-3, 1e-5, 1e-7):
            if amp is None:
                pi = np.full(N, 1.0 / N)
            else:
                x = rng.standard_normal(N)
                x -= x.mean()
                pi = np.maximum(pi_star + amp * x / np.abs(x).sum(), 0.0)
                pi /= pi.sum()
            ds, true = [], []
            for _ in range(400):
                y = pi @ P
                if noise:
                    y = y * (1.0 + noise * rng.standard_normal(N))
                y /= y.sum()
                ds.append(y - pi)
                pi = y
                true.append(np.abs(pi - pi_star).sum())
            k, st = rule(np.array(ds), tau=min(1.0, tau + 1e-6), warm=amp is not None)
            assert k != 0, (p, amp, st)
            if k > 0:
                assert true[k - 1] < TOL, (p, amp, k, true[k - 1], tau, st)
