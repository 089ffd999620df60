"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses quadrature,
LAPACK, an event-level Monte Carlo, an exact algebraic identity between two
independently written constructions, a closed-form special case, or a
convergence-order property.  Together they fail on a dropped term (the
Lambda indicator, the B/t_r background, the -Phi(-tau/sigma) offset), a wrong
sign, a wrong roll direction or shift, or a transposed power step.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2509_20500_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_settings.json")


def _px(**kw):
    base = dict(n_bins=1000, t_d=75.0, tau=30.0, sigma=0.5, S=0.5, B=0.5)
    base.update(kw)
    return W.as_dicts(W.pixel(**base))[0]


# ---------------------------------------------------------------- flux (Eq. 1, Thm 1)

@pytest.mark.parametrize("kw", [dict(), dict(tau=5.0, sigma=1.0, S=5.0, B=0.01),
                                dict(tau=94.0, sigma=0.2, S=0.01, B=5.0),
                                dict(tau=50.0, sigma=8.0, S=3.0, B=3.0)])
def test_F_is_integral_of_lambda(kw):
    """Theorem 1's F(t) = int_0^t lambda, checked by adaptive quadrature."""
    p = _px(**kw)
    lam = lambda t: oracle.flux_lambda(p, t)[0]
    for t in (0.0, 3.0, p["tau"] - p["sigma"], p["tau"], p["tau"] + 0.3, 77.7, 100.0):
        ref, err = integrate.quad(lam, 0.0, t, points=[p["tau"]] if 0 < p["tau"] < t else None,
                                  epsabs=1e-14, epsrel=1e-13, limit=400)
        assert abs(oracle.flux_F(p, t)[0] - ref) < 1e-11 + 1e-11 * abs(ref)


def test_lambda_shape():
    """Eq. 1: peak height S/(sigma sqrt(2 pi)) + B/t_r at tau, background far away."""
    p = _px(S=2.0, B=0.7, sigma=0.4)
    peak = oracle.flux_lambda(p, p["tau"])[0]
    assert peak == pytest.approx(2.0 / (0.4 * math.sqrt(2 * math.pi)) + 0.7 / 100.0, rel=1e-14)
    assert oracle.flux_lambda(p, 90.0)[0] == pytest.approx(0.7 / 100.0, rel=1e-14)


def test_Lambda_is_one_period_flux():
    """Lambda = F(t_r); equals S + B (Eq. 1) when the pulse is well inside the period,
    and loses the truncated tail otherwise."""
    p = _px(S=3.0, B=2.0)
    assert oracle.Lambda(p) == pytest.approx(5.0, abs=1e-13)
    p = _px(tau=1.0, sigma=1.0, S=3.0, B=2.0)        # pulse truncated at t = 0
    lost = 3.0 * special.ndtr(-1.0)
    assert oracle.Lambda(p) == pytest.approx(5.0 - lost, abs=1e-12)


# ---------------------------------------------------------------- dead-time shift (Thm 2)

def test_q_exact_for_grid_dead_times():
    """q = fmod(t_d,t_r) N / t_r is an exact integer for every dead time of the
    fixed workloads, so ceil() cannot flip on a rounding error."""
    for t_d, N, q in [(75, 1000, 750), (75, 2000, 1500), (10, 10000, 1000), (40, 10000, 4000),
                      (75, 10000, 7500), (130, 10000, 3000), (0, 1000, 0), (200, 1000, 0)]:
        p = _px(t_d=float(t_d), n_bins=N)
        assert oracle.shift_q(p) == q
        assert oracle.shift_l(p) == q
        assert oracle.shift_exact(p) == q


def test_q_from_delta_would_flip():
    """Why the shift is computed from N and t_r: the bin width 0.01 is not a
    binary fraction, so the quotient by it can land one ulp above an integer."""
    assert math.ceil(0.07 / 0.01) == 8               # 7.000000000000001
    assert oracle.shift_l(_px(t_d=7.0, n_bins=10000)) == 700


@pytest.mark.parametrize("k", range(12))
def test_theorem1_sequential_equals_reparam_with_exact_shift(k):
    """Eq. 4 (Rapp, sequential per entry, periodic replica with ceilings) equals
    Eq. 6 (indicator form) entry by entry when the row shift is the exact
    shift-then-quantise offset.  Covers t_d = 0, t_d > t_r, N from 2 to 64."""
    p = W.as_dicts(W.random_small(12, seed=11))[k]
    Ps = oracle.build_seq(p)
    Pr = oracle.build_reparam(p, oracle.shift_exact(p))
    assert np.all(Ps > 0)
    np.testing.assert_allclose(Pr, Ps, rtol=1e-12, atol=0)


@pytest.mark.parametrize("t_d,N", [(72.0, 20), (70.9, 16), (130.3, 16), (75.0, 16), (71.0, 20),
                                   (99.99, 37), (0.004, 64)])
def test_theorem2_quantise_then_shift(t_d, N):
    """Theorem 2: l = ceil(q) equals the exact shift when frac(q) is 0 or above
    1/2, and is one more when 0 < frac(q) <= 1/2; the rows then differ by
    exactly one circular roll."""
    p = _px(t_d=t_d, n_bins=N, sigma=2.0)
    q = oracle.shift_q(p)
    l, m = oracle.shift_l(p), oracle.shift_exact(p)
    fr = q - math.floor(q)
    if fr == 0.0 or fr > 0.5:
        assert l % N == m
    else:
        assert l % N == (m + 1) % N
    Pl = oracle.build_reparam(p, l)
    Pm = oracle.build_reparam(p, m)
    np.testing.assert_array_equal(Pl, np.roll(Pm, -((l - m) % N), axis=0))


def test_roll_direction_against_sequential():
    """E = J_l E_base takes row (i + l) mod N of E_base as row i (not i - l)."""
    p = _px(t_d=30.0, n_bins=10, sigma=2.0)
    Ps = oracle.build_seq(p)
    base = oracle.build_reparam(p, 0)
    np.testing.assert_allclose(Ps, np.roll(base, -3, axis=0), rtol=1e-12)
    assert not np.allclose(Ps, np.roll(base, 3, axis=0), rtol=1e-6)


# ---------------------------------------------------------------- kernel and normalisation

def test_rows_stochastic():
    """P~ rows sum to 1 (Sec. 2.3)."""
    p = _px(n_bins=300, S=5.0, B=0.01)
    Pt = oracle.normalize_rows(oracle.build_seq(p))
    np.testing.assert_allclose(Pt.sum(axis=1), 1.0, atol=1e-14)


def test_row_mass_is_a_riemann_sum_of_a_pdf():
    """Eq. 3 is a pdf in x_{k+1} (with its 1/(1 - e^-Lambda) factor), so
    Delta * sum_j P_ij -> 1 for every row, first order in Delta."""
    errs = []
    for N in (250, 500, 1000, 2000):
        p = _px(n_bins=N)
        m = (100.0 / N) * oracle.build_seq(p).sum(axis=1)
        errs.append(np.abs(m - 1.0).max())
    assert errs[-1] < 0.011
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


# ---------------------------------------------------------------- stationary distribution

@pytest.mark.parametrize("kw", [dict(), dict(n_bins=400, S=5.0, B=0.01, sigma=0.3),
                                dict(n_bins=333, t_d=130.0, S=3.0, B=6.0),
                                dict(n_bins=256, t_d=95.0, S=9.0, B=9.0)])
def test_power_iteration_is_lapack_left_eigenvector(kw):
    """pi P~ = pi: dense power iteration agrees with LAPACK's eigenvector of
    P~^T for eigenvalue 1 (Sec. 2.3), and that eigenvalue is simple."""
    p = _px(**kw)
    Pt = oracle.normalize_rows(oracle.build_seq(p))
    pi, it, last = oracle.power(Pt, tol=1e-13)
    assert it > 0
    w, V = np.linalg.eig(Pt.T)
    o = np.argsort(-np.abs(w))
    assert abs(w[o[0]] - 1.0) < 1e-12 and abs(w[o[1]]) < 1.0 - 1e-3
    v = np.real(V[:, o[0]])
    v = v / v.sum()
    assert np.abs(v - pi).sum() < 1e-11
    assert np.abs(pi @ Pt - pi).sum() < 1e-12


def test_start_vector_independence():
    """The chain is irreducible and aperiodic (Sec. 2.3), so any positive start
    reaches the same pi."""
    p = _px(n_bins=500, S=3.0, B=1.0)
    Pt = oracle.normalize_rows(oracle.build_seq(p))
    a, _, _ = oracle.power(Pt, tol=1e-14)
    b, _, _ = oracle.power(Pt, tol=1e-14, start=np.random.default_rng(0).uniform(0.1, 1, 500))
    assert np.abs(a - b).sum() < 1e-12


@pytest.mark.parametrize("t_d", [0.0, 33.3, 75.0, 130.0])
def test_pure_background_is_uniform(t_d):
    """S = 0: lambda is constant, P is circulant, so pi = 1/N exactly."""
    p = _px(n_bins=200, S=0.0, B=2.0, t_d=t_d)
    pi = oracle.stationary(p)
    assert np.abs(pi - 1.0 / 200).max() < 1e-15


def test_zero_dead_time_limit_first_order():
    """t_d = 0: timestamps are i.i.d. with density f_a = lambda / Lambda
    (Sec. 2.2), so pi -> lambda(s_j)/sum(lambda) as Delta -> 0; the
    discretisation error halves with each doubling of N."""
    errs = []
    for N in (250, 500, 1000, 2000):
        p = _px(n_bins=N, t_d=0.0)
        lam = oracle.flux_lambda(p, (np.arange(N) + 0.5) * 100.0 / N)
        errs.append(np.abs(oracle.stationary(p) - lam / lam.sum()).sum())
    for a, b in zip(errs, errs[1:]):
        assert 1.9 < a / b < 2.1
    assert errs[-1] < 5e-3


def _chi2_check(p, pi, hist):
    n = hist.sum()
    E = n * pi
    m = E >= 5
    z = (hist[m] - E[m]) / np.sqrt(E[m])
    dof = int(m.sum()) - 1
    chi = float((z ** 2).sum() / dof)
    zmax = special.ndtri(1 - 0.0005 / m.sum())
    assert abs(chi - 1.0) < 4 * math.sqrt(2.0 / dof), chi
    assert np.abs(z).max() < zmax, np.abs(z).max()


def test_event_monte_carlo_single_pixel():
    """About 1e6 registrations of an event-level simulation of a free-running SPAD
    (Poisson arrivals, non-paralysable dead time, X = T mod t_r) agree with pi
    bin by bin within Poisson noise."""
    p = W.as_dicts(W.single())[0]
    pi = oracle.stationary(p)
    hist = oracle.mc_histogram(p, 1_800_000, np.random.default_rng(1))
    assert hist.sum() > 1e6
    _chi2_check(p, pi, hist)


def test_event_monte_carlo_paper_grid():
    """Sec. 3.5 compares with Monte Carlo at 2^10 bins over S, B in {0.1,3,6,9};
    a subset of that grid at both dead times of Sec. 4.2."""
    g = json.load(open(GOLDEN))
    N = g["mc_fine"]["n_bins"]
    S_set, B_set = g["runtime_grid"]["S"], g["runtime_grid"]["B"]
    for k, (S, B) in enumerate([(S_set[0], B_set[0]), (S_set[1], B_set[1]),
                                (S_set[3], B_set[0]), (S_set[0], B_set[3]), (S_set[2], B_set[1])]):
        for t_d in g["dead_times_spectral"]["t_d"]:
            p = _px(n_bins=N, S=float(S), B=float(B), t_d=float(t_d))
            pi = oracle.stationary(p)
            hist = oracle.mc_histogram(p, 4 * g["mc_fine"]["cycles_per_histogram"],
                                       np.random.default_rng(100 + k))
            _chi2_check(p, pi, hist)


def test_monte_carlo_rejects_wrong_roll():
    """The Monte Carlo pin has power: the chain built with the roll reversed
    (shift -l) is rejected by the same histogram."""
    p = W.as_dicts(W.single())[0]
    hist = oracle.mc_histogram(p, 600_000, np.random.default_rng(2))
    bad = oracle.stationary(p, shift=-oracle.shift_l(p))
    with pytest.raises(AssertionError):
        _chi2_check(p, bad, hist)


def test_batch_matches_single():
    px = W.as_dicts(W.random_small(6, seed=5, n_min=20, n_max=90))
    out, off, iters, used = oracle.batch_stationary(px, nthreads=3)
    assert used == 3 and np.all(iters > 0)
    for k, p in enumerate(px):
        np.testing.assert_array_equal(out[off[k]:off[k + 1]], oracle.stationary(p))


# ---------------------------------------------------------------- spectral statements of Sec. 4

def _lambda2_grid(t_d, Ss=(0.1, 1.0, 3.0, 6.0, 9.0), Bs=(0.1, 1.0, 3.0, 6.0, 9.0), N=256):
    mod = np.zeros((len(Ss), len(Bs)))
    ph = np.zeros_like(mod)
    for a, S in enumerate(Ss):
        for b, B in enumerate(Bs):
            p = _px(n_bins=N, t_d=t_d, S=S, B=B)
            Pt = oracle.normalize_rows(oracle.build_reparam(p, oracle.shift_l(p)))
            w = np.linalg.eigvals(Pt)
            w = w[np.argsort(-np.abs(w))]
            mod[a, b], ph[a, b] = abs(w[1]), abs(np.angle(w[1]))
    return mod, ph


@pytest.mark.parametrize("t_d", [75.0, 95.0])
def test_spectral_gap_decreases_with_background(t_d):
    """Sec. 4.1: the gap 1 - |lambda_2| decreases as B increases."""
    mod, _ = _lambda2_grid(t_d)
    assert np.all(np.diff(mod, axis=1) > 0)


def test_phase_of_lambda2_patterns():
    """Sec. 4.2: at t_d = 75 the phase of lambda_2 grows with B; at t_d = 95 a
    large region (strong signal) has near-zero phase."""
    _, ph75 = _lambda2_grid(75.0)
    _, ph95 = _lambda2_grid(95.0)
    assert np.all(np.diff(ph75[:, 1:], axis=1) > 0)          # B >= 1
    assert np.all(ph95[3:, :] < 0.2)                           # S >= 6
    assert np.all(ph75[3:, 2:] > 0.5)                          # same region at t_d = 75 oscillates
