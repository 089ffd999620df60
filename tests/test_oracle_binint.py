"""Pins of the oracle's bin-integrated variant of Eq. 6 (an ablation beyond
the paper): the column weight of bin j is the exact integral of the
detection density over the bin, exp(-F(j Delta)) - exp(-F((j+1) Delta))
(relative to the re-arm point), where the paper's form takes its midpoint
value lambda(s_j) exp(-F(s_j)) Delta (Sec. 3.4)."""
import math

import numpy as np
import pytest

import oracle
from paper_2509_20500_gb300 import workloads as W


def _p(**kw):
    base = dict(n_bins=200, t_d=75.0, tau=30.0, sigma=0.5, S=3.0, B=1.0)
    base.update(kw)
    return W.as_dicts(W.pixel(**base))[0]


@pytest.mark.parametrize("kw", [dict(), dict(S=9.5, B=0.0, n_bins=64), dict(t_d=130.0, sigma=2.0, n_bins=97),
                                dict(tau=99.0, sigma=1.5, S=6.0, B=4.0)])
def test_row_sums_telescope(kw):
    """Summed over j the bin integrals telescope: a row re-armed at s_p
    sums to exp(F(s_p) - F(p Delta)) (1 - exp(-Lambda)), i.e. to
    exp(F(s_p) - F(p Delta)) / Delta on the builder's scale."""
    p = _p(**kw)
    N = int(p["n_bins"])
    Delta = 100.0 / N
    l = oracle.shift_l(p)
    P = oracle.build_binint(p, l)
    for i in range(N):
        q = (i + l) % N
        want = math.exp(oracle.flux_F(p, np.array([(q + 0.5) * Delta]))[0]
                        - oracle.flux_F(p, np.array([q * Delta]))[0]) / Delta
        assert abs(P[i].sum() - want) < 1e-12 * want


def test_second_order_agreement_with_point_form():
    """The point form is the midpoint rule of the bin integral, so the two
    stationary pmfs approach each other as Delta^2."""
    errs = []
    for N in (250, 500, 1000, 2000):
        p = _p(n_bins=N)
        l = oracle.shift_l(p)
        errs.append(np.abs(oracle.stationary(p, shift=l) - oracle.stationary(p, shift=l, flux="binint")).sum())
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4, errs


@pytest.mark.parametrize("t_d", [20.0, 75.0, 130.0])
def test_background_only_is_uniform(t_d):
    p = _p(S=0.0, B=2.0, t_d=t_d, n_bins=120)
    pi = oracle.stationary(p, shift=oracle.shift_l(p), flux="binint")
    assert np.abs(pi - 1.0 / 120).max() < 1e-14


@pytest.mark.parametrize("S,B", [(9.5, 0.0), (10.0, 0.5), (5.0, 1.0)])
def test_closer_to_monte_carlo_at_coarse_bins(S, B):
    """At 2^8 bins (Fig. 3c) and a bright pulse, the midpoint rule shows
    against the event Monte Carlo (25 x 50,000 cycles); the bin integral
    cuts the L1 gap at least in half."""
    p = _p(n_bins=256, S=S, B=B)
    h, _ = oracle.mc_philox_histograms([p], 25, 50000, seed=3)
    f = h.reshape(25, 256).sum(axis=0) / h.sum()
    l = oracle.shift_l(p)
    d_point = np.abs(oracle.stationary(p, shift=l) - f).sum()
    d_int = np.abs(oracle.stationary(p, shift=l, flux="binint") - f).sum()
    assert d_int < 0.5 * d_point, (d_point, d_int)
