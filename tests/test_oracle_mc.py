"""Pins of the oracle's counter-based event Monte Carlo (the Monte Carlo
reference of Sec. 5, Fig. 3b/3c), which the GPU Monte Carlo kernel is
compared with bin by bin.

- The random words are Philox4x64-10, checked against NumPy's independent
  implementation of the same published generator.
- The experiment's draw order, truncation, sort and dead-time filter are
  checked by an exact replay in plain Python on NumPy's Philox words.
- The statistics are checked against what the paper and the mathematics fix:
  with no dead time every photon registers, so bin counts are Poisson with
  the flux mass of the bin (Eq. 1 truncated to one period) as mean; with no
  signal the registrations are uniform (a circulant chain); at fine
  resolution the histogram follows the chain's pi (Sec. 5, Fig. 3b).
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2509_20500_gb300 import workloads as W

MASK = (1 << 64) - 1


def _numpy_block(counter, key):
    """Philox4x64-10 block at `counter` from NumPy (which increments its
    counter before generating, so it is seeded with counter - 1)."""
    c = [int(x) for x in counter]
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = MASK
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("counter,key", [([0, 0, 0, 0], [0, 0]), ([1, 0, 0, 0], [1, 2]),
                                         ([7, 3, 0, 0], [12345, (5 << 32) | 7]),
                                         ([MASK, MASK, MASK, MASK], [MASK, MASK]),
                                         ([0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0,
                                           0x082EFA98EC4E6C89], [0x452821E638D01377, 0xBE5466CF34E90C6C])])
def test_philox_matches_numpy(counter, key):
    np.testing.assert_array_equal(oracle.philox4x64(counter, key), _numpy_block(counter, key))


def _python_run(p, seed, k, r, cycles):
    """The experiment restated in plain Python on NumPy's Philox words."""
    t_r, t_d, tau, sg = float(p["t_r"]), float(p["t_d"]), float(p["tau"]), float(p["sigma"])
    S, B, N = float(p["S"]), float(p["B"]), int(p["n_bins"])
    key = [seed, (k << 32) | r]
    hist = np.zeros(N, dtype=np.int64)
    ready = -math.inf

    for c in range(cycles):
        words, b = [], 0

        def uni():
            nonlocal b
            if not words:
                words.extend(int(w) for w in _numpy_block([c, b, 0, 0], key))
                b += 1
            w = words.pop(0)
            return ((w >> 11) + 0.5) * 2.0 ** -53

        def poisson(mean):
            u = uni()
            pk = math.exp(-mean)
            F, n = pk, 0
            while u > F and n < 64:
                n += 1
                pk = (pk * mean) / n
                F = F + pk
            return n

        arr = []
        for _ in range(poisson(S)):
            u1, u2 = uni(), uni()
            x = tau + sg * (math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2))
            if 0.0 <= x < t_r:
                arr.append(x)
        for _ in range(poisson(B)):
            arr.append(uni() * t_r)
        arr.sort()   # stable
        for x in arr:
            if x >= ready:
                hist[min(int((x * N) / t_r), N - 1)] += 1
                ready = x + t_d
        ready = ready - t_r
    return hist


def test_mc_exact_replay_in_python():
    px = np.concatenate([W.pixel(64, 75.0, 30.0, 0.5, 3.0, 2.0), W.pixel(50, 130.0, 90.0, 4.0, 6.0, 0.0),
                         W.pixel(40, 0.0, 10.0, 1.0, 0.0, 5.0), W.pixel(33, 20.0, 2.0, 3.0, 9.0, 1.0)])
    pixels = W.as_dicts(px)
    runs, cycles, seed = 2, 150, 2024
    hist, off = oracle.mc_philox_histograms(pixels, runs, cycles, seed)
    for k, p in enumerate(pixels):
        N = int(p["n_bins"])
        for r in range(runs):
            got = hist[runs * off[k] + r * N: runs * off[k] + (r + 1) * N]
            np.testing.assert_array_equal(got, _python_run(p, seed, k, r, cycles))


def _chi2_ok(hist, E):
    m = E >= 5
    z = (hist[m] - E[m]) / np.sqrt(E[m])
    dof = int(m.sum())
    chi = float((z ** 2).sum() / dof)
    assert abs(chi - 1.0) < 4 * math.sqrt(2.0 / dof), chi
    assert np.abs(z).max() < special.ndtri(1 - 0.0005 / dof), np.abs(z).max()


@pytest.mark.parametrize("S,B,tau,sigma", [(5.0, 2.0, 30.0, 0.5), (8.0, 0.0, 3.0, 2.0), (2.0, 4.0, 98.0, 1.5)])
def test_mc_without_dead_time_is_the_flux_mass(S, B, tau, sigma):
    """t_d = 0: every photon registers, so the counts of bin j over C cycles
    are Poisson with mean C (F((j+1) Delta) - F(j Delta)) (Eq. 1, truncated
    to one period; the truncation shows when tau is within a few sigma of 0
    or t_r)."""
    N, runs, cycles = 200, 8, 20000
    p = W.as_dicts(W.pixel(N, 0.0, tau, sigma, S, B))[0]
    hist, _ = oracle.mc_philox_histograms([p], runs, cycles, seed=11)
    h = hist.reshape(runs, N).sum(axis=0).astype(np.float64)
    edges = np.arange(N + 1) * 100.0 / N
    F = oracle.flux_F(p, edges)
    E = runs * cycles * np.diff(F)
    _chi2_ok(h, E)
    # and the total is the truncated period flux, not S + B
    assert abs(h.sum() - runs * cycles * oracle.Lambda(p)) < 5 * math.sqrt(runs * cycles * oracle.Lambda(p))


@pytest.mark.parametrize("t_d", [20.0, 75.0, 130.0])
def test_mc_background_only_is_uniform(t_d):
    N, runs, cycles = 100, 8, 20000
    p = W.as_dicts(W.pixel(N, t_d, 30.0, 0.5, 0.0, 3.0))[0]
    hist, _ = oracle.mc_philox_histograms([p], runs, cycles, seed=12)
    h = hist.reshape(runs, N).sum(axis=0).astype(np.float64)
    _chi2_ok(h, np.full(N, h.sum() / N))


@pytest.mark.parametrize("S,B,t_d", [(0.5, 0.5, 75.0), (6.0, 3.0, 95.0), (9.0, 0.1, 75.0), (3.0, 6.0, 130.0)])
def test_mc_follows_the_chain_at_fine_bins(S, B, t_d):
    """Sec. 5: at 2^10 bins the chain's pi matches Monte Carlo within its
    noise (here about 1e6 registrations)."""
    N, runs, cycles = 1024, 24, 50000
    p = W.as_dicts(W.pixel(N, t_d, 30.0, 0.5, S, B))[0]
    pi = oracle.stationary(p)
    hist, _ = oracle.mc_philox_histograms([p], runs, cycles, seed=13)
    h = hist.reshape(runs, N).sum(axis=0).astype(np.float64)
    _chi2_ok(h, h.sum() * pi)


def test_mc_rejects_a_wrong_dead_time():
    """The chain comparison has power: pi at t_d = 70 is rejected by the
    histogram simulated at t_d = 75."""
    N, runs, cycles = 1024, 24, 50000
    p = W.as_dicts(W.pixel(N, 75.0, 30.0, 0.5, 6.0, 3.0))[0]
    hist, _ = oracle.mc_philox_histograms([p], runs, cycles, seed=14)
    h = hist.reshape(runs, N).sum(axis=0).astype(np.float64)
    wrong = oracle.stationary(W.as_dicts(W.pixel(N, 70.0, 30.0, 0.5, 6.0, 3.0))[0])
    with pytest.raises(AssertionError):
        _chi2_ok(h, h.sum() * wrong)


def test_single_run_entry_matches_the_batch():
    px = W.as_dicts(np.concatenate([W.pixel(64, 75.0, 30.0, 0.5, 3.0, 2.0), W.pixel(80, 95.0, 60.0, 1.0, 7.0, 1.0)]))
    hist, off = oracle.mc_philox_histograms(px, 3, 500, seed=9)
    for k, p in enumerate(px):
        N = int(p["n_bins"])
        for r in range(3):
            np.testing.assert_array_equal(hist[3 * off[k] + r * N: 3 * off[k] + (r + 1) * N],
                                          oracle.mc_philox_run(p, k, r, 500, seed=9))
