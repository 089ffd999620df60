"""GPU event Monte Carlo (the Monte Carlo reference of Sec. 5) against the
oracle's implementation of the same exactly specified experiment: the same
Philox4x64-10 streams, so every histogram bin of every run must be equal.

Both sides evaluate the photon times in FP64; a registration or bin could
only differ where a time lies within a few units in the last place of a
decision boundary (the two sides' log and cos may differ in the last bit),
an event of probability about 1e-15 per photon.
"""
import numpy as np
import pytest

import oracle
from paper_2509_20500_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_20500_gb300 import build, spl as S
    build.build()
    S.lib()
    return S


def _compare(spl, px, runs, cycles, seed):
    h, off = spl.mc_histograms(px, runs, cycles, seed)
    ref, roff = oracle.mc_philox_histograms(W.as_dicts(px), runs, cycles, seed)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(h.cpu().numpy().view(np.uint32), ref)
    return ref, off


def test_mc_small_cases_bit_exact(spl):
    """Ragged bins, t_d = 0, t_d > t_r, no background, no signal, a pulse cut
    by the period boundary."""
    px = np.concatenate([W.pixel(64, 75.0, 30.0, 0.5, 3.0, 2.0), W.pixel(50, 130.0, 90.0, 4.0, 6.0, 0.0),
                         W.pixel(40, 0.0, 10.0, 1.0, 0.0, 5.0), W.pixel(33, 20.0, 2.0, 3.0, 9.0, 1.0),
                         W.pixel(2, 95.0, 99.5, 2.0, 16.0, 16.0), W.pixel(257, 5.0, 50.0, 0.2, 0.3, 0.01)])
    ref, _ = _compare(spl, px, runs=3, cycles=3000, seed=2024)
    assert ref.sum() > 0


def test_mc_grid_corners_bit_exact(spl):
    """The accuracy grid's extremes at its 256 bins (S, B in {0, 5, 10})."""
    g = W.accuracy_grid(256, steps=3)
    _compare(spl, g, runs=4, cycles=20000, seed=77)


@pytest.mark.parametrize("n_bins", [1024, 4096, 16384])
def test_mc_large_bin_counts_bit_exact(spl, n_bins):
    """Shared-memory histograms with fewer threads per block (1024: 32,
    4096: 8, 16384: 2)."""
    px = np.concatenate([W.pixel(n_bins, 75.0, 30.0, 0.5, 4.0, 3.0), W.pixel(n_bins, 95.0, 70.0, 1.0, 1.0, 8.0),
                         W.pixel(n_bins // 2 + 3, 40.0, 10.0, 0.3, 10.0, 0.5)])
    _compare(spl, px, runs=3, cycles=1500, seed=n_bins)


def test_mc_full_grid_sampled_runs(spl):
    """The accuracy-grid launch the benchmark times (440 pixels x 25 runs x
    50,000 cycles at 256 bins): sampled runs equal the oracle's, and every
    run's histogram is complete."""
    g = W.accuracy_grid()
    runs, cycles, seed = 25, 50000, 3
    h, off = spl.mc_histograms(g, runs, cycles, seed)
    h = h.cpu().numpy().view(np.uint32).reshape(len(g), runs, 256)
    rng = np.random.default_rng(0)
    pixels = W.as_dicts(g)
    for k in list(rng.choice(len(g), 10, replace=False)) + [0, len(g) - 1]:
        r = int(rng.integers(runs))
        np.testing.assert_array_equal(h[k, r], oracle.mc_philox_run(pixels[k], int(k), r, cycles, seed))
    # registrations per cycle never exceed one per dead time plus one
    per_cycle = h.sum(axis=2) / cycles
    assert per_cycle.min() > 0 and per_cycle.max() <= 100.0 / 75.0 + 1.0


def test_mc_matches_the_chain(spl):
    """Sec. 5: at fine bins the GPU histogram (24 x 50,000 cycles) follows
    the chain's stationary pmf from the batch solver within Poisson noise.
    The cases keep the chain's own discretisation error (the midpoint rule
    of the point flux over a bin, about (lambda Delta)^2 / 24 at the pulse
    peak) well below the noise of ~1e6 registrations: moderate flux at 2^10
    bins, a bright narrow pulse at 2^12 bins."""
    px = np.concatenate([W.pixel(1024, 75.0, 30.0, 1.0, 3.0, 1.0), W.pixel(1024, 95.0, 60.0, 2.0, 2.0, 4.0),
                         W.pixel(4096, 95.0, 30.0, 0.5, 9.0, 0.1)])
    nb = [1024, 1024, 4096]
    h, off = spl.mc_histograms(px, 24, 50000, seed=5)
    pi, poff, rep = spl.batch_stationary(px, tol=1e-6)
    h = h.cpu().numpy().view(np.uint32)
    pi = pi.cpu().numpy().astype(np.float64)
    from scipy import special
    for k in range(3):
        hk = h[24 * off[k]: 24 * off[k + 1]].reshape(24, nb[k]).sum(axis=0).astype(np.float64)
        E = hk.sum() * pi[poff[k]:poff[k + 1]]
        m = E >= 5
        z = (hk[m] - E[m]) / np.sqrt(E[m])
        chi = float((z ** 2).mean())
        assert abs(chi - 1.0) < 4 * np.sqrt(2.0 / m.sum()), chi
        assert np.abs(z).max() < special.ndtri(1 - 0.0005 / m.sum())


def test_mc_invalid_input(spl):
    with pytest.raises(RuntimeError):
        spl.mc_histograms(W.pixel(100, 75.0, 30.0, 0.5, 20.0, 1.0), 2, 10, 1)
