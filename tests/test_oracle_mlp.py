"""Pins of the FP64 reference network (oracle/mlp.py) by central finite
differences on a small network, plus the invariants of its start vector."""
import numpy as np
import pytest

from oracle import mlp
from paper_2509_20500_gb300 import workloads as W

SIZES = [5, 7, 6, 6, 7, 24]


def _pixels(n, N=24, seed=0):
    px = W.array_pixels(n, seed=seed, n_bins=N)
    return W.as_dicts(px)


def test_gradient_matches_finite_differences():
    pixels = _pixels(3)
    rng = np.random.default_rng(1)
    targets = [t / t.sum() for t in rng.uniform(0.1, 1.0, (3, 24))]
    params = mlp.init_params(SIZES, seed=3)
    # non-zero biases so every term is exercised
    params = [(Wm, rng.normal(0, 0.3, b.shape)) for Wm, b in params]
    vec = mlp.pack(params)
    loss, grads = mlp.loss_and_grad(params, pixels, targets)
    g = mlp.pack(grads)
    h = 1e-6
    for k in rng.choice(vec.size, 60, replace=False):
        vp, vm = vec.copy(), vec.copy()
        vp[k] += h
        vm[k] -= h
        lp, _ = mlp.loss_and_grad(mlp.unpack(vp, SIZES), pixels, targets)
        lm, _ = mlp.loss_and_grad(mlp.unpack(vm, SIZES), pixels, targets)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 + 1e-5 * abs(fd), (k, fd, g[k])


def test_start_vector_is_pmf_and_follows_prior_at_zero_output():
    """With a zero last layer the start vector is the normalised flux prior
    lambda(s_j) / sum lambda (Eq. 1), whatever the frame roll."""
    pixels = _pixels(4, N=50, seed=5)
    params = mlp.init_params([5, 8, 8, 8, 8, 50], seed=2)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros(50))
    for p, q in zip(pixels, mlp.start_vectors(params, pixels)):
        lam = np.exp(mlp.log_prior(p))
        np.testing.assert_allclose(q, lam / lam.sum(), rtol=1e-12)


def test_frame_roll_follows_pulse_bin():
    """A one-hot output bias at frame index 0 puts the start vector's excess
    mass on the pulse bin c = floor(tau / Delta)."""
    pixels = _pixels(5, N=40, seed=6)
    params = mlp.init_params([5, 8, 8, 8, 8, 40], seed=2)
    b = np.zeros(40)
    b[0] = 30.0
    params[-1] = (np.zeros_like(params[-1][0]), b)
    for p, q in zip(pixels, mlp.start_vectors(params, pixels)):
        _, c = mlp.features(p)
        assert int(np.argmax(q)) == c == int(np.floor(p["tau"] * 40 / p["t_r"]))


def test_loss_is_minimised_by_the_target():
    """Cross-entropy -sum t log q over pmfs q is smallest at q = t (Gibbs)."""
    pixels = _pixels(1, N=30, seed=7)
    p = pixels[0]
    params = mlp.init_params([5, 4, 4, 4, 4, 30], seed=0)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros(30))
    q0 = mlp.start_vectors(params, pixels)[0]
    l_at, _ = mlp.loss_and_grad(params, pixels, [q0])
    rng = np.random.default_rng(0)
    for _ in range(5):
        t = q0 * rng.uniform(0.5, 1.5, 30)
        t /= t.sum()
        l_t, _ = mlp.loss_and_grad(params, pixels, [t])
        # loss(q0 | t) >= entropy(t), loss(q0 | q0) = entropy(q0)
        assert l_t >= -float(t @ np.log(t)) - 1e-12
    assert abs(l_at + float(q0 @ np.log(q0))) < 1e-12


def test_gelu_tanh_form_against_x_phi_and_its_derivative():
    """The activation is the tanh form of GELU: within 5e-4 of x Phi(x)
    (Phi from math.erfc) on [-8, 8], odd part x/2 exactly (GELU(x) - GELU(-x)
    = x), and its derivative matches central differences."""
    import math
    x = np.linspace(-8.0, 8.0, 4001)
    exact = x * 0.5 * np.array([math.erfc(-v / math.sqrt(2.0)) for v in x])
    assert np.abs(mlp.gelu(x) - exact).max() < 5e-4
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, rtol=0, atol=1e-12)
    h = 1e-5
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=0, atol=1e-8)
