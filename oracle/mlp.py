"""FP64 NumPy reference of the learned warm-start network.

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the GPU library).

The network maps a pixel's parameters to a start vector for the power
iteration.  Inputs (scaled to about [-1, 1]):
  f0 = 2 (tau / Delta - c) - 1     (sub-bin pulse position, c = floor(tau / Delta))
  f1 = (sigma - 0.6) / 0.4
  f2 = (log S + 1.5) / 3.1
  f3 = (log B + 1.5) / 3.1
  f4 = 2 (t_d mod t_r) / t_r - 1
Layers: 4 hidden layers h = GELU(W h + b) with GELU in its tanh form
x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) (an approximation of x Phi(x)), then
z = W h + b with one output per bin of the learned frame.  Output index i
corresponds to bin (i + c) mod N; the start vector is
  q_j = softmax_j( z_{(j - c) mod N} + log lambda(s_j) )
with lambda the Eq. 1 flux at bin centres.  Training loss: the mean over
pixels of the cross-entropy -sum_j t_j log q_j against a target pmf t.

Parameters are a list of (W, b) with W of shape [out, in]; the packed order
(layer by layer, W row-major then b) is the one the C ABI uses.

Parity status: forward and backward are pinned by central finite
differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import math

import numpy as np


def features(p) -> tuple[np.ndarray, int]:
    N = int(p["n_bins"])
    t_r, tau = float(p["t_r"]), float(p["tau"])
    c = min(max(int(math.floor(tau * N / t_r)), 0), N - 1)
    pos = tau * N / t_r
    f = np.array([2.0 * (pos - c) - 1.0,
                  (float(p["sigma"]) - 0.6) / 0.4,
                  (math.log(max(float(p["S"]), 1e-30)) + 1.5) / 3.1,
                  (math.log(max(float(p["B"]), 1e-30)) + 1.5) / 3.1,
                  2.0 * math.fmod(float(p["t_d"]), t_r) / t_r - 1.0])
    return f, c


def log_prior(p) -> np.ndarray:
    """log lambda(s_j), Eq. 1 at the bin centres."""
    N = int(p["n_bins"])
    t_r, tau, sig = float(p["t_r"]), float(p["tau"]), float(p["sigma"])
    s = (np.arange(N) + 0.5) * t_r / N
    z = (s - tau) / sig
    lam = float(p["S"]) * np.exp(-0.5 * z * z) / (sig * math.sqrt(2.0 * math.pi)) + float(p["B"]) / t_r
    return np.log(lam)


GELU_K = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(x):
    """GELU in its tanh form (Hendrycks and Gimpel, 2016):
    x/2 (1 + tanh(k (x + a x^3))), k = sqrt(2/pi), a = 0.044715; within 5e-4
    of x Phi(x) everywhere."""
    return 0.5 * x * (1.0 + np.tanh(GELU_K * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    t = np.tanh(GELU_K * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_A * x * x)


def init_params(sizes, seed):
    """Uniform fan-in initialisation; sizes = [in, h1, ..., out]."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = math.sqrt(3.0 / a)
        params.append((rng.uniform(-lim, lim, (b, a)), np.zeros(b)))
    return params


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unpack(vec, sizes):
    params, k = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = vec[k:k + a * b].reshape(b, a)
        k += a * b
        bb = vec[k:k + b]
        k += b
        params.append((np.array(W, dtype=np.float64), np.array(bb, dtype=np.float64)))
    return params


def forward(params, X):
    """X [m, in] -> (z [m, out], cache)."""
    hs, pres = [X], []
    h = X
    for W, b in params[:-1]:
        a = h @ W.T + b
        pres.append(a)
        h = gelu(a)
        hs.append(h)
    W, b = params[-1]
    return h @ W.T + b, (hs, pres)


def start_vectors(params, pixels) -> list[np.ndarray]:
    """The network's start vector q for each pixel."""
    X = np.stack([features(p)[0] for p in pixels])
    z, _ = forward(params, X)
    out = []
    for k, p in enumerate(pixels):
        N = int(p["n_bins"])
        c = features(p)[1]
        e = z[k, (np.arange(N) - c) % N] + log_prior(p)
        e -= e.max()
        q = np.exp(e)
        out.append(q / q.sum())
    return out


def loss_and_grad(params, pixels, targets):
    """Mean cross-entropy and its gradient (list of (dW, db))."""
    m = len(pixels)
    X = np.stack([features(p)[0] for p in pixels])
    z, (hs, pres) = forward(params, X)
    dz = np.zeros_like(z)
    loss = 0.0
    for k, p in enumerate(pixels):
        N = int(p["n_bins"])
        c = features(p)[1]
        idx = (np.arange(N) - c) % N
        e = z[k, idx] + log_prior(p)
        mx = e.max()
        lse = mx + math.log(np.exp(e - mx).sum())
        q = np.exp(e - lse)
        t = np.asarray(targets[k], dtype=np.float64)
        loss -= float(t @ (e - lse))
        dz[k, idx] = (q - t)
    loss /= m
    dz /= m
    grads = [None] * len(params)
    W, b = params[-1]
    grads[-1] = (dz.T @ hs[-1], dz.sum(axis=0))
    dh = dz @ W
    for l in range(len(params) - 2, -1, -1):
        da = dh * gelu_grad(pres[l])
        grads[l] = (da.T @ hs[l], da.sum(axis=0))
        W, _ = params[l]
        dh = da @ W
    return loss, grads
