"""Training driver of the learned warm start.

The training set is made by the method itself: stationary pmfs of seeded
pixels (N = 2000) computed by the plain batch solver to 1e-6 L1.  The
network is then fitted with the library's own forward/backward kernels and
AdamW (spl_mlp_train_step).  Checkpoints are the packed FP32 parameters plus
the step count and seed in a .npz file.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import spl, workloads


def make_training_set(n: int = 200_000, seed: int = 2, tol: float = 1e-6):
    """Pixels drawn like the 128x128 array workload and their stationary pmfs
    (device tensor [n, 2000]) from the plain batch solver."""
    px = workloads.training(n, seed)
    out, _, reps = spl.batch_stationary(px, tol=tol, reports=True)
    if not np.all(reps["status"] == 0):
        raise RuntimeError("training targets did not converge")
    return px, out.view(n, 2000)


def train(px, targets, epochs: int = 20, batch: int = 4096, lr: float = 2e-3, warmup: int = 100,
          weight_decay: float = 0.0, seed: int = 1, net=None, log=None, max_batch: int = 0):
    """Fits the network on (px, targets) with a linear warm-up then cosine
    learning-rate decay.  Returns the network; max_batch (>= batch) sizes it
    for later inference on larger batches."""
    import torch
    n = len(px)
    nb = n // batch
    if net is None:
        net = spl.MLP(max_batch=max(batch, max_batch), seed=seed)
    rng = np.random.default_rng(seed)
    total = epochs * nb
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = rng.permutation(n)
        # pixel order of this epoch; targets are gathered on the device
        idx_t = torch.from_numpy(perm).to(targets.device)
        tg = targets.index_select(0, idx_t)
        pxe = px[perm]
        loss = None
        for b in range(nb):
            lo = b * batch
            frac = step / max(1, total - 1)
            cur = lr * min(1.0, (step + 1) / warmup) * 0.5 * (1.0 + math.cos(math.pi * frac))
            want = log is not None and b == nb - 1
            loss = net.train_step(spl.pixels_to_c(pxe[lo:lo + batch]), batch, tg[lo:lo + batch], lr=cur,
                                  weight_decay=weight_decay, want_loss=want)
            step += 1
        if log is not None:
            log(f"epoch {ep}: loss {loss:.6f} ({time.perf_counter() - t0:.1f} s)")
    torch.cuda.synchronize()
    return net


def save(net, path: str, seed: int = 0, steps: int = 0):
    """Checkpoint: FP32 parameters, the AdamW moments and step count (so
    training resumes exactly), the seed and the caller's step count."""
    state, opt_step = net.get_state()
    np.savez(path, params=net.get_params(), adam=state, adam_step=opt_step, seed=seed, steps=steps)


def load(path: str, max_batch: int = 4096):
    d = np.load(path)
    net = spl.MLP(max_batch=max_batch, seed=int(d["seed"]))
    net.set_params(d["params"])
    if "adam" in d:
        net.set_state(d["adam"], int(d["adam_step"]))
    return net
