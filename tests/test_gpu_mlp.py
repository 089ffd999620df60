"""Tensor-core GEMM and the learned warm-start network on the GPU.

The GEMM (tcgen05, BF16 operands, FP32 accumulation) is compared with a
plain PyTorch FP32 matmul of the same BF16 operands.  The network's loss and
gradients are compared with the FP64 NumPy reference (oracle/mlp.py, pinned
by finite differences) at the same parameters; BF16 weights and activations
bound the agreement at about 1e-2 relative.  The learned batch path is
checked against the FP64 oracle (1e-6 L1) and for what it gains in power
steps over the plain start.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref_mlp
from paper_2509_20500_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [5, 512, 512, 512, 512, 2000]


@pytest.fixture(scope="module")
def spl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_20500_gb300 import build, spl as S
    build.build()
    S.lib()
    return S


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 256, 512), (384, 96, 192), (128, 2048, 512),
                                   (2048, 512, 4096)])
def test_gemm_bf16_vs_torch(spl, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = spl.gemm_bf16(A, B)
    ref = A.float() @ B.float().T
    err = (D - ref).abs().max().item()
    scale = (A.float().abs() @ B.float().abs().T).max().item()
    assert err <= 1e-5 * scale, (err, scale)


def _targets(n, seed):
    rng = np.random.default_rng(seed)
    t = rng.gamma(1.0, 1.0, (n, 2000))
    return t / t.sum(axis=1, keepdims=True)


def test_mlp_loss_and_gradients_vs_fp64_reference(spl):
    px = W.array_pixels(96, seed=61)
    pixels = W.as_dicts(px)
    params = ref_mlp.init_params(SIZES, seed=4)
    rng = np.random.default_rng(2)
    params = [(Wm, rng.normal(0, 0.05, b.shape)) for Wm, b in params]
    vec = ref_mlp.pack(params).astype(np.float32)
    net = spl.MLP(max_batch=256, seed=0)
    net.set_params(vec)
    np.testing.assert_array_equal(net.get_params(), vec)
    tg = _targets(len(px), 3)
    loss, g = net.loss_grad(px, torch.tensor(tg, dtype=torch.float32, device="cuda"))
    # reference at the FP32-rounded parameters
    rparams = ref_mlp.unpack(vec.astype(np.float64), SIZES)
    rloss, rgrads = ref_mlp.loss_and_grad(rparams, pixels, tg)
    assert abs(loss - rloss) < 1e-2 * abs(rloss)
    k = 0
    for (dW, db) in rgrads:
        for ref in (dW.ravel(), db):
            got = g[k:k + ref.size].astype(np.float64)
            k += ref.size
            rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
            cos = float(got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30))
            assert rel < 3e-2 and cos > 0.999, (rel, cos)
    assert k == g.size
    net.close()


def test_mlp_start_vector_vs_fp64_reference(spl):
    """The batch kernel's learned start (logits rolled to the pulse bin plus
    the log flux prior, softmax) against the reference start vector: one
    power step from each agrees, and so does the start itself via
    max_iter = 1 semantics (compare the network logits directly)."""
    px = W.array_pixels(40, seed=62)
    pixels = W.as_dicts(px)
    params = ref_mlp.init_params(SIZES, seed=5)
    vec = ref_mlp.pack(params).astype(np.float32)
    net = spl.MLP(max_batch=128, seed=0)
    net.set_params(vec)
    z = net.forward(px).cpu().numpy()[:, :2000].astype(np.float64)
    X = np.stack([ref_mlp.features(p)[0] for p in pixels])
    rz, _ = ref_mlp.forward(ref_mlp.unpack(vec.astype(np.float64), SIZES), X)
    assert np.abs(z - rz).max() < 2e-2 * np.abs(rz).max()
    net.close()


def test_learned_warm_start_gains_iterations(spl):
    """Trained on stationary pmfs the method itself produces, the network's
    start needs fewer power steps than the uniform start, and the result is
    unchanged: the plain iteration still runs to the stop rule and agrees
    with the FP64 oracle to 1e-6 L1."""
    train = W.training(16384, seed=2)
    tgt, off, _ = spl.batch_stationary(train, tol=1e-6)
    tgt = tgt.view(len(train), 2000)
    net = spl.MLP(max_batch=1024, seed=1)
    c_all = [spl.pixels_to_c(train[i:i + 1024]) for i in range(0, len(train), 1024)]
    step = 0
    for epoch in range(12):
        for b, cpx in enumerate(c_all):
            lr = 2e-3 * min(1.0, (step + 1) / 50)
            net.train_step(cpx, 1024, tgt[b * 1024:(b + 1) * 1024], lr=lr)
            step += 1
    torch.cuda.synchronize()
    test = W.array_pixels(2048, seed=77)
    plain, off, rp = spl.batch_stationary(test, tol=1e-6)
    learned, off2, rl = net.batch_stationary(test, tol=1e-6)
    assert np.all(rl["status"] == 0)
    assert rl["iters"].mean() < rp["iters"].mean() - 0.5, (rl["iters"].mean(), rp["iters"].mean())
    o_l = learned.cpu().numpy().astype(np.float64)
    idx = W.sample_indices(len(test), 16, seed=9)
    refs, roff, _, _ = oracle.batch_stationary(W.as_dicts(test[idx]), tol=1e-12)
    for r, k in enumerate(idx):
        assert np.abs(o_l[off[k]:off[k + 1]] - refs[roff[r]:roff[r + 1]]).sum() < 1e-6
    net.close()


def test_learned_start_with_structured_step(spl):
    """The learned warm start also feeds the O(N) form of the step; results
    match the dense form within the parity tolerance."""
    train = W.training(8192, seed=2)
    tgt, _, _ = spl.batch_stationary(train, tol=1e-6)
    net = spl.MLP(max_batch=1024, seed=1)
    tg = tgt.view(len(train), 2000)
    for ep in range(4):
        for b in range(8):
            net.train_step(spl.pixels_to_c(train[b * 1024:(b + 1) * 1024]), 1024, tg[b * 1024:(b + 1) * 1024],
                           lr=2e-3)
    test = W.array_pixels(1500, seed=78)
    d, off, rd = net.batch_stationary(test, tol=1e-6)
    s, _, rs = net.batch_stationary(test, tol=1e-6, pass_kind=spl.SPL_PASS_STRUCTURED)
    assert np.all(rs["status"] == 0)
    d, s = d.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    # each form is within 1e-6 of the exact pmf, so they agree within 2e-6
    for k in range(len(test)):
        assert np.abs(d[off[k]:off[k + 1]] - s[off[k]:off[k + 1]]).sum() < 2e-6
    idx = W.sample_indices(len(test), 12, seed=10)
    refs, roff, _, _ = oracle.batch_stationary(W.as_dicts(test[idx]), tol=1e-12)
    for r, k in enumerate(idx):
        assert np.abs(s[off[k]:off[k + 1]] - refs[roff[r]:roff[r + 1]]).sum() < 1e-6
    net.close()


def test_headline_launch_array256_learned_sampled(spl):
    """The launch the benchmark times: the 256 x 256 array (65536 pixels,
    N = 2000) with the learned start in one persistent launch, dense steps
    with the row sums from the scans (SPL_PASS_DENSE_ROWSCAN), the launch
    configuration chosen by the autotuner; 32 pixels sampled by seed against
    the FP64 oracle (L1 and max-abs), every pmf normalised, every pixel
    converged; the dense-row-pass form on the same network within the
    tolerance of it."""
    train = W.training(16384, seed=2)
    tgt, _, _ = spl.batch_stationary(train, tol=1e-6)
    tgt = tgt.view(len(train), 2000)
    net = spl.MLP(max_batch=65536, seed=1)
    c_all = [spl.pixels_to_c(train[i:i + 4096]) for i in range(0, len(train), 4096)]
    step = 0
    for epoch in range(10):
        for b, cpx in enumerate(c_all):
            net.train_step(cpx, 4096, tgt[b * 4096:(b + 1) * 4096], lr=3e-3 * min(1.0, (step + 1) / 20))
            step += 1
    px = W.array256()
    out, off, reps = net.batch_stationary(px, tol=1e-6, pass_kind=spl.SPL_PASS_DENSE_ROWSCAN)
    assert np.all(reps["status"] == 0)
    o = out.cpu().numpy().astype(np.float64)
    sums = np.add.reduceat(o, off[:-1])
    assert np.abs(sums - 1).max() < 1e-5
    idx = W.sample_indices(len(px), 32, seed=34)
    refs, roff, _, _ = oracle.batch_stationary(W.as_dicts(px[idx]), tol=1e-12)
    dif = [np.abs(o[off[k]:off[k + 1]] - refs[roff[r]:roff[r + 1]]) for r, k in enumerate(idx)]
    worst = max(d.sum() for d in dif)
    assert worst < 1e-6 and max(d.max() for d in dif) <= worst, worst
    d2, _, r2 = net.batch_stationary(px, tol=1e-6, pass_kind=spl.SPL_PASS_DENSE)
    assert np.all(r2["status"] == 0)
    d2 = d2.cpu().numpy().astype(np.float64)
    for k in idx:
        assert np.abs(d2[off[k]:off[k + 1]] - o[off[k]:off[k + 1]]).sum() < 1e-6
    net.close()


def test_checkpoint_resumes_training_exactly(spl, tmp_path):
    """train.save / train.load keep the parameters, the AdamW moments and the
    step count: 3 steps, a checkpoint, a new network loaded from it and 3 more
    steps give the same parameters bit for bit as 6 steps without a break."""
    from paper_2509_20500_gb300 import train as T
    data = W.training(2048, seed=4)
    tgt, _, _ = spl.batch_stationary(data, tol=1e-6)
    tgt = tgt.view(len(data), 2000)
    c = [spl.pixels_to_c(data[i:i + 1024]) for i in (0, 1024)]
    lrs = [1e-3, 2e-3, 3e-3, 3e-3, 2e-3, 1e-3]

    def step(net, k):
        b = k % 2
        net.train_step(c[b], 1024, tgt[b * 1024:(b + 1) * 1024], lr=lrs[k], weight_decay=1e-4)

    a = spl.MLP(max_batch=1024, seed=7)
    for k in range(6):
        step(a, k)
    b = spl.MLP(max_batch=1024, seed=7)
    for k in range(3):
        step(b, k)
    T.save(b, str(tmp_path / "ck.npz"), seed=7, steps=3)
    b.close()
    r = T.load(str(tmp_path / "ck.npz"), max_batch=1024)
    for k in range(3, 6):
        step(r, k)
    np.testing.assert_array_equal(r.get_params(), a.get_params())
    sa, na = a.get_state()
    sr, nr = r.get_state()
    assert na == nr == 6
    np.testing.assert_array_equal(sr, sa)
    a.close()
    r.close()


def test_learned_host_entry_point_matches_device_path(spl):
    """spl_batch_stationary_learned_host (eight ranges copied back while the
    kernel runs, for a batch of one size) gives the device path's pmfs and
    reports bit for bit, into pinned host memory."""
    train = W.training(4096, seed=2)
    tgt, _, _ = spl.batch_stationary(train, tol=1e-6)
    tgt = tgt.view(len(train), 2000)
    net = spl.MLP(max_batch=8192, seed=1)
    for b in range(4):
        net.train_step(spl.pixels_to_c(train[b * 1024:(b + 1) * 1024]), 1024, tgt[b * 1024:(b + 1) * 1024], lr=2e-3)
    px = W.array_pixels(8192, seed=79)           # eight ranges of 1024 pixels
    pk = spl.SPL_PASS_DENSE_ROWSCAN              # the timed path's pass kind
    d, off, rd = net.batch_stationary(px, tol=1e-6, pass_kind=pk)
    h, off2, rh = net.batch_stationary_host(px, tol=1e-6, pass_kind=pk)
    assert np.array_equal(off, off2)
    np.testing.assert_array_equal(h.numpy(), d.cpu().numpy())
    for k in ("iters", "status", "last_step_l1"):
        np.testing.assert_array_equal(rh[k], rd[k])
    net.close()
