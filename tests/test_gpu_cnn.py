"""Warm-start network kernels against the FP64 reference (oracle/cnn.py), and the trained
network's effect on the solver.

Tolerances: the convolutions read BF16 operands (8-bit mantissa, relative rounding 2^-9) and the
activations between blocks are stored in BF16, so each of the five layers adds ~0.2-0.4 % relative
error; the bars below (relative L2 2e-2, cosine 0.999) leave room for five such layers and catch
any wrong index, sign or tap (those give O(1) errors)."""
import os

import numpy as np
import pytest

from oracle import cnn as ref

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


def _theta(seed):
    from paper_2206_11009_gb300 import learn
    th = learn.init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    lay, _ = ref.param_layout()
    for e in lay:   # non-trivial biases and gains
        th[e["b"]:e["b"] + e["cout"]] = 0.1 * rng.standard_normal(e["cout"])
        if e["norm"]:
            th[e["g"]:e["g"] + e["cout"]] = 1.0 + 0.2 * rng.standard_normal(e["cout"])
    return th.astype(np.float32)


def test_layout_matches_reference():
    from paper_2206_11009_gb300 import _lib, learn
    lib = _lib.load()
    assert lib.ot_cnn_param_count(32) == ref.param_layout()[1]
    assert lib.ot_cnn_param_count(16) == -1
    th = learn.init_params(3)
    np.testing.assert_allclose(th, ref.init_params(3).astype(np.float32), rtol=0, atol=0)


def test_features_match_reference():
    from paper_2206_11009_gb300 import learn, synth
    inst = synth.image_pair(8, 0)
    np.testing.assert_allclose(learn.features(inst.a, inst.b, 8), ref.features(inst.a, inst.b, 8)[0], rtol=1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("k,B", [(12, 2), (19, 3), (64, 12)])
def test_forward_backward_match_reference(k, B):
    """Ragged tiles (288 and 1,083 pixels: tiles of 128 pixels, chunks of 128 for the weight
    gradient), dilations up to 8 on a 12-pixel image (most taps outside), and 64x64 x 12 = 384 tiles:
    more than the 2 x 152 persistent CTAs of the tensor-core convolution, so some take a second
    tile (the mbarrier's second phase)."""
    from paper_2206_11009_gb300.learn import WarmNet
    th = _theta(11)
    rng = np.random.default_rng(k)
    x = rng.standard_normal((B, 2, k, k)).astype(np.float32)
    dy = rng.standard_normal((B, 2, k, k)).astype(np.float32)
    y_ref, cache = ref.forward(th.astype(np.float64), x.astype(np.float64))
    g_ref, gx_ref = ref.backward(th.astype(np.float64), cache, dy.astype(np.float64))
    net = WarmNet(th)
    xd = torch.from_numpy(x).cuda()
    y = net.forward(xd).cpu().numpy()
    assert _rel(y, y_ref) < 2e-2
    dx = torch.empty_like(xd)
    g = net.backward(xd, torch.from_numpy(dy).cuda(), dx).cpu().numpy()
    gx = dx.cpu().numpy()
    assert _rel(g, g_ref) < 3e-2 and _cos(g, g_ref) > 0.999
    assert _rel(gx, gx_ref) < 3e-2 and _cos(gx, gx_ref) > 0.999
    # per layer: every block's weight gradient points the same way as the reference's
    lay, _ = ref.param_layout()
    for e in lay:
        sl = slice(e["W"], e["b"])
        assert _cos(g[sl], g_ref[sl]) > 0.99
    net.close()


@pytest.mark.gpu
def test_loss_matches_reference():
    from paper_2206_11009_gb300.learn import WarmNet
    th = _theta(12)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 2, 10, 10)).astype(np.float32)
    tgt = rng.standard_normal((2, 2, 10, 10)).astype(np.float32)
    net = WarmNet(th)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(tgt).cuda()
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    L = net.loss_and_grad(xd, td)
    L_ref, gy_ref = ref.loss(y, tgt.astype(np.float64))
    assert abs(L - L_ref) <= 1e-5 * L_ref
    # the loss gradient fed to backward equals the reference's (checked through sum(dy * y))
    g1 = net.grad.clone()
    g2 = net.backward(xd, torch.from_numpy(gy_ref.astype(np.float32)).cuda())
    assert _rel(g1.cpu().numpy(), g2.cpu().numpy()) < 1e-5
    net.close()


@pytest.mark.gpu
def test_adam_step_matches_numpy():
    from paper_2206_11009_gb300.learn import WarmNet
    th = _theta(13)
    net = WarmNet(th)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(th.size).astype(np.float32)
    net.grad.copy_(torch.from_numpy(g).cuda())
    net.adam(1e-3)
    m = 0.1 * g
    v = 0.001 * g * g
    want = th - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    np.testing.assert_allclose(net.params(), want, rtol=2e-6, atol=2e-7)
    net.close()


@pytest.mark.gpu
def test_training_reduces_loss():
    from paper_2206_11009_gb300 import learn
    # targets from another network: a task the architecture can represent exactly
    teacher = learn.WarmNet(_theta(21))
    rng = np.random.default_rng(7)
    X = rng.standard_normal((24, 2, 16, 16)).astype(np.float32)
    Y = teacher.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    teacher.close()
    net = learn.WarmNet(learn.init_params(22))
    hist = learn.train(net, {16: (X, Y)}, steps=150, batch=8, lr=3e-3, verbose=False)
    assert np.mean(hist[-10:]) < 0.5 * np.mean(hist[:10])
    net.close()


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [0, 1])
def test_trained_warm_start_on_heldout_pairs(seed):
    """What the trained network gains over the cold start on held-out 32x32 pairs: the solve
    with the network's duals reaches the same optimum, never takes more iterations than the cold
    one (a warm start that loses to the cold starting point is dropped at creation), and the
    recorded iteration counts say what it gained."""
    from paper_2206_11009_gb300 import Solver, learn, synth
    if not os.path.exists(learn.WEIGHTS):
        pytest.skip("no trained parameters in the package")
    k = 32
    inst = synth.image_pair(k, seed)
    net = learn.WarmNet.load()
    u, v = net.predict(inst.a, inst.b, k)
    net.close()
    with Solver(inst.a, inst.b, grid=(k, k)) as s:
        cold = s.solve()
    with Solver(inst.a, inst.b, grid=(k, k), warm=(u, v)) as s:
        warm = s.solve()
    assert abs(warm.obj - cold.obj) <= 1e-6 * abs(cold.obj)
    assert warm.iters <= cold.iters + (0 if warm.warm_restarts else 10)
    print(f"seed {seed}: cold {cold.iters} iterations, warm {warm.iters} "
          f"(added {warm.warm_added}, dropped {warm.warm_restarts})")
