"""Pins of the FP64 warm-start network reference (oracle/cnn.py) against mathematics that does
not go through its own code: finite differences, the impulse response of a dilated correlation,
the 1x1 special case, the scale invariance of the RMS normalisation, and the gauge invariance of
the loss."""
import numpy as np
import pytest

from oracle import cnn


def _small(seed, ch=4, k=7, B=2):
    rng = np.random.default_rng(seed)
    lay, total = cnn.param_layout(ch)
    theta = rng.standard_normal(total) * 0.4
    for e in lay:
        if e["norm"]:
            theta[e["g"]:e["g"] + e["cout"]] = 1.0 + 0.1 * rng.standard_normal(e["cout"])
    x = rng.standard_normal((B, 2, k, k))
    return theta, x


def test_impulse_response_of_dilated_conv():
    # a unit impulse at (y0, x0) lands tap (ty, tx) at (y0 - (ty-1) d, x0 - (tx-1) d)
    rng = np.random.default_rng(0)
    for d in (1, 2, 3):
        W = rng.standard_normal((3, 2, 3, 3))
        x = np.zeros((1, 2, 11, 11))
        x[0, 1, 5, 5] = 1.0
        out = cnn.conv(x, W, np.zeros(3), d)
        for ty in range(3):
            for tx in range(3):
                y, xx = 5 - (ty - 1) * d, 5 - (tx - 1) * d
                np.testing.assert_allclose(out[0, :, y, xx], W[:, 1, ty, tx], rtol=0, atol=1e-15)
        # everything else is zero
        mask = np.ones((11, 11), bool)
        for ty in range(3):
            for tx in range(3):
                mask[5 - (ty - 1) * d, 5 - (tx - 1) * d] = False
        assert np.all(out[0][:, mask] == 0.0)


def test_center_tap_conv_is_channel_matmul():
    rng = np.random.default_rng(1)
    W = np.zeros((5, 3, 3, 3))
    W[:, :, 1, 1] = rng.standard_normal((5, 3))
    b = rng.standard_normal(5)
    x = rng.standard_normal((2, 3, 6, 4))
    want = np.einsum("oc,bchw->bohw", W[:, :, 1, 1], x) + b[None, :, None, None]
    np.testing.assert_allclose(cnn.conv(x, W, b, 4), want, rtol=1e-13, atol=1e-13)


def test_zero_padding_border():
    # a constant input: an interior pixel sees all 9 taps, a corner pixel only 4 (d = 1)
    W = np.ones((1, 1, 3, 3))
    x = np.ones((1, 1, 5, 5))
    out = cnn.conv(x, W, np.zeros(1), 1)
    assert out[0, 0, 2, 2] == 9.0 and out[0, 0, 0, 0] == 4.0 and out[0, 0, 0, 2] == 6.0


def test_rmsnorm_removes_scale_of_first_layer():
    theta, x = _small(2)
    lay, _ = cnn.param_layout(4)
    e = lay[0]
    y1, _ = cnn.forward(theta, x, ch=4)
    t2 = theta.copy()
    t2[e["W"]:e["b"] + e["cout"]] *= 7.5   # W and bias of the first conv
    y2, _ = cnn.forward(t2, x, ch=4)
    # equal up to the eps inside the square root
    np.testing.assert_allclose(y2, y1, rtol=0, atol=5e-5 * np.abs(y1).max())


def test_silu_values():
    assert cnn.silu(np.array(0.0)) == 0.0
    np.testing.assert_allclose(cnn.silu(np.array([30.0, -30.0])), [30.0, 0.0], atol=1e-11)
    np.testing.assert_allclose(cnn.silu(np.array(1.0)), 1.0 / (1.0 + np.exp(-1.0)), rtol=1e-15)


def test_loss_gauge_invariance_and_zero():
    rng = np.random.default_rng(3)
    y = rng.standard_normal((2, 2, 5, 5))
    tgt = rng.standard_normal((2, 2, 5, 5))
    L0, _ = cnn.loss(y, tgt)
    y2 = y.copy()
    y2[:, 0] += 3.7
    y2[:, 1] -= 3.7
    L1, _ = cnn.loss(y2, tgt)
    assert abs(L1 - L0) < 1e-12
    # a prediction that differs only by a gauge has zero loss
    t = tgt.copy()
    t[:, 0] -= 1.25
    t[:, 1] += 1.25
    assert cnn.loss(t, tgt)[0] < 1e-28


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(4)
    y = rng.standard_normal((2, 2, 4, 3))
    tgt = rng.standard_normal((2, 2, 4, 3))
    _, g = cnn.loss(y, tgt)
    h = 1e-6
    for idx in [(0, 0, 1, 2), (1, 1, 3, 0), (0, 1, 0, 0), (1, 0, 2, 1)]:
        yp, ym = y.copy(), y.copy()
        yp[idx] += h
        ym[idx] -= h
        fd = (cnn.loss(yp, tgt)[0] - cnn.loss(ym, tgt)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8


@pytest.mark.parametrize("seed", [5, 6])
def test_backward_finite_differences(seed):
    theta, x = _small(seed)
    y, cache = cnn.forward(theta, x, ch=4)
    rng = np.random.default_rng(seed + 100)
    dy = rng.standard_normal(y.shape)
    grad, gx = cnn.backward(theta, cache, dy, ch=4)

    def f(th, xx):
        return float(np.sum(dy * cnn.forward(th, xx, ch=4)[0]))

    h = 1e-6
    idxs = rng.choice(theta.size, 40, replace=False)
    lay, _ = cnn.param_layout(4)
    idxs = np.concatenate([idxs, [e["g"] for e in lay if e["norm"]], [e["b"] for e in lay]])
    for i in idxs:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (f(tp, x) - f(tm, x)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * (1.0 + abs(fd)), (i, fd, grad[i])
    for idx in [(0, 0, 3, 3), (1, 1, 0, 6), (0, 1, 6, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (f(theta, xp) - f(theta, xm)) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * (1.0 + abs(fd))


def test_layout_size_and_receptive_field():
    lay, total = cnn.param_layout()
    # 2->32, three 32->32, 32->2 convolutions; biases; gains of the four normalised blocks
    assert total == (32 * 2 * 9 + 3 * 32 * 32 * 9 + 2 * 32 * 9) + (4 * 32 + 2) + 4 * 32
    # receptive field: 1 + 2 * (1 + 2 + 4 + 8 + 1) = 33: a pixel 16 away still matters, 17 not
    theta, _ = _small(7, ch=32, k=1)
    x = np.zeros((1, 2, 41, 41))
    y0, _ = cnn.forward(theta, x, ch=32)
    x16 = x.copy(); x16[0, 0, 20, 36] = 1.0
    x17 = x.copy(); x17[0, 0, 20, 37] = 1.0
    y16, _ = cnn.forward(theta, x16, ch=32)
    y17, _ = cnn.forward(theta, x17, ch=32)
    assert np.abs(y16[0, :, 20, 20] - y0[0, :, 20, 20]).max() > 0
    assert np.abs(y17[0, :, 20, 20] - y0[0, :, 20, 20]).max() == 0
