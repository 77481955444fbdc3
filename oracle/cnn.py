"""FP64 reference of the warm-start network (test infrastructure only; the solver never imports it).

The paper has no network: its conclusion names a better starting support as future work, and the
warm start built on that hook predicts dual potentials from the two marginals.  The network:

    input    x  (B, 2, k, k): log(a * m), log(b * m)  (masses scaled to mean 1)
    block l  (l = 0..3):  h <- silu(rmsnorm(conv3x3_dil(h; W_l, b_l, dilation 2^l); g_l))
    head     y  (B, 2, k, k) = conv3x3(h; W_4, b_4)   -> predicted (u, v) / k^2

conv3x3_dil: out[b, o, y, x] = bias[o] + sum_{c, ty, tx} W[o, c, ty, tx] in[b, c, y + (ty-1) d, x + (tx-1) d]
with zeros outside the image.  rmsnorm over channels per pixel: g_c x_c / sqrt(mean_c x_c^2 + eps).
silu(t) = t / (1 + exp(-t)).  Loss (gauge invariant, u + t, v - t is the same potential pair):
    r_u = yu - u - t*, r_v = yv - v + t*,  t* = mean(((yu - u) - (yv - v)) / 2) per image,
    L = mean over images, channels and pixels of r^2  (so L = mean_b mean_pix (r_u^2 + r_v^2) / 2).
Every function is a plain restatement of these definitions; backward() is the chain rule written
out and is pinned by finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

EPS = 1e-5
CH = 32
DILATIONS = (1, 2, 4, 8)


def layer_shapes(ch: int = CH):
    """[(cin, cout, dilation, has_norm)] for the four blocks and the head."""
    shapes = []
    cin = 2
    for d in DILATIONS:
        shapes.append((cin, ch, d, True))
        cin = ch
    shapes.append((cin, 2, 1, False))
    return shapes


def param_layout(ch: int = CH):
    """Flat parameter order: per layer W (cout, cin, 3, 3), bias (cout), then gain (cout) if normed."""
    lay = []
    off = 0
    for cin, cout, d, norm in layer_shapes(ch):
        ent = {"cin": cin, "cout": cout, "dil": d, "norm": norm, "W": off}
        off += cout * cin * 9
        ent["b"] = off
        off += cout
        if norm:
            ent["g"] = off
            off += cout
        lay.append(ent)
    return lay, off


def unpack(theta: np.ndarray, ch: int = CH):
    lay, total = param_layout(ch)
    assert theta.size == total
    out = []
    for e in lay:
        W = theta[e["W"]:e["W"] + e["cout"] * e["cin"] * 9].reshape(e["cout"], e["cin"], 3, 3)
        b = theta[e["b"]:e["b"] + e["cout"]]
        g = theta[e["g"]:e["g"] + e["cout"]] if e["norm"] else None
        out.append((W, b, g, e["dil"]))
    return out


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray, d: int) -> np.ndarray:
    """Dilated 3x3 correlation with zero padding, by shifting the whole input per tap."""
    B, C, H, Wd = x.shape
    out = np.zeros((B, W.shape[0], H, Wd)) + b[None, :, None, None]
    for ty in range(3):
        for tx in range(3):
            oy, ox = (ty - 1) * d, (tx - 1) * d
            sh = np.zeros_like(x)
            ys, ye = max(0, -oy), min(H, H - oy)
            xs, xe = max(0, -ox), min(Wd, Wd - ox)
            if ys < ye and xs < xe:
                sh[:, :, ys:ye, xs:xe] = x[:, :, ys + oy:ye + oy, xs + ox:xe + ox]
            out += np.einsum("oc,bchw->bohw", W[:, :, ty, tx], sh)
    return out


def conv_backward(x: np.ndarray, W: np.ndarray, d: int, dout: np.ndarray):
    """Gradients of sum(dout * conv(x)) with respect to x, W and the bias."""
    B, C, H, Wd = x.shape
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for ty in range(3):
        for tx in range(3):
            oy, ox = (ty - 1) * d, (tx - 1) * d
            ys, ye = max(0, -oy), min(H, H - oy)
            xs, xe = max(0, -ox), min(Wd, Wd - ox)
            if not (ys < ye and xs < xe):
                continue
            xin = x[:, :, ys + oy:ye + oy, xs + ox:xe + ox]
            g = dout[:, :, ys:ye, xs:xe]
            dW[:, :, ty, tx] += np.einsum("bohw,bchw->oc", g, xin)
            dx[:, :, ys + oy:ye + oy, xs + ox:xe + ox] += np.einsum("oc,bohw->bchw", W[:, :, ty, tx], g)
    db = dout.sum(axis=(0, 2, 3))
    return dx, dW, db


def silu(t):
    return t / (1.0 + np.exp(-t))


def forward(theta: np.ndarray, x: np.ndarray, ch: int = CH):
    """Prediction y and the cache backward() needs."""
    cache = []
    h = x
    for W, b, g, d in unpack(theta, ch):
        z = conv(h, W, b, d)
        if g is None:
            cache.append((h, z, None, None))
            h = z
            continue
        r = np.sqrt(np.mean(z * z, axis=1, keepdims=True) + EPS)
        yn = g[None, :, None, None] * z / r
        cache.append((h, z, r, yn))
        h = silu(yn)
    return h, cache


def backward(theta: np.ndarray, cache, dy: np.ndarray, ch: int = CH):
    """Gradients of sum(dy * forward(theta, x)) with respect to theta and x."""
    layers = unpack(theta, ch)
    lay, total = param_layout(ch)
    grad = np.zeros(total)
    g_h = dy
    for li in range(len(layers) - 1, -1, -1):
        W, b, g, d = layers[li]
        h_in, z, r, yn = cache[li]
        e = lay[li]
        if g is not None:
            s = 1.0 / (1.0 + np.exp(-yn))
            dyn = g_h * (s + yn * s * (1.0 - s))
            xh = z / r
            grad[e["g"]:e["g"] + e["cout"]] = np.sum(dyn * xh, axis=(0, 2, 3))
            dxh = dyn * g[None, :, None, None]
            dz = (dxh - xh * np.mean(dxh * xh, axis=1, keepdims=True)) / r
        else:
            dz = g_h
        dx, dW, db = conv_backward(h_in, W, d, dz)
        grad[e["W"]:e["W"] + W.size] = dW.ravel()
        grad[e["b"]:e["b"] + b.size] = db
        g_h = dx
    return grad, g_h


def loss(y: np.ndarray, target: np.ndarray):
    """Gauge-invariant mean squared error and its gradient with respect to y."""
    B = y.shape[0]
    du = y[:, 0] - target[:, 0]
    dv = y[:, 1] - target[:, 1]
    t = np.mean(du - dv, axis=(1, 2), keepdims=True) / 2.0
    ru, rv = du - t, dv + t
    npix = y.shape[2] * y.shape[3]
    L = float(np.sum(ru * ru + rv * rv) / (2.0 * B * npix))
    gy = np.stack([ru, rv], axis=1) / (B * npix)
    return L, gy


def features(a: np.ndarray, b: np.ndarray, k: int) -> np.ndarray:
    """Network input for one pair of k x k images (masses in raster order, i = x + k y)."""
    m = k * k
    fa = np.log(np.maximum(a * (m / a.sum()), 1e-30)).reshape(k, k)
    fb = np.log(np.maximum(b * (m / b.sum()), 1e-30)).reshape(k, k)
    return np.stack([fa, fb])[None]


def init_params(seed: int, ch: int = CH) -> np.ndarray:
    """He-scaled normal weights from the seeded generator, zero biases, unit gains."""
    from paper_2206_11009_gb300.synth import normal
    lay, total = param_layout(ch)
    theta = np.zeros(total)
    z = normal(seed, total)
    for e in lay:
        n = e["cout"] * e["cin"] * 9
        theta[e["W"]:e["W"] + n] = z[e["W"]:e["W"] + n] * np.sqrt(2.0 / (e["cin"] * 9))
        if e["norm"]:
            theta[e["g"]:e["g"] + e["cout"]] = 1.0
    return theta
