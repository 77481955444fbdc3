"""Learned warm start: binding to the ot_cnn_* entry points, training and inference.

The network (see include/ot_ipm.h, "Warm-start network") maps log-masses of a k x k image pair
to predicted dual potentials (u, v) / k^2.  Training data are solutions the solver itself
produces (cold start, mixed precision), with the gauge fixed by sum(v) = 0.  All arithmetic runs
in the library's kernels; this module only moves arrays and calls the C ABI.

Command line (writes the parameters and a JSON record next to them):
    python -m paper_2206_11009_gb300.learn --out DIR [--instances N] [--steps S]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import time

import numpy as np

from . import _lib
from ._lib import OTError

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_cnn.f32")
CHANNELS = 32
TRAIN_SIZES = (32, 40, 48, 56, 64)     # image sides of the training set (32^2 .. 64^2)
TRAIN_SEED0 = 1000                     # training instances use seeds TRAIN_SEED0 + i


def features(a: np.ndarray, b: np.ndarray, k: int) -> np.ndarray:
    """(2, k, k) float32 input: log(a m / sum a), log(b m / sum b), raster order i = x + k y."""
    m = k * k
    fa = np.log(np.maximum(np.asarray(a, np.float64) * (m / np.sum(a)), 1e-30))
    fb = np.log(np.maximum(np.asarray(b, np.float64) * (m / np.sum(b)), 1e-30))
    return np.stack([fa.reshape(k, k), fb.reshape(k, k)]).astype(np.float32)


def targets(u: np.ndarray, v: np.ndarray, k: int) -> np.ndarray:
    """(2, k, k) float32 label: duals with sum(v) = 0, divided by k^2."""
    t = float(np.mean(v))
    return np.stack([(u + t).reshape(k, k), (v - t).reshape(k, k)]).astype(np.float32) / (k * k)


def init_params(seed: int) -> np.ndarray:
    """He-scaled normal weights (seeded generator), zero biases, unit gains: the reference's rule."""
    from .synth import normal
    lib = _lib.load()
    n = int(lib.ot_cnn_param_count(CHANNELS))
    theta = np.zeros(n)
    z = normal(seed, n)
    off, cin = 0, 2
    for layer in range(5):
        cout = CHANNELS if layer < 4 else 2
        w = cout * cin * 9
        theta[off:off + w] = z[off:off + w] * np.sqrt(2.0 / (cin * 9))
        off += w + cout
        if layer < 4:
            theta[off:off + cout] = 1.0
            off += cout
        cin = cout
    assert off == n
    return theta.astype(np.float32)


class WarmNet:
    """One network handle (device parameters and activations); inputs are torch CUDA tensors."""

    def __init__(self, params: np.ndarray, stream=None):
        import torch
        self._torch = torch
        self._lib = _lib.load()
        self.n = int(self._lib.ot_cnn_param_count(CHANNELS))
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != self.n:
            raise ValueError(f"expected {self.n} parameters, got {params.size}")
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else None)
        self._check(self._lib.ot_cnn_create(CHANNELS, params.ctypes.data_as(ctypes.c_void_p), st, ctypes.byref(h)))
        self.h = h
        self.grad = torch.zeros(self.n, device="cuda", dtype=torch.float32)
        self.steps = 0

    def _check(self, code):
        if code != 0:
            msg = self._lib.ot_cnn_last_error(getattr(self, "h", None))
            raise OTError(code, (msg or b"").decode())

    @classmethod
    def load(cls, path: str = WEIGHTS, stream=None) -> "WarmNet":
        return cls(np.fromfile(path, dtype="<f4"), stream)

    def params(self) -> np.ndarray:
        out = np.zeros(self.n, np.float32)
        self._check(self._lib.ot_cnn_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p), self.n))
        return out

    def save(self, path: str, record: dict | None = None):
        self.params().astype("<f4").tofile(path)
        if record is not None:
            with open(path + ".json", "w") as f:
                json.dump(record, f, indent=1)

    def forward(self, x):
        """x: (B, 2, k, k) float32 CUDA tensor -> prediction of the same shape."""
        torch = self._torch
        x = x.contiguous()
        B, _, k, _ = x.shape
        y = torch.empty_like(x)
        self._check(self._lib.ot_cnn_forward(self.h, B, k, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())))
        return y

    def loss_and_grad(self, x, target, dx=None):
        """Forward, gauge-invariant loss and the parameter gradient (self.grad); returns the loss."""
        torch = self._torch
        self.forward(x)
        dy = torch.empty_like(target)
        loss = ctypes.c_float(0.0)
        self._check(self._lib.ot_cnn_loss(self.h, ctypes.c_void_p(target.contiguous().data_ptr()),
                                          ctypes.c_void_p(dy.data_ptr()), ctypes.byref(loss)))
        self._check(self._lib.ot_cnn_backward(self.h, ctypes.c_void_p(dy.data_ptr()), ctypes.c_void_p(self.grad.data_ptr()),
                                              ctypes.c_void_p(dx.data_ptr()) if dx is not None else None))
        return float(loss.value)

    def backward(self, x, dy, dx=None):
        """Gradients of sum(dy * net(x)): parameters into self.grad, input into dx (optional)."""
        self.forward(x)
        self._check(self._lib.ot_cnn_backward(self.h, ctypes.c_void_p(dy.contiguous().data_ptr()),
                                              ctypes.c_void_p(self.grad.data_ptr()),
                                              ctypes.c_void_p(dx.data_ptr()) if dx is not None else None))
        return self.grad

    def adam(self, lr: float, betas=(0.9, 0.999), eps: float = 1e-8):
        self.steps += 1
        self._check(self._lib.ot_cnn_adam(self.h, ctypes.c_void_p(self.grad.data_ptr()), lr, betas[0], betas[1], eps,
                                          self.steps))

    def predict(self, a, b, k: int):
        """Predicted duals (u, v) in cost units for one k x k pair (host arrays)."""
        torch = self._torch
        x = torch.from_numpy(features(a, b, k)[None]).cuda()
        y = self.forward(x)[0].double().cpu().numpy() * (k * k)
        return y[0].ravel(), y[1].ravel()

    def close(self):
        if getattr(self, "h", None):
            self._lib.ot_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_dataset(count: int, sizes=TRAIN_SIZES, seed0: int = TRAIN_SEED0, verbose: bool = True):
    """Solve `count` seeded instances (cold start) and return {k: (X, Y)} float32 arrays."""
    from . import synth
    from .api import Solver
    data = {}
    t0 = time.time()
    for i in range(count):
        k = sizes[i % len(sizes)]
        inst = synth.image_pair(k, seed0 + i)
        with Solver(inst.a, inst.b, grid=(k, k)) as s:
            r = s.solve(raise_on_error=False)
            if r.status != 0:
                continue
            _, _, _, u, v = s.solution()
        X, Y = data.setdefault(k, ([], []))
        X.append(features(inst.a, inst.b, k))
        Y.append(targets(u, v, k))
        if verbose and (i + 1) % 50 == 0:
            print(f"  dataset {i + 1}/{count} ({time.time() - t0:.1f} s)", flush=True)
    return {k: (np.stack(X), np.stack(Y)) for k, (X, Y) in data.items()}


def train(net: WarmNet, data, steps: int, batch: int = 16, lr: float = 2e-3, seed: int = 0, verbose: bool = True):
    """Adam with a cosine learning-rate decay; each step draws one image size, then a batch."""
    import torch
    rng = np.random.default_rng(seed)
    dev = {k: (torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()) for k, (X, Y) in data.items()}
    ks = sorted(dev)
    hist = []
    for s in range(steps):
        k = ks[rng.integers(len(ks))]
        X, Y = dev[k]
        idx = torch.from_numpy(rng.choice(X.shape[0], size=min(batch, X.shape[0]), replace=False)).cuda()
        cur = lr * 0.5 * (1.0 + np.cos(np.pi * s / steps))
        loss = net.loss_and_grad(X[idx], Y[idx])
        net.adam(cur)
        hist.append(loss)
        if verbose and (s + 1) % max(1, steps // 10) == 0:
            print(f"  step {s + 1}/{steps} loss {np.mean(hist[-50:]):.3e}", flush=True)
    return hist


def evaluate(net: WarmNet, data):
    """Mean gauge-invariant loss per image size (no update)."""
    import torch
    out = {}
    for k, (X, Y) in data.items():
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        ls = []
        for i in range(0, X.shape[0], 16):
            ls.append(net.loss_and_grad(Xd[i:i + 16], Yd[i:i + 16]))
        out[k] = float(np.mean(ls))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--out", default=os.path.dirname(WEIGHTS))
    ap.add_argument("--instances", type=int, default=400)
    ap.add_argument("--holdout", type=int, default=40)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=7)
    args = ap.parse_args(argv)
    t0 = time.time()
    train_data = make_dataset(args.instances)
    hold = make_dataset(args.holdout, seed0=TRAIN_SEED0 + 100000)
    t1 = time.time()
    net = WarmNet(init_params(args.seed))
    before = evaluate(net, hold)
    hist = train(net, train_data, args.steps, args.batch, args.lr, args.seed)
    after = evaluate(net, hold)
    t2 = time.time()
    rec = {"channels": CHANNELS, "sizes": list(TRAIN_SIZES), "instances": args.instances, "holdout": args.holdout,
           "train_seed0": TRAIN_SEED0, "holdout_seed0": TRAIN_SEED0 + 100000, "steps": args.steps,
           "batch": args.batch, "lr": args.lr, "init_seed": args.seed, "final_train_loss": float(np.mean(hist[-100:])),
           "holdout_loss_before": before, "holdout_loss_after": after, "data_seconds": t1 - t0,
           "train_seconds": t2 - t1}
    os.makedirs(args.out, exist_ok=True)
    path = os.path.join(args.out, os.path.basename(WEIGHTS))
    net.save(path, rec)
    print(json.dumps(rec, indent=1))
    return rec


if __name__ == "__main__":
    main()
