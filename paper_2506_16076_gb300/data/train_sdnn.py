"""Train the stand-in smoothness classifier (SDNN) and write sdnn_standin.txt.

The paper classifies the smoothness of the proxy Phi with a pre-trained neural
network whose weights are loaded from disc at initialisation (Sec. 5.1); the
network, its inputs and its weights are described in an earlier paper and are
not reproduced. This script trains a stand-in with the same role:

  input : 7 consecutive proxy values along one grid direction, shifted to
          minimum 0 and scaled to range 1;
  output: 4 logits; class = argmax + 1 in {1: jump, 2: kink, 3: curvature
          jump, 4: smooth}, which the viscosity weight R maps to 1.5/1/0.5/0.
  net   : ReLU MLP 7 -> 16 -> 16 -> 4, evaluated in FP32.

Training data are seeded synthetic windows: smooth backgrounds (low-degree
polynomials plus a resolved sinusoid) with, for classes 1-3, a step, a kink
(|x - x0|) or a curvature jump (max(x - x0, 0)^2) at a random non-grid
location inside the window. Plain numpy Adam on softmax cross-entropy.
Run: python train_sdnn.py   (a few seconds; numpy only)
"""
import os

import numpy as np

SEED = 20250616
H1, H2 = 16, 16


def windows(rng, n):
    x = np.arange(-3, 4, dtype=float)[None, :]
    cls = rng.integers(0, 4, n)
    a = rng.normal(0, 1, (n, 1))
    b = rng.normal(0, 0.3, (n, 1))
    c = rng.normal(0, 0.05, (n, 1))
    om = rng.uniform(0.0, 0.6, (n, 1))
    ph = rng.uniform(0, 2 * np.pi, (n, 1))
    amp_s = rng.uniform(0, 0.3, (n, 1))
    f = a + b * x + c * x * x + amp_s * np.sin(om * x + ph)
    x0 = rng.uniform(-2.5, 2.5, (n, 1))
    A = rng.choice([-1.0, 1.0], (n, 1)) * rng.uniform(1.0, 4.0, (n, 1))
    step = (x > x0).astype(float)
    kink = np.abs(x - x0)
    curv = np.maximum(x - x0, 0.0) ** 2
    f = f + A * np.where(cls[:, None] == 0, step, 0.0)
    f = f + 0.6 * A * np.where(cls[:, None] == 1, kink, 0.0)
    f = f + 0.25 * A * np.where(cls[:, None] == 2, curv, 0.0)
    lo = f.min(axis=1, keepdims=True)
    rg = f.max(axis=1, keepdims=True) - lo
    return ((f - lo) / np.maximum(rg, 1e-300)), cls


def train():
    rng = np.random.default_rng(SEED)
    X, y = windows(rng, 200000)
    W1 = rng.normal(0, np.sqrt(2 / 7), (H1, 7)); b1 = np.zeros(H1)
    W2 = rng.normal(0, np.sqrt(2 / H1), (H2, H1)); b2 = np.zeros(H2)
    W3 = rng.normal(0, np.sqrt(2 / H2), (4, H2)); b3 = np.zeros(4)
    params = [W1, b1, W2, b2, W3, b3]
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    lr, B1, B2 = 3e-3, 0.9, 0.999
    for it in range(1, 6001):
        idx = rng.integers(0, len(X), 1024)
        xb, yb = X[idx], y[idx]
        z1 = xb @ W1.T + b1; h1 = np.maximum(z1, 0)
        z2 = h1 @ W2.T + b2; h2 = np.maximum(z2, 0)
        o = h2 @ W3.T + b3
        o -= o.max(axis=1, keepdims=True)
        pr = np.exp(o); pr /= pr.sum(axis=1, keepdims=True)
        g = pr.copy(); g[np.arange(len(yb)), yb] -= 1; g /= len(yb)
        gW3 = g.T @ h2; gb3 = g.sum(0)
        gh2 = g @ W3 * (z2 > 0)
        gW2 = gh2.T @ h1; gb2 = gh2.sum(0)
        gh1 = gh2 @ W2 * (z1 > 0)
        gW1 = gh1.T @ xb; gb1 = gh1.sum(0)
        grads = [gW1, gb1, gW2, gb2, gW3, gb3]
        if it == 4000:
            lr *= 0.3
        for k, (p, gr) in enumerate(zip(params, grads)):
            m[k] = B1 * m[k] + (1 - B1) * gr
            v[k] = B2 * v[k] + (1 - B2) * gr * gr
            p -= lr * (m[k] / (1 - B1 ** it)) / (np.sqrt(v[k] / (1 - B2 ** it)) + 1e-8)
    Xt, yt = windows(np.random.default_rng(SEED + 1), 20000)
    h = np.maximum(Xt @ W1.T + b1, 0); h = np.maximum(h @ W2.T + b2, 0)
    acc = float(((h @ W3.T + b3).argmax(1) == yt).mean())
    return [p.astype(np.float32) for p in params], acc


def main():
    params, acc = train()
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "sdnn_standin.txt"), "w") as f:
        f.write(f"# SDNN stand-in, ReLU MLP 7-16-16-4, FP32 values; seed {SEED}; held-out accuracy {acc:.4f}\n")
        for n, p in zip(names, params):
            shape = p.shape if p.ndim == 2 else (p.shape[0], 1)
            f.write(f"{n} {shape[0]} {shape[1]}\n")
            for row in p.reshape(shape):
                f.write(" ".join(repr(float(v)) for v in row) + "\n")
    print("held-out accuracy", acc)


if __name__ == "__main__":
    main()
