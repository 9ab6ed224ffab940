"""FP64 oracle of the warm-start CNN (forward, MSE loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY: the plain restatement the CUDA network kernels
are checked against; nothing in the product imports it.

Network: six 3x3 convolutions with zero padding ("same"), channels
1 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU after the first five, residual
output u0 = f + conv6(...).  A convolution is the cross-correlation
y[p, o] = b[o] + sum_{tap, i} x[p + tap, i] w[tap, i, o], tap = (dy + 1) * 3 +
(dx + 1) over dy, dx in {-1, 0, 1}.  Loss: mean over pixels of (u0 - u*)^2.

Parameter layout (one flat FP32 vector, the order the C ABI uses):
  W1 [9, 32] (tap, out), b1 [32];
  W2..W5 [9, 32, 32] (tap, in, out), b2..b5 [32];
  W6 [9, 32] (tap, in), b6 [1].
"""
from __future__ import annotations

import numpy as np

C = 32
SHAPES = [("W1", (9, C)), ("b1", (C,))]
for _l in range(2, 6):
    SHAPES += [(f"W{_l}", (9, C, C)), (f"b{_l}", (C,))]
SHAPES += [("W6", (9, C)), ("b6", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape)
        off += n
    return out


def pack(params):
    return np.concatenate([np.asarray(params[name], np.float64).ravel() for name, _ in SHAPES])


def _shifts(x):
    """x: (N, H, W, Ci) -> (N, H, W, 9, Ci): x[p + tap] with zero padding."""
    N, H, W, Ci = x.shape
    xp = np.zeros((N, H + 2, W + 2, Ci))
    xp[:, 1:-1, 1:-1] = x
    cols = [xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return np.stack(cols, axis=3)


def conv(x, w, b):
    """x (N,H,W,Ci), w (9,Ci,Co), b (Co,) -> (N,H,W,Co): im2col then a matmul."""
    X = _shifts(x)                                   # N,H,W,9,Ci
    N, H, W = x.shape[:3]
    y = X.reshape(N * H * W, -1) @ w.reshape(-1, w.shape[-1])
    return y.reshape(N, H, W, -1) + b


def forward(params, f):
    """f (N,H,W) -> (u0, cache)."""
    p = params if isinstance(params, dict) else unpack(params)
    x0 = np.asarray(f, np.float64)[..., None]
    acts = [x0]
    z = conv(x0, p["W1"][:, None, :], p["b1"])
    a = np.maximum(z, 0)
    acts.append(a)
    for l in range(2, 6):
        z = conv(a, p[f"W{l}"], p[f"b{l}"])
        a = np.maximum(z, 0)
        acts.append(a)
    out = conv(a, p["W6"][:, :, None], p["b6"])[..., 0]
    u0 = x0[..., 0] + out
    return u0, acts


def loss(params, f, ustar):
    u0, _ = forward(params, f)
    return float(np.mean((u0 - np.asarray(ustar, np.float64)) ** 2))


def _conv_grads(x, w, dy):
    """Gradients of y = conv(x, w, b) given dy: (dx, dw, db)."""
    N, H, W, Ci = x.shape
    Co = w.shape[-1]
    X = _shifts(x).reshape(N * H * W, 9 * Ci)
    G = dy.reshape(N * H * W, Co)
    dw = (X.T @ G).reshape(9, Ci, Co)
    db = G.sum(axis=0)
    # dx[p, i] = sum_{tap, o} dy[p - tap, o] w[tap, i, o]
    dX = (G @ w.reshape(9 * Ci, Co).T).reshape(N, H, W, 9, Ci)
    dx = np.zeros((N, H + 2, W + 2, Ci))
    t = 0
    for ddy in (-1, 0, 1):
        for ddx in (-1, 0, 1):
            dx[:, 1 + ddy:1 + ddy + H, 1 + ddx:1 + ddx + W] += dX[:, :, :, t]
            t += 1
    return dx[:, 1:-1, 1:-1], dw, db


def gradients(params, f, ustar):
    """Returns (loss, flat gradient) of the mean squared error."""
    p = params if isinstance(params, dict) else unpack(params)
    u0, acts = forward(p, f)
    n = u0.size
    d = 2.0 * (u0 - np.asarray(ustar, np.float64)) / n      # dL/dout
    g = {}
    dx, dw, db = _conv_grads(acts[5], p["W6"][:, :, None], d[..., None])
    g["W6"], g["b6"] = dw[:, :, 0], db
    dz = dx * (acts[5] > 0)
    for l in range(5, 1, -1):
        dx, dw, db = _conv_grads(acts[l - 1], p[f"W{l}"], dz)
        g[f"W{l}"], g[f"b{l}"] = dw, db
        dz = dx * (acts[l - 1] > 0)
    _, dw, db = _conv_grads(acts[0], p["W1"][:, None, :], dz)
    g["W1"], g["b1"] = dw[:, 0, :], db
    return float(np.mean((u0 - ustar) ** 2)), pack(g)


def adam_step(theta, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction; t >= 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int, zero_last: bool = True):
    """He-normal weights for the ReLU layers (std sqrt(2 / fan_in)), zero
    biases; the last layer zero so that the untrained network returns f."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(2 / 9), (9, C)), "b1": np.zeros(C)}
    for l in range(2, 6):
        p[f"W{l}"] = rng.normal(0, np.sqrt(2 / (9 * C)), (9, C, C))
        p[f"b{l}"] = np.zeros(C)
    p["W6"] = np.zeros((9, C)) if zero_last else rng.normal(0, np.sqrt(1 / (9 * C)), (9, C))
    p["b6"] = np.zeros(1)
    return pack(p)
