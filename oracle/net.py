"""CPU oracle of the learned photon count / subpixel network — TEST
INFRASTRUCTURE (only tests, the smoke check and the benchmark's CPU baseline
may import it; it shares no code with the CUDA path).

The paper reports that deep-learning models it tried lost photon information
(abstract and section "Methods") and proposes its fixed filters as a starting
point for future learned models (section "Conclusions").  The network here is
that starting point: it refines the classical count and centre of mass of a
hit from the 5x5 neighbourhood of the seed.

Layers (all in float64 here; the GPU path rounds GEMM operands to bfloat16):
    x0  [B, 25]            5x5 patch of e / photon_kev, row-major (y, x)
    h1  = relu(conv3x3(x0; W1 [32, 9], b1))            [B, 25, 32]
    h2  = relu(conv3x3(h1; W2 [32, 9*32], b2))         [B, 25, 32]
    h3  = relu(flat(h2) [B, 800] @ W3.T + b3), W3 [64, 800]
    out = h3 @ W4.T + b4, W4 [7, 64]: logits = out[:, :5] (count 0..4),
          reg = out[:, 5:7] (dx, dy in pixel pitches)
Convolutions are 'same' with zero padding; the 3x3 offset k = 3*(dy+1) +
(dx+1), and the im2col column of conv2 is k*32 + c_in.
Loss (mean over the batch):
    L = mean_b CE(logits_b, n_b) + lam * sum_b m_b |reg_b - t_b|^2 / max(1, sum m)
where m_b = 1 for hits with a regression target.
"""
from __future__ import annotations

import numpy as np

NPOS, C1, C2, NH, NOUT = 25, 32, 32, 64, 7
SHAPES = {"W1": (C1, 9), "b1": (C1,), "W2": (C2, 9 * C1), "b2": (C2,),
          "W3": (NH, NPOS * C2), "b3": (NH,), "W4": (NOUT, NH), "b4": (NOUT,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]


def n_params() -> int:
    return int(sum(np.prod(SHAPES[k]) for k in ORDER))


def unflatten(flat):
    flat = np.asarray(flat, np.float64)
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = flat[o:o + n].reshape(SHAPES[k])
        o += n
    assert o == flat.size
    return out


def flatten(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k in ORDER])


def neighbour_table():
    """nb[p, k] = position of the neighbour of p at offset k, or -1 outside."""
    nb = -np.ones((NPOS, 9), np.int64)
    for p in range(NPOS):
        y, x = divmod(p, 5)
        for k in range(9):
            dy, dx = k // 3 - 1, k % 3 - 1
            if 0 <= y + dy < 5 and 0 <= x + dx < 5:
                nb[p, k] = (y + dy) * 5 + (x + dx)
    return nb


NB = neighbour_table()


def im2col(a):
    """a [B, 25, C] -> [B, 25, 9*C] with column k*C + c (zero outside)."""
    B, _, C = a.shape
    out = np.zeros((B, NPOS, 9, C))
    for p in range(NPOS):
        for k in range(9):
            q = NB[p, k]
            if q >= 0:
                out[:, p, k, :] = a[:, q, :]
    return out.reshape(B, NPOS, 9 * C)


def col2im(g, C):
    """Adjoint of im2col: g [B, 25, 9*C] -> [B, 25, C]."""
    B = g.shape[0]
    g = g.reshape(B, NPOS, 9, C)
    out = np.zeros((B, NPOS, C))
    for p in range(NPOS):
        for k in range(9):
            q = NB[p, k]
            if q >= 0:
                out[:, q, :] += g[:, p, k, :]
    return out


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, x0, operand=None):
    """operand: optional rounding applied to both operands of every
    contraction (e.g. bf16, to mirror tensor-core inputs)."""
    r = operand if operand is not None else (lambda a: a)
    P = params
    x0 = np.asarray(x0, np.float64).reshape(-1, NPOS, 1)
    X1 = im2col(x0)                                   # [B, 25, 9]
    z1 = r(X1) @ r(P["W1"]).T + P["b1"]
    h1 = relu(z1)
    X2 = im2col(h1)                                   # [B, 25, 288]
    z2 = r(X2) @ r(P["W2"]).T + P["b2"]
    h2 = relu(z2)
    f = h2.reshape(h2.shape[0], NPOS * C2)            # column p*32 + c
    z3 = r(f) @ r(P["W3"]).T + P["b3"]
    h3 = relu(z3)
    out = r(h3) @ r(P["W4"]).T + P["b4"]
    cache = dict(X1=X1, z1=z1, h1=h1, X2=X2, z2=z2, h2=h2, f=f, z3=z3, h3=h3)
    return out, cache


def loss_and_dout(out, counts, targets, mask, lam):
    """Softmax cross-entropy on out[:, :5] plus masked squared error on
    out[:, 5:7]; returns (loss, dL/dout)."""
    B = out.shape[0]
    logits = out[:, :5]
    mx = logits.max(axis=1, keepdims=True)
    ex = np.exp(logits - mx)
    sm = ex / ex.sum(axis=1, keepdims=True)
    counts = np.asarray(counts, np.int64)
    ce = -np.log(sm[np.arange(B), counts]).mean()
    d = np.zeros_like(out)
    d[:, :5] = sm
    d[np.arange(B), counts] -= 1.0
    d[:, :5] /= B
    mask = np.asarray(mask, np.float64).reshape(-1)
    nreg = max(1.0, mask.sum())
    diff = (out[:, 5:7] - np.asarray(targets, np.float64)) * mask[:, None]
    mse = (diff ** 2).sum() / nreg
    d[:, 5:7] = 2.0 * lam * diff / nreg
    return ce + lam * mse, d


def backward(params, cache, dout, operand=None):
    """operand: optional rounding of both operands of every contraction."""
    r = operand if operand is not None else (lambda a: a)
    P = params
    g = {}
    B = dout.shape[0]
    g["W4"] = r(dout).T @ r(cache["h3"])
    g["b4"] = dout.sum(axis=0)
    dh3 = r(dout) @ r(P["W4"])
    dz3 = dh3 * (cache["z3"] > 0)
    g["W3"] = r(dz3).T @ r(cache["f"])
    g["b3"] = dz3.sum(axis=0)
    df = r(dz3) @ r(P["W3"])
    dz2 = df.reshape(B, NPOS, C2) * (cache["z2"] > 0)
    g["W2"] = r(dz2.reshape(-1, C2)).T @ r(cache["X2"].reshape(-1, 9 * C1))
    g["b2"] = dz2.sum(axis=(0, 1))
    dX2 = r(dz2) @ r(P["W2"])                          # [B, 25, 288]
    dh1 = col2im(dX2, C1)
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = r(dz1.reshape(-1, C1)).T @ r(cache["X1"].reshape(-1, 9))
    g["b1"] = dz1.sum(axis=(0, 1))
    return g


def loss_and_grad(params, x0, counts, targets, mask, lam, operand=None):
    out, cache = forward(params, x0, operand)
    loss, dout = loss_and_dout(out, counts, targets, mask, lam)
    return loss, backward(params, cache, dout, operand), out


def init_params(seed: int = 0):
    """Weights and biases uniform in +-1/sqrt(fan_in) (float64)."""
    rng = np.random.default_rng(seed)
    P = {}
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4")):
        bound = 1.0 / np.sqrt(SHAPES[w][1])
        P[w] = rng.uniform(-bound, bound, SHAPES[w])
        P[b] = rng.uniform(-bound, bound, SHAPES[b])
    return P


def bf16(x):
    """Round float64/float32 values to bfloat16 (ties to even), as float64."""
    a = np.asarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
