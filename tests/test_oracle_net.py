"""Pins of the CPU oracle of the learned network: every analytic gradient
against central finite differences of the loss, closed forms for the loss at
zero weights, and the adjointness of im2col / col2im.  No GPU needed."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import net


def _batch(rng, B):
    x = rng.normal(0.0, 0.4, (B, 25))
    x[:, 12] += rng.uniform(0.5, 3.0, B)
    counts = rng.integers(0, 5, B)
    t = rng.uniform(-0.5, 0.5, (B, 2))
    mask = (rng.random(B) < 0.7).astype(np.float64)
    return x, counts, t, mask


def test_zero_weights_give_uniform_softmax():
    P = {k: np.zeros(s) for k, s in net.SHAPES.items()}
    x, counts, t, mask = _batch(np.random.default_rng(0), 16)
    loss, g, out = net.loss_and_grad(P, x, counts, t, mask, 10.0)
    assert np.all(out == 0.0)
    mse = ((t * mask[:, None]) ** 2).sum() / mask.sum()
    assert abs(loss - (np.log(5.0) + 10.0 * mse)) < 1e-12


def test_im2col_col2im_adjoint():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(3, 25, 4))
    g = rng.normal(size=(3, 25, 36))
    assert abs((net.im2col(a) * g).sum() - (a * net.col2im(g, 4)).sum()) < 1e-10
    # the centre column is the identity
    assert np.array_equal(net.im2col(a).reshape(3, 25, 9, 4)[:, :, 4, :], a)


@pytest.mark.parametrize("name", net.ORDER)
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(2)
    P = net.init_params(3)
    for k in net.ORDER:  # non-zero biases so every ReLU region is exercised
        if k.startswith("b"):
            P[k] = rng.normal(0, 0.1, P[k].shape)
    x, counts, t, mask = _batch(rng, 6)
    loss, g, _ = net.loss_and_grad(P, x, counts, t, mask, 10.0)
    flat = P[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
    h = 1e-6
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp, _, _ = net.loss_and_grad(P, x, counts, t, mask, 10.0)
        flat[i] = old - h
        lm, _, _ = net.loss_and_grad(P, x, counts, t, mask, 10.0)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        an = g[name].reshape(-1)[i]
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (name, i, fd, an)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2)
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5],
                 np.float32)
    r = net.bf16(v)
    # 1 + 2^-8 ties between 1 and 1 + 2^-7: to even -> 1;
    # 1 + 3*2^-8 ties between 1 + 2^-7 and 1 + 2^-6: to even -> 1 + 2^-6
    assert list(r) == [1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5]
