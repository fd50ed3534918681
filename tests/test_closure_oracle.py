"""Pins of the FP64 closure oracle (the MLP of the learned closure): exact
gradients against central finite differences, closed forms of the loss and of
Adam's first step.  CPU only."""
import numpy as np
import pytest

from oracle import closure_oracle as CO
from paper_2303_07819_gb300 import inputs as I


def _data(rng, B=37):
    X = rng.normal(size=(B, 16)) * np.linspace(0.5, 3.0, 16) + np.arange(16)
    Y = rng.normal(size=(B, 4)) * np.array([1e-3, 2e-3, 1e-6, 5e-5]) + np.array([1e-3, 0, 0, 1e-4])
    return X, Y


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    X, Y = _data(rng)
    norm = CO.normalisation(X, Y)
    p = I.mlp_init(seed=5)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    loss, g = CO.loss_and_grads(p, X, Y, norm)
    h = 1e-6
    for k in CO.NAMES:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = CO.loss_and_grads(p, X, Y, norm)
            flat[idx] = old - h
            lm, _ = CO.loss_and_grads(p, X, Y, norm)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-4), (k, idx, fd, an)


def test_zero_network_loss_closed_form():
    rng = np.random.default_rng(1)
    X, Y = _data(rng)
    norm = CO.normalisation(X, Y)
    p = {k: np.zeros_like(v) for k, v in I.mlp_init().items()}
    loss, g = CO.loss_and_grads(p, X, Y, norm)
    yt = (Y - norm["mu_y"]) / norm["sd_y"]
    assert abs(loss - np.mean(yt ** 2)) < 1e-14
    # only the output bias sees a gradient: 2 mean(yh - yt) / 4 per output
    assert np.allclose(g["b4"], -2 * yt.sum(0) / (4 * X.shape[0]), atol=1e-15)
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    X, Y = _data(rng)
    norm = CO.normalisation(X, Y)
    p = I.mlp_init()
    p0 = {k: v.copy() for k, v in p.items()}
    _, g = CO.loss_and_grads(p, X, Y, norm)
    CO.adam_step(p, g, {}, lr=1e-3)
    for k in CO.NAMES:
        expect = p0[k] - 1e-3 * g[k] / (np.abs(g[k]) + 1e-8)
        assert np.allclose(p[k], expect, rtol=0, atol=1e-15), k


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(512, 16))
    Y = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], np.tanh(X[:, 3]), X[:, 4] ** 2], 1)
    norm = CO.normalisation(X, Y)
    p = I.mlp_init()
    st = {}
    l0, _ = CO.loss_and_grads(p, X, Y, norm)
    for _ in range(200):
        l, g = CO.loss_and_grads(p, X, Y, norm)
        CO.adam_step(p, g, st, lr=3e-3)
    assert l < 0.2 * l0
