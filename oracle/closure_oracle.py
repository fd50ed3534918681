"""FP64 NumPy oracle of the learned closure (a small MLP), the part the
particle-continuum method gains from a learned model of the bulk feedback.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs).  Shares
no code with the CUDA closure kernels.

Network (the definition both sides implement):
    xh = (x - mu_x) / sd_x                         16 cell features, z-scored
    h1 = tanh(W1 xh + b1)                          128
    h2 = tanh(W2 h1 + b2)                          128
    h3 = tanh(W3 h2 + b3)                          128
    yh = W4 h3 + b4                                4 outputs, in z-scored units
    y  = mu_y + sd_y * yh
Loss on a batch of B samples: L = sum((yh - (y_t - mu_y)/sd_y)^2) / (4 B).
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
      p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
Weights are W[out][in] (row = output unit).
"""
from __future__ import annotations

import numpy as np

LAYERS = [(16, 128), (128, 128), (128, 128), (128, 4)]
NAMES = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]


def forward(p: dict, X: np.ndarray, norm: dict, keep: bool = False):
    """X: [B, 16] raw features.  Returns yh [B, 4] (z-scored), and the
    activations when keep."""
    xh = (X - norm["mu_x"]) / norm["sd_x"]
    h1 = np.tanh(xh @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    yh = h3 @ p["W4"].T + p["b4"]
    if keep:
        return yh, (xh, h1, h2, h3)
    return yh


def predict(p: dict, X: np.ndarray, norm: dict) -> np.ndarray:
    return norm["mu_y"] + norm["sd_y"] * forward(p, X, norm)


def loss_and_grads(p: dict, X: np.ndarray, Y: np.ndarray, norm: dict):
    """Mean-squared error in z-scored output units and its exact gradient by
    the chain rule, layer by layer."""
    B = X.shape[0]
    yh, (xh, h1, h2, h3) = forward(p, X, norm, keep=True)
    yt = (Y - norm["mu_y"]) / norm["sd_y"]
    r = yh - yt
    loss = float(np.sum(r * r) / (4 * B))
    dy = 2.0 * r / (4 * B)                      # dL/dyh
    g = {}
    g["W4"] = dy.T @ h3
    g["b4"] = dy.sum(0)
    dz3 = (dy @ p["W4"]) * (1.0 - h3 * h3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ xh
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_step(p: dict, g: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def normalisation(X: np.ndarray, Y: np.ndarray, floor: float = 1e-12) -> dict:
    return {"mu_x": X.mean(0), "sd_x": np.maximum(X.std(0), floor),
            "mu_y": Y.mean(0), "sd_y": np.maximum(Y.std(0), floor)}
