"""FP64 reference of the learned J-closure network: a 17 -> 128 -> 128 -> 1
multilayer perceptron with the tanh form of GELU (Hendrycks & Gimpel,
"Gaussian Error Linear Units", 2016), its backward pass for a mean-squared-
error loss and the Adam update.

TEST INFRASTRUCTURE ONLY (imported by tests, the smoke check and the CPU
baseline; never by the product library).

The closure is not in the paper: it stands in for the Sec. 5.2 velocity-space
solve (the f_1x update and the Jx moment) with a network fed by a cell's
recent E history and its density.  Layout: row-major weights W1 [17,128],
W2 [128,128], W3 [128,1]; a batch is X [B,17].
"""
from __future__ import annotations

import math

import numpy as np

GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(x):
    """0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), the tanh form of x Phi(x)."""
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + GELU_A * x ** 3)))


def gelu_grad(x):
    """Derivative of the tanh form: 0.5 (1 + t) + 0.5 x (1 - t^2) sqrt(2/pi) (1 + 3 * 0.044715 x^2)."""
    t = np.tanh(GELU_C * (x + GELU_A * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * x * x)


def init_params(rng: np.random.Generator, n_in=17, n_h=128):
    """He-style init in FP64."""
    return dict(
        W1=rng.standard_normal((n_in, n_h)) * math.sqrt(2.0 / n_in), b1=np.zeros(n_h),
        W2=rng.standard_normal((n_h, n_h)) * math.sqrt(2.0 / n_h), b2=np.zeros(n_h),
        W3=rng.standard_normal((n_h, 1)) * math.sqrt(1.0 / n_h), b3=np.zeros(1),
    )


def forward(P, X):
    """Returns y [B] and the cache the backward pass needs."""
    z1 = X @ P["W1"] + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"] + P["b2"]
    h2 = gelu(z2)
    y = (h2 @ P["W3"] + P["b3"])[:, 0]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(P, X, T):
    """L = mean_b (y_b - t_b)^2 and dL/dP by the chain rule."""
    y, (X, z1, h1, z2, h2) = forward(P, X)
    B = X.shape[0]
    r = y - T
    L = float(np.mean(r * r))
    dy = (2.0 / B) * r[:, None]                      # [B,1]
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = dy.sum(0)
    dz2 = (dy @ P["W3"].T) * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"].T) * gelu_grad(z1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return L, g


def adam_init(P):
    return dict(t=0, m={k: np.zeros_like(v) for k, v in P.items()}, v={k: np.zeros_like(v) for k, v in P.items()})


def adam_step(P, g, st, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Kingma & Ba (2015) Adam with bias correction; updates P in place."""
    st["t"] += 1
    t = st["t"]
    for k in P:
        st["m"][k] = b1 * st["m"][k] + (1 - b1) * g[k]
        st["v"][k] = b2 * st["v"][k] + (1 - b2) * g[k] * g[k]
        mh = st["m"][k] / (1 - b1 ** t)
        vh = st["v"][k] / (1 - b2 ** t)
        P[k] -= lr * mh / (np.sqrt(vh) + eps)
    return P
