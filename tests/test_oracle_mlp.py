"""Pins of the FP64 closure-network reference (P-l): GELU against normal-CDF
values, backward pass against central finite differences, Adam's first step
and convergence on a problem with a known minimum."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_gelu_values():
    """The tanh form of GELU: exact identities (value 0 at 0, gelu(x) - gelu(-x) = x
    because tanh is odd, the limits x and 0), its distance from the erf form
    x Phi(x) (math.erf, independent of the tanh form; Phi(1) = 0.841344746068543
    from normal tables), and the derivative against central differences."""
    assert M.gelu(np.array([0.0]))[0] == 0.0
    xs = np.linspace(-6, 6, 241)
    assert np.allclose(M.gelu(xs) - M.gelu(-xs), xs, rtol=0, atol=1e-15)
    assert np.allclose(M.gelu(np.array([9.0, -9.0])), [9.0, 0.0], atol=1e-12)
    erf_form = np.array([0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0))) for x in xs])
    assert 0.5 * (1 + math.erf(1 / math.sqrt(2))) == pytest.approx(0.841344746068543, abs=1e-15)
    dev = np.abs(M.gelu(xs) - erf_form).max()
    print(f"max |tanh form - erf form| on [-6, 6]: {dev:.3e}")
    assert 1e-5 < dev < 5e-4
    h = 1e-6
    fd = (M.gelu(xs + h) - M.gelu(xs - h)) / (2 * h)
    assert np.allclose(fd, M.gelu_grad(xs), atol=1e-9)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    P = M.init_params(rng)
    X = rng.standard_normal((16, 17))
    T = rng.standard_normal(16)
    L, g = M.loss_and_grads(P, X, T)
    h = 1e-6
    for k in P:
        flat = P[k].ravel()
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            Lp, _ = M.loss_and_grads(P, X, T)
            flat[i] = old - h
            Lm, _ = M.loss_and_grads(P, X, T)
            flat[i] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].ravel()[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, i, fd, an)


def test_adam_first_step_and_convergence():
    P = {"w": np.array([3.0, -2.0])}
    st = M.adam_init(P)
    g = {"w": np.array([0.5, -4.0])}
    M.adam_step(P, g, st, lr=0.1)
    # bias-corrected first step moves each parameter by lr * sign(g)
    assert np.allclose(P["w"], [3.0 - 0.1, -2.0 + 0.1], atol=1e-8)
    # minimise |w - c|^2
    c = np.array([1.0, 2.0])
    for _ in range(3000):
        M.adam_step(P, {"w": 2 * (P["w"] - c)}, st, lr=0.01)
    assert np.allclose(P["w"], c, atol=1e-3)


def test_network_can_fit_a_smooth_map():
    """A few hundred Adam steps reduce the loss of a smooth 17 -> 1 map."""
    rng = np.random.default_rng(5)
    P = M.init_params(rng)
    X = rng.standard_normal((256, 17))
    T = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]
    st = M.adam_init(P)
    L0, _ = M.loss_and_grads(P, X, T)
    for _ in range(300):
        L, g = M.loss_and_grads(P, X, T)
        M.adam_step(P, g, st, lr=3e-3)
    assert L < 0.1 * L0
