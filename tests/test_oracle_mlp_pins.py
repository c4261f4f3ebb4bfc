"""Pins of the oracle's surrogate-network forward and backward pass: central
differences of the loss for sampled parameters of every block, and closed
forms of degenerate networks."""
import numpy as np
import pytest

import oracle

H = 128
OFF = {"W1": 0, "b1": 2 * H, "W2": 3 * H, "b2": 3 * H + H * H, "W3": 4 * H + H * H, "b3": 4 * H + 2 * H * H,
       "W4": 5 * H + 2 * H * H, "b4": 7 * H + 2 * H * H}


def _params(rng, scale=0.3):
    p = rng.normal(0, scale, oracle.mlp_nparams())
    p[OFF["W2"]:OFF["b2"]] /= np.sqrt(H)
    p[OFF["W3"]:OFF["b3"]] /= np.sqrt(H)
    p[OFF["W4"]:OFF["b4"]] /= np.sqrt(H)
    return p


def test_layout_size():
    assert oracle.mlp_nparams() == 2 * H + H + H * H + H + H * H + H + 2 * H + 2 == 33666


def test_output_bias_only_network():
    rng = np.random.default_rng(0)
    p = np.zeros(oracle.mlp_nparams())
    p[OFF["b4"]:OFF["b4"] + 2] = [0.25, -1.5]
    X = rng.uniform(-1, 1, (5, 2))
    assert np.allclose(oracle.mlp_forward(p, X), [[0.25, -1.5]] * 5, atol=0)


def test_single_path_closed_form():
    """One unit per layer carries the signal: y = w4 silu(w3 silu(w2 silu(w1 x)))."""
    p = np.zeros(oracle.mlp_nparams())
    p[OFF["W1"] + 0] = 0.7          # W1[0][0]
    p[OFF["W2"] + 0] = -1.1         # W2[0][0]
    p[OFF["W3"] + 0] = 0.9          # W3[0][0]
    p[OFF["W4"] + H + 0] = 2.0      # W4[1][0]
    silu = lambda v: v / (1 + np.exp(-v))
    for x0 in (-0.8, 0.3, 1.2):
        y = oracle.mlp_forward(p, [[x0, 0.4]])[0]
        assert y[0] == 0.0
        assert y[1] == pytest.approx(2.0 * silu(0.9 * silu(-1.1 * silu(0.7 * x0))), rel=1e-14)


def test_loss_gradient_vs_central_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    X = rng.uniform(-1, 1, (6, 2))
    T = rng.normal(0, 1, (6, 2))
    loss, g = oracle.mlp_loss_grad(p, X, T)
    assert loss == pytest.approx(np.mean(np.sum((oracle.mlp_forward(p, X) - T) ** 2, axis=1)), rel=1e-13)
    idx = []
    for name, off in OFF.items():
        size = {"W1": 2 * H, "b1": H, "W2": H * H, "b2": H, "W3": H * H, "b3": H, "W4": 2 * H, "b4": 2}[name]
        idx += list(off + rng.choice(size, min(6, size), replace=False))
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, X, T)[0] - oracle.mlp_loss_grad(pm, X, T)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i
