"""Pins for the proposal-network oracle: its backward pass against central finite
differences of its forward pass, and the rotation invariance of its features."""

import numpy as np
import pytest

from oracle import nn


def _setup(seed=0, B=3, M=8, Q=8, NT=5):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(B, M, 2 * Q)) + 1j * rng.normal(size=(B, M, 2 * Q))
    x0, lin = nn.features(a, 1e-3)
    p = nn.init_params(M, Q, NT, rng, ch=(4, 6, 6, 5), hidden=7)
    for k in p:
        if k.startswith(("b", "g")):
            p[k] = rng.normal(scale=0.1, size=p[k].shape)
    label = rng.integers(0, NT, B)
    target = rng.normal(size=(B, 2))
    return p, x0, lin, label, target, NT


def _loss(p, x0, lin, label, target, NT):
    out, _ = nn.forward(p, x0, lin)
    return nn.loss_and_grad_out(out, label, target, NT, 0.3)[0]


@pytest.mark.parametrize("name", ["w1", "b1", "w2", "b2", "w3", "b3", "w4", "b4", "f1", "g1", "f2", "g2"])
def test_backward_matches_finite_differences(name):
    p, x0, lin, label, target, NT = _setup()
    out, cache = nn.forward(p, x0, lin)
    _, dout = nn.loss_and_grad_out(out, label, target, NT, 0.3)
    g = nn.backward(p, cache, dout)[name]
    rng = np.random.default_rng(1)
    flat = p[name].reshape(-1)
    for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        h = 1e-6
        old = flat[idx]
        flat[idx] = old + h
        lp = _loss(p, x0, lin, label, target, NT)
        flat[idx] = old - h
        lm = _loss(p, x0, lin, label, target, NT)
        flat[idx] = old
        num = (lp - lm) / (2 * h)
        assert abs(num - g.reshape(-1)[idx]) < 1e-6 + 1e-5 * abs(num), (name, idx, num, g.reshape(-1)[idx])


def test_magnitude_features_are_rotation_invariant():
    # Section 3: a rotation by gamma multiplies a(k; q) by exp(-i q gamma).
    rng = np.random.default_rng(4)
    M, Q = 6, 12
    a = rng.normal(size=(2, M, 2 * Q)) + 1j * rng.normal(size=(2, M, 2 * Q))
    q = np.arange(2 * Q)
    q = np.where(q >= Q, q - 2 * Q, q)
    ar = a * np.exp(-1j * q * 0.7)[None, None, :]
    assert np.allclose(nn.features(a, 1e-3)[0], nn.features(ar, 1e-3)[0], atol=1e-12)
