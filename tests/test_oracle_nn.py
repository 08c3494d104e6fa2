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


def test_adam_first_step_moves_by_lr_times_sign():
    # with m = v = 0, the bias-corrected first step is lr * g / (|g| + eps)
    rng = np.random.default_rng(5)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    p1, m, v = nn.adam(p0, g, np.zeros(50), np.zeros(50), 1, 1e-2, 0.9, 0.999, 1e-12)
    assert np.allclose(p1, p0 - 1e-2 * np.sign(g), atol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_keeps_unit_steps():
    # a constant gradient keeps mhat = g and vhat = g^2 at every step
    p, m, v = np.array([1.0, -2.0]), np.zeros(2), np.zeros(2)
    g = np.array([0.3, -4.0])
    for t in range(1, 6):
        p_old = p
        p, m, v = nn.adam(p, g, m, v, t, 0.5, 0.8, 0.9, 0.0)
        assert np.allclose(p_old - p, 0.5 * np.sign(g), atol=1e-12)


def test_topk_and_confidence_on_hand_examples():
    x = np.array([[0.0, 3.0, 1.0, 3.0, -1.0], [5.0, 5.0, 5.0, 5.0, 5.0]])
    assert nn.topk(x, 3).tolist() == [[1, 3, 2], [0, 1, 2]]
    c = nn.confidence(x)
    assert abs(c[1] - 0.2) < 1e-15
    e = np.exp([0.0, 3.0, 1.0, 3.0, -1.0])
    assert abs(c[0] - e[1] / e.sum()) < 1e-15
    m = nn.confidence(x, [[1, 3], [4, 0]])
    assert abs(m[0] - 2 * e[1] / e.sum()) < 1e-15 and abs(m[1] - 0.4) < 1e-15
    assert abs(nn.confidence(x, [[0, 1, 2, 3, 4], [0, 1, 2, 3, 4]])[0] - 1.0) < 1e-15


def _eq_setup(seed=7, B=3, M=5, two_Q=24, NT=4, Mh=3, Qh=5):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(B, M, two_Q)) + 1j * rng.normal(size=(B, M, two_Q))
    W = rng.normal(size=(NT, Mh, 2 * Qh + 1)) + 1j * rng.normal(size=(NT, Mh, 2 * Qh + 1))
    beta = rng.normal(size=NT)
    g = rng.normal(size=(B, NT))
    return a, W, beta, g, Mh, Qh


def test_eqhead_backward_matches_finite_differences():
    a, W, beta, g, Mh, Qh = _eq_setup()
    f = lambda W_, b_: float(np.sum(g * nn.eqhead_forward(W_, b_, a, 0.7)[0]))  # noqa: E731
    logits, rstar = nn.eqhead_forward(W, beta, a, 0.7)
    dW, db = nn.eqhead_backward(a, rstar, g, 0.7, Mh, Qh)
    h = 1e-6
    rng = np.random.default_rng(2)
    for _ in range(8):
        idx = tuple(rng.integers(0, s) for s in W.shape)
        for unit, part in ((1.0, dW[idx].real), (1j, dW[idx].imag)):
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += unit * h
            Wm[idx] -= unit * h
            num = (f(Wp, beta) - f(Wm, beta)) / (2 * h)
            assert abs(num - part) < 1e-6 + 1e-6 * abs(num), (idx, unit, num, part)
    assert np.allclose(db, g.sum(axis=0))


def test_eqhead_recovers_grid_rotation_of_a_template():
    # image = template rotated by a grid angle: with W = conj(template) the maximum sits at the
    # rotation that undoes it and equals sum |b|^2 over the band
    rng = np.random.default_rng(9)
    M, two_Q, Mh, Qh = 4, 32, 3, 6
    b = rng.normal(size=(1, M, two_Q)) + 1j * rng.normal(size=(1, M, two_Q))
    q = np.arange(two_Q)
    q = np.where(q >= two_Q // 2, q - two_Q, q)
    for r0 in (0, 5, 17):
        gam0 = 2 * np.pi * r0 / two_Q
        a = b * np.exp(-1j * q * gam0)[None, None, :]
        qq = np.arange(-Qh, Qh + 1)
        W = np.conj(b[:, :Mh, qq % two_Q])
        logits, rstar = nn.eqhead_forward(W, np.zeros(1), a, 1.0)
        assert abs(logits[0, 0] - np.sum(np.abs(W) ** 2)) < 1e-9
        assert rstar[0, 0] == (-r0) % two_Q


def test_shared_spectral_weight_gradient_matches_finite_differences():
    # logits through W = rho W0 (one real weight per ring and angular frequency, shared by
    # all templates): d/d rho by the chain rule against central differences of the forward
    a, W0, beta, g, Mh, Qh = _eq_setup()
    rng = np.random.default_rng(4)
    rho = rng.uniform(0.5, 1.5, size=W0.shape[1:])
    f = lambda r_: float(np.sum(g * nn.eqhead_forward(nn.scale_filters(W0, r_), beta, a, 0.7)[0]))  # noqa: E731
    W = nn.scale_filters(W0, rho)
    assert np.allclose(W[3], rho * W0[3])
    _, rstar = nn.eqhead_forward(W, beta, a, 0.7)
    dW, _ = nn.eqhead_backward(a, rstar, g, 0.7, Mh, Qh)
    drho = nn.scale_filters_backward(W0, dW)
    h = 1e-6
    for _ in range(8):
        idx = tuple(rng.integers(0, s) for s in rho.shape)
        rp, rm = rho.copy(), rho.copy()
        rp[idx] += h
        rm[idx] -= h
        num = (f(rp) - f(rm)) / (2 * h)
        assert abs(num - drho[idx]) < 1e-6 + 1e-6 * abs(num), (idx, num, drho[idx])
