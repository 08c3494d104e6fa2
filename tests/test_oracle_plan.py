"""Pins for the oracle's FTK plan (operator SVD of J_l), against the values the
paper prints, the bounds it proves and properties the SVD must satisfy (no GPU)."""

import json
import math
import os

import numpy as np
import pytest
import scipy.special as sps

from oracle import svd_plan as sp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def plan_w1():
    return sp.build_plan(1.0, 1e-2, K=1.0)


def test_paper_worked_example_rank(plan_w1):
    g = json.load(open(os.path.join(GOLDEN, "paper_rank_W1_eps1e-2.json")))
    for l, h in g["H_l"].items():
        assert plan_w1.H_l(int(l)) == h
    assert plan_w1.H in (g["H_total"], g["H_total"] + 2)


def test_singular_values_symmetric_in_order(plan_w1):
    # J_{-l} = (-1)^l J_l, so the modal kernels for l and -l share singular values.
    for l in range(1, 6):
        a = sp.modal_svd(l, 1.0, 1e-2).sigma_all[:8]
        b = sp.modal_svd(-l, 1.0, 1e-2).sigma_all[:8]
        assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("W,eps", [(1.0, 1e-2), (1.5, 1e-3), (2.0, 1e-4)])
def test_rank_within_lemma1_and_theorem1_bounds(W, eps):
    plan = sp.build_plan(W, eps, K=1.0)
    for l in plan.modes:
        assert plan.H_l(l) <= sp.lemma1_bound(l, W, eps)
    assert plan.H <= 2.0 * sp.theorem1_calH(W, eps) ** 2


def test_empirical_rank_fit():
    g = json.load(open(os.path.join(GOLDEN, "paper_empirical_rank_fit.json")))
    for W, eps in g["cases"]:
        plan = sp.build_plan(W, eps, K=1.0)
        for l in range(0, 10):
            fit = 2.0 * (W - abs(l) / (2 * math.pi)) + 0.5 * math.log(1.0 / eps)
            if fit < 1:
                continue
            assert abs(plan.H_l(l) - fit) <= g["tolerance_terms"], (W, eps, l, plan.H_l(l), fit)


def _gl(nq, a, b):
    t, v = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (b - a) * (t + 1) + a, 0.5 * (b - a) * v


@pytest.mark.parametrize("l", [0, 2, 5])
def test_singular_functions_orthonormal(l):
    # eq. (Jsvd): U orthonormal for x dx on [0, 2 pi W], V for y dy on [0, 1];
    # checked with an independent Gauss-Legendre rule.
    W = 1.5
    m = sp.modal_svd(l, W, 1e-4)
    x, wx = _gl(200, 0.0, 2 * math.pi * W)
    y, wy = _gl(200, 0.0, 1.0)
    U, V = m.U(x), m.V(y)
    assert np.allclose((U * (wx * x)[:, None]).T @ U, np.eye(U.shape[1]), atol=1e-10)
    assert np.allclose((V * (wy * y)[:, None]).T @ V, np.eye(V.shape[1]), atol=1e-10)


@pytest.mark.parametrize("l", [0, 3])
def test_truncation_residual_equals_tail_singular_values(l):
    # eq. (EFl2)/(efrob): the weighted L2 residual of the rank-H_l expansion is
    # sum_{eta > H_l} Sigma_eta(l)^2, evaluated here by direct quadrature.
    W, eps = 1.0, 1e-3
    m = sp.modal_svd(l, W, eps)
    x, wx = _gl(160, 0.0, 2 * math.pi * W)
    y, wy = _gl(160, 0.0, 1.0)
    approx = (m.U(x) * m.sigma[None, :]) @ m.V(y).T
    resid = sps.jv(l, np.outer(x, y)) - approx
    E2 = float(np.einsum("a,b,ab->", wx * x, wy * y, resid ** 2))
    tail = float(np.sum(m.sigma_all[m.sigma.size:] ** 2))
    assert abs(E2 - tail) < 1e-8 + 1e-6 * tail


def test_svd_discretization_converged():
    # Remark r:svd: refining the polynomial projection changes nothing retained.
    a = sp.modal_svd(1, 2.0, 1e-4)
    b = sp.modal_svd(1, 2.0, 1e-4, nb=a.nb + 24, nq=a.nb + 60)
    assert a.sigma.size == b.sigma.size
    assert np.allclose(a.sigma, b.sigma, rtol=0, atol=1e-12)


def test_rank_grows_with_W_and_digits():
    h = {(W, e): sp.build_plan(W, e, K=1.0).H for W in (1.0, 2.0) for e in (1e-2, 1e-4)}
    assert h[(1.0, 1e-2)] < h[(2.0, 1e-2)] and h[(1.0, 1e-2)] < h[(1.0, 1e-4)]
