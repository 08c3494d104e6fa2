"""Pins for the spectrally weighted plan (Section 4.5, the remark on alternative weight
functions after Remark r:svd): the modal SVD taken in the norm rho(y) y dy over the
frequency disk, rho(y) = exp(-beta y^2) normalized to unit mean. Checked against what the
weighted SVD must satisfy (independent quadrature, Eckart-Young optimality, the beta -> 0
limit) and against the remark's claim on images of known spectral decay (no GPU)."""

import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sps

from oracle import brute, ftk_steps, quadrature as quad, svd_plan as sp, transform as tr
from workloads import make_workload

DECAY = 10.0   # (pi sigma)^2 for blobs of sigma = 1 px: their power spectrum falls at least this fast


def _gl(nq, a, b):
    t, v = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (b - a) * (t + 1) + a, 0.5 * (b - a) * v


def _weighted_error2(m, h, W, decay, nq=160):
    """int int (J_l(x y) - sum_{eta < h} U Sigma V)^2 x rho(y) y dx dy by Gauss-Legendre."""
    x, wx = _gl(nq, 0.0, 2 * math.pi * W)
    y, wy = _gl(nq, 0.0, 1.0)
    approx = (m.U(x)[:, :h] * m.sigma[None, :h]) @ m.V(y)[:, :h].T
    resid = sps.jv(m.l, np.outer(x, y)) - approx
    rho = sp.spectral_weight(y, decay)
    return float(np.einsum("a,b,ab->", wx * x, wy * y * rho, resid ** 2))


@pytest.mark.parametrize("decay", [0.5, DECAY, 40.0])
def test_weight_has_unit_mean_over_the_disk(decay):
    val, _ = si.quad(lambda y: float(sp.spectral_weight(np.array([y]), decay)[0]) * y, 0.0, 1.0,
                     epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 0.5) < 1e-12
    assert sp.spectral_weight(np.array([0.3]), decay)[0] / sp.spectral_weight(np.array([0.0]), decay)[0] == \
        pytest.approx(math.exp(-decay * 0.09), rel=1e-13)


@pytest.mark.parametrize("l", [0, 2, 5])
def test_weighted_singular_functions_orthonormal(l):
    # U orthonormal for x dx; V orthonormal for rho(y) y dy (not for y dy)
    W = 1.0
    m = sp.modal_svd(l, W, 1e-4, decay=DECAY)
    x, wx = _gl(200, 0.0, 2 * math.pi * W)
    y, wy = _gl(200, 0.0, 1.0)
    U, V = m.U(x), m.V(y)
    rho = sp.spectral_weight(y, DECAY)
    assert np.allclose((U * (wx * x)[:, None]).T @ U, np.eye(U.shape[1]), atol=1e-10)
    assert np.allclose((V * (wy * y * rho)[:, None]).T @ V, np.eye(V.shape[1]), atol=1e-9)
    plain = (V * (wy * y)[:, None]).T @ V
    assert not np.allclose(plain, np.eye(V.shape[1]), atol=1e-3)


@pytest.mark.parametrize("l", [0, 3])
def test_weighted_truncation_residual_equals_tail_singular_values(l):
    # U Sigma V reconstructs J_l itself; its rho-weighted L2 residual is the tail sum of Sigma^2
    W, eps = 1.0, 1e-3
    m = sp.modal_svd(l, W, eps, decay=DECAY)
    E2 = _weighted_error2(m, m.sigma.size, W, DECAY)
    tail = float(np.sum(m.sigma_all[m.sigma.size:] ** 2))
    assert abs(E2 - tail) < 1e-8 + 1e-6 * tail


@pytest.mark.parametrize("l", [0, 1, 4])
def test_weighted_svd_is_optimal_in_its_norm(l):
    # Eckart-Young: at every rank h the weighted SVD has the smallest rho-weighted residual;
    # the plain SVD truncated to the same rank does worse in that norm
    W = 1.0
    mw = sp.modal_svd(l, W, 1e-12, decay=DECAY)
    mp = sp.modal_svd(l, W, 1e-12)
    for h in (1, 2, 3):
        ew = _weighted_error2(mw, h, W, DECAY)
        ep = _weighted_error2(mp, h, W, DECAY)
        assert abs(ew - float(np.sum(mw.sigma_all[h:] ** 2))) < 1e-9 + 1e-6 * ew
        assert ew < 0.9 * ep, (l, h, ew, ep)


def test_small_decay_reduces_to_the_plain_plan():
    a = sp.modal_svd(2, 1.5, 1e-4, decay=1e-9)
    b = sp.modal_svd(2, 1.5, 1e-4)
    assert a.sigma.size == b.sigma.size
    assert np.allclose(a.sigma_all[:10], b.sigma_all[:10], rtol=0, atol=1e-9)


def test_weight_lowers_the_rank():
    ranks = [sp.build_plan(1.0, 1e-3, K=1.0, decay=d).H for d in (0.0, 4.0, DECAY, 30.0)]
    assert ranks[0] > ranks[1] > ranks[2] > ranks[3]


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_fewer_terms_reach_the_accuracy_on_images_of_that_decay(eps):
    # the remark's claim: noise-free blob images (widths >= 1 px, so their spectra fall at
    # least like exp(-(pi sigma)^2 y^2)) need fewer terms under the weight, and O2 stays
    # within eps of the exact inner products O1 (Section 5.2's accuracy) with both plans
    wl = make_workload("n32_tiny", n_images=3, n_templates=3, noise=False)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    Ah = tr.polar_fourier(wl.images.astype(np.float64), k, wl.two_Q)
    Bh = tr.polar_fourier(wl.templates.astype(np.float64), k, wl.two_Q)
    a, b = tr.ring_coefficients(Ah), tr.ring_coefficients(Bh)
    delta = brute.shift_vectors(wl.shifts_px, wl.n)
    plans = {d: sp.build_plan(wl.W, eps, K, decay=d) for d in (0.0, DECAY)}
    assert plans[DECAY].H < 0.8 * plans[0.0].H
    for d, plan in plans.items():
        for i in range(3):
            X = ftk_steps.ftk_scores(a[i], b, k, w, plan, delta)
            for j in range(3):
                ref = brute.bandlimited_inner_products(Ah[i], Bh[j], k, w, delta)
                assert np.abs(X[j] - ref).max() < eps * np.abs(ref).max(), (d, i, j)
