"""Pins for O2, the step-by-step FTK oracle, against O1 (no GPU).

Section 5.2: the FTK error is controlled by Sigma_{H+1} <= eps, so O2 converges to
O1 as eps -> 0 and stays within an eps-sized relative error.
"""

import numpy as np
import pytest

from oracle import brute, ftk_steps, quadrature as quad, svd_plan as sp, transform as tr
from workloads import make_workload


@pytest.fixture(scope="module")
def tiny():
    wl = make_workload("n32_tiny", n_images=3, n_templates=3)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    Ah = tr.polar_fourier(wl.images, k, wl.two_Q)
    Bh = tr.polar_fourier(wl.templates, k, wl.two_Q)
    delta = brute.shift_vectors(wl.shifts_px, wl.n)
    X1 = np.stack([[brute.bandlimited_inner_products(Ah[i], Bh[j], k, w, delta) for j in range(3)]
                   for i in range(3)])
    return dict(wl=wl, K=K, k=k, w=w, a=tr.ring_coefficients(Ah), b=tr.ring_coefficients(Bh),
                delta=delta, X1=X1)


def _rel(X, ref):
    return float(np.abs(X - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("eps,tol", [(1e-2, 1e-2), (1e-3, 1e-3), (1e-8, 1e-6)])
def test_o2_within_eps_of_o1(tiny, eps, tol):
    plan = sp.build_plan(tiny["wl"].W, eps, tiny["K"])
    for i in range(3):
        X2 = ftk_steps.ftk_scores(tiny["a"][i], tiny["b"], tiny["k"], tiny["w"], plan, tiny["delta"])
        assert _rel(X2, tiny["X1"][i]) < tol


def test_o2_error_decreases_with_eps(tiny):
    errs = []
    for eps in (1e-2, 1e-4, 1e-6):
        plan = sp.build_plan(tiny["wl"].W, eps, tiny["K"])
        X2 = ftk_steps.ftk_scores(tiny["a"][0], tiny["b"][0], tiny["k"], tiny["w"], plan, tiny["delta"])
        errs.append(_rel(X2, tiny["X1"][0, 0]))
    assert errs[0] > errs[1] > errs[2]


def test_o2_imaginary_part_small(tiny):
    plan = sp.build_plan(tiny["wl"].W, 1e-3, tiny["K"])
    X2 = ftk_steps.ftk_scores(tiny["a"][1], tiny["b"][2], tiny["k"], tiny["w"], plan, tiny["delta"],
                              return_complex=True)
    assert np.abs(X2.imag).max() < 1e-10 * np.abs(X2.real).max()


def test_o2_zero_shift_uses_only_order_zero(tiny):
    # J_l(0) = 0 for l != 0: at delta = 0 only the l = 0 terms contribute, and the
    # result is the pure rotational correlation of O1 within eps.
    plan = sp.build_plan(tiny["wl"].W, 1e-6, tiny["K"])
    zero = np.zeros((1, 2))
    X2 = ftk_steps.ftk_scores(tiny["a"][0], tiny["b"][0], tiny["k"], tiny["w"], plan, zero)
    p0 = sp.Plan(W=plan.W, eps=plan.eps, K=plan.K, modes={0: plan.modes[0]})
    X2_l0 = ftk_steps.ftk_scores(tiny["a"][0], tiny["b"][0], tiny["k"], tiny["w"], p0, zero)
    Ah0 = tiny["X1"][0, 0]
    ref = brute.bandlimited_inner_products(
        tr.polar_fourier(tiny["wl"].images[:1], tiny["k"], tiny["wl"].two_Q)[0],
        tr.polar_fourier(tiny["wl"].templates[:1], tiny["k"], tiny["wl"].two_Q)[0],
        tiny["k"], tiny["w"], zero)
    assert _rel(X2, ref) < 1e-5
    assert _rel(X2_l0, X2) < 1e-5
    assert Ah0.shape[1] == X2.shape[1]


def test_o1_off_grid_equals_o1_on_the_grid(tiny):
    wl, k, w = tiny["wl"], tiny["k"], tiny["w"]
    Ah = tr.polar_fourier(wl.images[:1], k, wl.two_Q)[0]
    Bh = tr.polar_fourier(wl.templates[1:2], k, wl.two_Q)[0]
    Q = wl.two_Q // 2
    X = brute.bandlimited_inner_products_rot(Ah, Bh, k, w, tiny["delta"], np.pi * np.arange(wl.two_Q) / Q)
    assert _rel(X, tiny["X1"][0, 1]) < 1e-12


def test_o2_on_a_finer_rotation_grid(tiny):
    # Step 2 zero-padded to R = 4 * 2Q: every 4th rotation is the 2Q-grid result, and at
    # eps -> 0 the whole grid converges to the off-grid brute force
    wl, k, w = tiny["wl"], tiny["k"], tiny["w"]
    R = 4 * wl.two_Q
    plan = sp.build_plan(wl.W, 1e-8, tiny["K"])
    Xf = ftk_steps.ftk_scores(tiny["a"][2], tiny["b"][0], k, w, plan, tiny["delta"], n_rot=R)
    Xc = ftk_steps.ftk_scores(tiny["a"][2], tiny["b"][0], k, w, plan, tiny["delta"])
    assert _rel(Xf[:, ::4], Xc) < 1e-12
    Ah = tr.polar_fourier(wl.images[2:3], k, wl.two_Q)[0]
    Bh = tr.polar_fourier(wl.templates[:1], k, wl.two_Q)[0]
    X1f = brute.bandlimited_inner_products_rot(Ah, Bh, k, w, tiny["delta"], 2 * np.pi * np.arange(R) / R)
    assert _rel(Xf, X1f) < 1e-6


def test_off_grid_rotation_peaks_at_the_true_angle():
    # a noise-free template rotated analytically by a fraction of a grid step: the
    # off-grid inner product at zero shift peaks at gamma = -theta (translate, then rotate: R_gamma T_delta)
    from workloads.synthetic import render_blobs
    wl = make_workload("n32_tiny", n_images=1, n_templates=1, noise=False)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    c, s, amp = wl.template_blobs[0]
    Q = wl.two_Q // 2
    theta = 0.37 * np.pi / Q
    rot = np.stack([np.cos(theta) * c[:, 0] - np.sin(theta) * c[:, 1],
                    np.sin(theta) * c[:, 0] + np.cos(theta) * c[:, 1]], axis=1)
    img = render_blobs(wl.n, rot, s, amp)[None]
    Ah = tr.polar_fourier(img, k, wl.two_Q)[0]
    Bh = tr.polar_fourier(wl.templates[:1].astype(np.float64), k, wl.two_Q)[0]
    offs = np.linspace(-0.5, 0.5, 21) * (np.pi / Q)
    X = brute.bandlimited_inner_products_rot(Ah, Bh, k, w, np.zeros((1, 2)), -theta + offs)[0]
    assert abs(int(np.argmax(X)) - 10) <= 1
