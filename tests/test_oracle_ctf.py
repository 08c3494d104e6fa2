"""Pins for the CTF-parametrized plan of the oracle (Section 7.1), no GPU.

The brute-force reference filters the template by C(k_m; tau) on every ring and
evaluates eq. (Xdg) as O1 does; the factorized O2 must converge to it as eps -> 0
and stay within eps, and a constant CTF must reduce to the plain plan.
"""

import math

import numpy as np
import pytest

from oracle import brute, ftk_steps, quadrature as quad, svd_plan as sp, transform as tr
from workloads import make_workload

TAUS = (0.5, 1.5, 3.0)
PHASE = 0.07


@pytest.fixture(scope="module")
def tiny():
    wl = make_workload("n32_tiny", n_images=2, n_templates=2)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    Ah = tr.polar_fourier(wl.images, k, wl.two_Q)
    Bh = tr.polar_fourier(wl.templates, k, wl.two_Q)
    delta = brute.shift_vectors(wl.shifts_px, wl.n)
    return dict(wl=wl, K=K, k=k, w=w, Ah=Ah, Bh=Bh, a=tr.ring_coefficients(Ah), b=tr.ring_coefficients(Bh),
                delta=delta)


def _rel(X, ref):
    return float(np.abs(X - ref).max() / np.abs(ref).max())


def _o1_ctf(t, i, j, taus, phase):
    rows = []
    for tau in taus:
        C = sp.ctf(t["k"], t["K"], tau, phase)[:, None]
        rows.append(brute.bandlimited_inner_products(t["Ah"][i], t["Bh"][j] * C, t["k"], t["w"], t["delta"]))
    return np.concatenate(rows, axis=0)   # rows (tau_b, shift s), b-major


def test_ctf_formula():
    K = 10.0
    assert abs(sp.ctf(0.0, K, 2.0, 0.07) + math.sin(0.07)) < 1e-15
    assert abs(sp.ctf(K, K, 1.0, 0.0)) < 1e-12            # -sin(pi) at k = K
    assert abs(sp.ctf(K / math.sqrt(2), K, 1.0, 0.0) + 1.0) < 1e-12   # -sin(pi / 2)


def test_constant_ctf_reduces_to_the_plain_plan(tiny):
    # tau = 0, phase = pi/2: C = -1 everywhere, so the scores flip sign and the ranks agree
    W = tiny["wl"].W
    plain = sp.build_plan(W, 1e-3, tiny["K"])
    flat = sp.build_plan_ctf(W, 1e-3, tiny["K"], (0.0,), 0.5 * math.pi)
    assert flat.H == plain.H
    X0 = ftk_steps.ftk_scores(tiny["a"][0], tiny["b"], tiny["k"], tiny["w"], plain, tiny["delta"])
    X1 = ftk_steps.ftk_scores(tiny["a"][0], tiny["b"], tiny["k"], tiny["w"], flat, tiny["delta"])
    assert _rel(X1, -X0) < 1e-9


# The joint SVD truncates the stacked kernel of n_tau defocus values at eps with each value
# weighted 1/n_tau, so one defocus value's kernel error is up to sqrt(n_tau) eps in the
# norm that bounds the unfiltered scores (Section 5.2), and the CTF zeros make the filtered
# scores smaller than the unfiltered ones. Bound used: 2 sqrt(n_tau) eps times the ratio of
# the unfiltered to the filtered peak; the strong pin is convergence as eps -> 0.
@pytest.mark.parametrize("eps", [1e-3, 1e-8])
def test_ctf_plan_matches_filtered_brute_force(tiny, eps):
    plan = sp.build_plan_ctf(tiny["wl"].W, eps, tiny["K"], TAUS, PHASE)
    for i, j in [(0, 0), (1, 0)]:
        X2 = ftk_steps.ftk_scores(tiny["a"][i], tiny["b"][j], tiny["k"], tiny["w"], plan, tiny["delta"])
        X1 = _o1_ctf(tiny, i, j, TAUS, PHASE)
        assert X2.shape == X1.shape == (len(TAUS) * tiny["delta"].shape[0], tiny["wl"].two_Q)
        X0 = brute.bandlimited_inner_products(tiny["Ah"][i], tiny["Bh"][j], tiny["k"], tiny["w"], tiny["delta"])
        bound = 2.0 * math.sqrt(len(TAUS)) * eps * np.abs(X0).max() / np.abs(X1).max()
        assert _rel(X2, X1) < max(bound, 1e-6 if eps < 1e-6 else 0.0)


def test_ctf_rank_exceeds_plain_rank(tiny):
    W = tiny["wl"].W
    assert sp.build_plan_ctf(W, 1e-3, tiny["K"], TAUS, PHASE).H > sp.build_plan(W, 1e-3, tiny["K"]).H
