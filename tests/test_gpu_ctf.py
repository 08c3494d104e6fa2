"""CTF-filtered templates (Section 7.1) on the GPU: the plan of ftk_plan_create_ctf
against the oracle's joint SVD (O2 with the same defocus values) and the filtered
brute force (O1 with each template ring multiplied by C(k_m; tau)).

Tolerances as for translations alone: FP32 2e-5 and BF16x3 2e-4 of the pair's
peak vs O2; vs O1 the bound of tests/test_oracle_ctf.py (2 sqrt(n_tau) eps times the
ratio of the unfiltered to the filtered peak).
"""

import math

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from oracle.best import best_pose
from workloads import make_workload

TAUS = (0.5, 1.5, 3.0)
PHASE = 0.07


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


@pytest.fixture(scope="module")
def case():
    wl = make_workload("n32_tiny", n_images=3, n_templates=4)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    Ah = tr.polar_fourier(wl.images, k, wl.two_Q)
    Bh = tr.polar_fourier(wl.templates, k, wl.two_Q)
    a, b = tr.ring_coefficients(Ah), tr.ring_coefficients(Bh)
    plan_o = svd_plan.build_plan_ctf(wl.W, wl.eps, K, TAUS, PHASE)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px, defocus=TAUS, phase=PHASE)
    delta = brute.shift_vectors(wl.shifts_px, wl.n)
    return dict(wl=wl, K=K, k=k, w=w, Ah=Ah, Bh=Bh, a=a, b=b, plan_o=plan_o, plan=plan, delta=delta,
                ad=torch.from_numpy(a.astype(np.complex64)).cuda(), bd=torch.from_numpy(b.astype(np.complex64)).cuda())


def test_ctf_plan_shape_and_rank(case):
    plan, wl = case["plan"], case["wl"]
    assert plan.n_defocus == len(TAUS)
    assert plan.N == len(TAUS) * wl.shifts_px.shape[0]
    assert plan.H == case["plan_o"].H
    l, sig = plan.terms()
    ref = sorted((lz, s) for lz, m in case["plan_o"].modes.items() if lz >= 0 for s in m.sigma)
    got = sorted(zip(l.tolist(), sig.tolist()))
    assert all(x[0] == y[0] and abs(x[1] - y[1]) < 1e-8 for x, y in zip(got, ref))


@pytest.mark.parametrize("precision,tol", [(ftk.FP32, 2e-5), (ftk.BF16X3, 2e-4)])
def test_ctf_scores_match_oracle(case, precision, tol):
    X = case["plan"].align_scores(case["ad"], case["bd"], precision).cpu().numpy().astype(np.float64)
    for i in range(3):
        ref = ftk_steps.ftk_scores(case["a"][i], case["b"], case["k"], case["w"], case["plan_o"], case["delta"])
        for j in range(4):
            assert _rel(X[i, j], ref[j]) < tol, (i, j)
    # against the filtered brute force
    i, j = 2, 1
    X1 = np.concatenate([brute.bandlimited_inner_products(
        case["Ah"][i], case["Bh"][j] * svd_plan.ctf(case["k"], case["K"], t, PHASE)[:, None], case["k"], case["w"],
        case["delta"]) for t in TAUS])
    X0 = brute.bandlimited_inner_products(case["Ah"][i], case["Bh"][j], case["k"], case["w"], case["delta"])
    bound = 2.0 * math.sqrt(len(TAUS)) * case["wl"].eps * np.abs(X0).max() / np.abs(X1).max()
    assert _rel(X[i, j], X1) < bound


def test_ctf_best_pose_over_defocus(case):
    tpl, rot, row, score = [t.cpu().numpy() for t in case["plan"].align_best(case["ad"], case["bd"], ftk.BF16X3)]
    N = case["wl"].shifts_px.shape[0]
    for i in range(3):
        ref = ftk_steps.ftk_scores(case["a"][i], case["b"], case["k"], case["w"], case["plan_o"], case["delta"])
        t, r, s, v = best_pose(ref)
        scale = np.abs(ref).max()
        assert abs(score[i] - v) < 2e-4 * scale
        assert ref[tpl[i], row[i], rot[i]] > v - 4e-4 * scale
        assert 0 <= row[i] < len(TAUS) * N   # defocus row[i] // N, shift row[i] % N
