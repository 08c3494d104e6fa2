"""The spectrally weighted plan (Section 4.5, the remark on alternative weight functions
after Remark r:svd) on the GPU: its terms against the oracle's weighted SVD, FP32 and
BF16x3 scores against O2 under the same weight, the best pose, the accuracy against the
exact inner products O1 on noise-free images of that spectral decay, and plan files
that keep the weight. Tolerances as for the plain plan (tests/test_gpu_parity.py)."""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle import svd_plan
from oracle.best import best_pose
from tests.test_gpu_parity import Case

pytestmark = pytest.mark.gpu

DECAY = 10.0   # (pi sigma)^2 for blobs of sigma = 1 px


def _weighted(case):
    wl = case.wl
    case.plan_o = svd_plan.build_plan(wl.W, case.eps, case.K, decay=DECAY)
    case.plan = ftk.Plan(wl.n, wl.W, case.eps, wl.M, wl.two_Q, wl.shifts_px, decay=DECAY)
    return case


@pytest.fixture(scope="module")
def wtiny():
    return _weighted(Case("n32_tiny", 6, 5))


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def test_weighted_plan_matches_oracle(wtiny):
    plain = ftk.Plan(wtiny.wl.n, wtiny.wl.W, wtiny.eps, wtiny.wl.M, wtiny.wl.two_Q, wtiny.wl.shifts_px)
    assert wtiny.plan.decay == DECAY and plain.decay == 0.0
    assert wtiny.plan.H == wtiny.plan_o.H < plain.H
    l, sig = wtiny.plan.terms()
    ref = sorted((lz, s) for lz, m in wtiny.plan_o.modes.items() if lz >= 0 for s in m.sigma)
    got = sorted(zip(l.tolist(), sig.tolist()))
    assert len(got) == len(ref)
    assert all(a[0] == b[0] and abs(a[1] - b[1]) < 1e-9 for a, b in zip(got, ref))


@pytest.mark.parametrize("prec,tol", [(ftk.FP32, 2e-5), (ftk.BF16X3, 2e-4)])
def test_weighted_scores_match_oracle(wtiny, prec, tol):
    a, b = wtiny.dev_coeffs()
    X = wtiny.plan.align_scores(a, b, prec).cpu().numpy()
    wtiny.plan.stream_check()
    for i in range(a.shape[0]):
        assert _rel(X[i], wtiny.o2(i)) < tol, i


def test_weighted_best_pose_matches_oracle(wtiny):
    a, b = wtiny.dev_coeffs()
    tpl, rot, shift, score = [t.cpu().numpy() for t in wtiny.plan.align_best(a, b, ftk.BF16X3)]
    wtiny.plan.stream_check()
    tol = 2e-4
    for i in range(a.shape[0]):
        X = wtiny.o2(i)
        t, r, s, v = best_pose(X)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < tol * scale
        Xs = np.sort(X.reshape(-1))
        if Xs[-1] - Xs[-2] > 2 * tol * scale:
            assert (tpl[i], rot[i], shift[i]) == (t, r, s), i


def test_weighted_plan_meets_eps_on_images_of_that_decay():
    # noise-free blobs of width >= 1 px: fewer terms, still within eps of O1 (Section 5.2)
    case = Case("n32_tiny", 3, 3)
    from workloads import make_workload
    from oracle import brute, transform as tr
    wl = make_workload("n32_tiny", n_images=3, n_templates=3, noise=False)
    case.wl = wl
    case.Ah = tr.polar_fourier(wl.images, case.k, wl.two_Q)
    case.Bh = tr.polar_fourier(wl.templates, case.k, wl.two_Q)
    case.a, case.b = tr.ring_coefficients(case.Ah), tr.ring_coefficients(case.Bh)
    _weighted(case)
    a, b = case.dev_coeffs()
    X = case.plan.align_scores(a, b, ftk.FP32).cpu().numpy()
    case.plan.stream_check()
    for i in range(3):
        for j in range(3):
            ref = brute.bandlimited_inner_products(case.Ah[i], case.Bh[j], case.k, case.w, case.delta)
            assert _rel(X[i, j], ref) < case.eps, (i, j)


def test_weighted_plan_file_keeps_the_weight(wtiny, tmp_path):
    path = str(tmp_path / "w.ftk")
    wtiny.plan.save(path)
    back = ftk.Plan.load(path)
    assert back.decay == DECAY and back.H == wtiny.plan.H
    a, b = wtiny.dev_coeffs()
    assert torch.equal(wtiny.plan.align_scores(a, b, ftk.FP32), back.align_scores(a, b, ftk.FP32))
    back.stream_check()


def test_spectral_weight_not_offered_with_ctf(wtiny):
    wl = wtiny.wl
    with pytest.raises(ValueError):
        ftk.Plan(wl.n, wl.W, wtiny.eps, wl.M, wl.two_Q, wl.shifts_px, defocus=[0.5], decay=DECAY)
