"""Steps 2 and 3 of eq. (fbk3) fused in one tcgen05 kernel (the DFT over q per pair
in shared memory, the shift factors resident in tensor memory as the A operand)
against the FP64 oracle and against the separate Step-2 and Step-3 kernels.

Tolerances, relative to the largest |X| of the image: 2e-4 for BF16x3 vs O2 (as
for the separate kernels). Between the fused and the separate kernels the DFT over
q is a different factorization, so Z differs by FP32 rounding before its split into
bf16 hi + lo (16 mantissa bits kept): best scores agree to 5e-5, and the pose is the
same unless another pose is within that of the best.
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle.best import best_pose
from tests.test_gpu_parity import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    return Case("n32_tiny", 16, 16)     # 2Q = 96: DFT 8 x 12, 32-rotation MMAs; 256 pairs


@pytest.fixture(scope="module")
def mid():
    return Case("n64_1k", 5, 7)         # 2Q = 192: DFT 16 x 12, 441 shifts (4 tiles, ragged)


def _run(plan, a, b, prec, fused):
    plan.tune("step23", 1 if fused else 0)
    try:
        plan.profile_begin()
        out = [t.cpu().numpy() for t in plan.align_best(a, b, prec)]
        prof = plan.profile_end()
        plan.stream_check()
    finally:
        plan.tune("step23", 1)
    assert ("step23_tc" in prof) == fused, prof
    assert ("fft_pack" in prof) != fused, prof
    return out


def _check_vs_oracle(case, out, tol=2e-4):
    tpl, rot, shift, score = out
    for i in range(len(tpl)):
        X = case.o2(i)
        t, r, s, v = best_pose(X)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < tol * scale, i
        Xs = np.sort(X.reshape(-1))
        if Xs[-1] - Xs[-2] > 2 * tol * scale:
            assert (tpl[i], rot[i], shift[i]) == (t, r, s), i
        else:
            assert X[tpl[i], shift[i], rot[i]] > v - tol * scale, i


def _check_vs_separate(f, u, scale, tol=5e-5, plan=None, a=None, b=None, prec=ftk.BF16X3, lists=None):
    """Best scores agree to tol; with the coefficients given, the fused search's pose also
    scores within tol of the maximum of the separate kernels' all-scores output (over the
    image's shortlist when `lists` is given, and shifts outside a window not counted)."""
    assert np.all(np.abs(f[3] - u[3]) <= tol * scale)
    if plan is not None:
        for i in range(len(f[0])):
            X = plan.align_scores(a[i:i + 1], b, prec).cpu().numpy()[0]
            plan.stream_check()
            ref = u[3][i] if lists is not None else X.max()
            assert X[f[0][i], f[2][i], f[1][i]] >= ref - tol * scale, i
    return ((f[0] == u[0]) & (f[1] == u[1]) & (f[2] == u[2])).mean()


@pytest.mark.parametrize("case_name", ["tiny", "mid"])
def test_fused_best_matches_oracle(case_name, request):
    case = request.getfixturevalue(case_name)
    a, b = case.dev_coeffs()
    _check_vs_oracle(case, _run(case.plan, a, b, ftk.BF16X3, True))


@pytest.mark.parametrize("prec", [ftk.BF16X3, ftk.BF16])
def test_fused_matches_separate_kernels_many_pairs_per_cta(mid, prec):
    # 40 x 9 = 360 pairs on at most 152 CTAs: each CTA cycles through both Z slots
    # and both accumulators several times
    wl = mid.wl
    from workloads import make_workload
    big = make_workload("n64_1k", n_images=40, n_templates=9, seed=5)
    a = mid.plan.transform(torch.from_numpy(big.images).cuda())
    b = mid.plan.transform(torch.from_numpy(big.templates).cuda())
    f = _run(mid.plan, a, b, prec, True)
    u = _run(mid.plan, a, b, prec, False)
    scale = np.abs(u[3]).max()
    if prec == ftk.BF16X3:
        assert _check_vs_separate(f, u, scale) > 0.9
        _check_vs_separate([x[:6] for x in f], [x[:6] for x in u], scale, plan=mid.plan, a=a[:6], b=b)
    else:  # one bf16 term: Z rounds to 8 mantissa bits, differently where the FP32 values differ
        assert np.all(np.abs(f[3] - u[3]) <= 2e-2 * scale)
    assert wl.two_Q == 192


def test_fused_bf16_single_vs_exact(tiny):
    a, b = tiny.dev_coeffs()
    tpl, rot, shift, score = _run(tiny.plan, a, b, ftk.BF16, True)
    for i in (0, 7):
        X1 = np.stack([tiny.o1(i, j) for j in range(16)])
        scale = np.abs(X1).max()
        assert abs(score[i] - X1.max()) < 3e-2 * scale


def test_fused_zero_image_takes_the_first_pose(mid):
    a, b = mid.dev_coeffs()
    a = a.clone()
    a[2] = 0
    tpl, rot, shift, score = _run(mid.plan, a, b, ftk.BF16X3, True)
    assert (tpl[2], rot[2], shift[2], score[2]) == (0, 0, 0, 0.0)


def test_fused_shortlist_with_window_matches_separate(mid):
    from paper_1905_12317_gb300.proposal import align_best_shortlist
    a, b = mid.dev_coeffs()
    sl = torch.tensor([[6, 1, 3], [0, 2, 4], [5, 5, 1], [3, 6, 0], [2, 1, 6]], dtype=torch.int32, device="cuda")
    cen = torch.tensor([[0.5, -1.0], [0.0, 0.0], [2.0, 1.0], [-1.5, 0.5], [1.0, 1.0]], dtype=torch.float32,
                       device="cuda")
    res = {}
    for fused in (True, False):
        mid.plan.tune("step23", 1 if fused else 0)
        try:
            mid.plan.profile_begin()
            res[fused] = [t.cpu().numpy() for t in align_best_shortlist(mid.plan, a, b, sl, cen, 1.25, ftk.BF16X3)]
            prof = mid.plan.profile_end()
            mid.plan.stream_check()
        finally:
            mid.plan.tune("step23", 1)
        assert ("step23_tc" in prof) == fused
    f, u = res[True], res[False]
    scale = np.abs(u[3]).max()
    _check_vs_separate(f, u, scale, plan=mid.plan, a=a, b=b, lists=sl)
    shifts = mid.wl.shifts_px
    for i in range(5):
        assert f[0][i] in sl[i].tolist()
        assert np.all(np.abs(shifts[f[2][i]] - cen[i].cpu().numpy()) <= 1.25)


def test_fused_with_odd_term_count():
    # W = 1, eps = 3e-4: H' = 31 terms, so Zhat rows are padded to 32 and the last
    # zeta block of the DFT pass is partly empty; 2Q = 96 (DFT 8 x 12), 49 shifts
    case = Case("n32_tiny", 6, 9, eps=3e-4)
    assert case.plan.H_half % 2 == 1
    a, b = case.dev_coeffs()
    _check_vs_oracle(case, _run(case.plan, a, b, ftk.BF16X3, True))


def test_separate_kernels_where_the_shift_factors_do_not_fit_tmem():
    # n = 64, eps = 3e-4: H' = 49, K padded to 112; 4 tiles of 128 shifts x 112 TMEM
    # columns leave no room for the accumulators, so the best-pose search keeps the
    # separate Step-2 and Step-3 kernels
    case = Case("n64_1k", 2, 3, eps=3e-4)
    assert case.plan.H_half == 49
    a, b = case.dev_coeffs()
    case.plan.profile_begin()
    out = [t.cpu().numpy() for t in case.plan.align_best(a, b, ftk.BF16X3)]
    prof = case.plan.profile_end()
    case.plan.stream_check()
    assert "step23_tc" not in prof and "fft_pack" in prof and "step3_tc" in prof
    _check_vs_oracle(case, out)


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_checked_run_equals_plain_run(name, request):
    # with every index checked against its buffer the results are bit-identical and no
    # index error is latched (ftk_stream_check would raise)
    case = request.getfixturevalue(name)
    a, b = case.dev_coeffs()
    ref = _run(case.plan, a, b, ftk.BF16X3, True)
    case.plan.tune("checks", 1)
    try:
        got = _run(case.plan, a, b, ftk.BF16X3, True)
    finally:
        case.plan.tune("checks", 0)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_fused_two_shift_tiles_at_96_rotations():
    # n = 32, 2Q = 96 with a 0.25-pixel shift lattice inside the 2 W = 2 pixel disk
    # (~200 shifts: two 128-shift tiles, the second ragged; 96-rotation accumulators)
    from workloads import make_workload
    wl = make_workload("n32_tiny", n_images=12, n_templates=10)
    h = 0.25
    g = np.arange(-8, 9) * h
    sx, sy = np.meshgrid(g, g, indexing="ij")
    keep = np.hypot(sx, sy) <= 2.0 * wl.W - 1e-9
    shifts = np.stack([sx[keep], sy[keep]], axis=1)
    assert 129 <= len(shifts) <= 256
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, shifts)
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    for prec in (ftk.BF16X3, ftk.BF16):
        f = _run(plan, a, b, prec, True)
        u = _run(plan, a, b, prec, False)
        scale = np.abs(u[3]).max()
        if prec == ftk.BF16X3:
            _check_vs_separate(f, u, scale, plan=plan, a=a, b=b)
        else:
            assert np.all(np.abs(f[3] - u[3]) <= 2e-2 * scale)
        assert np.all((f[2] >= 0) & (f[2] < len(shifts)))
