"""GPU parity of the tensor-core (tcgen05) pair engine against the FP64 oracle.

Tolerances (relative to the largest |X| of the compared block):
  * BF16x3 vs O2 (same eps, same coefficients): 2e-4 (split-BF16 products, FP32 accumulate)
  * BF16x3 vs O1 (exact inner products):          eps (Section 5.2)
  * plain BF16 vs O1:                             3e-2 (reported precision, eps >= 1e-2 only)
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle.best import best_pose
from tests.test_gpu_parity import Case, _rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    return Case("n32_tiny", 16, 16)


@pytest.fixture(scope="module")
def mid():
    return Case("n64_1k", 5, 7)


def test_bf16x3_scores_tiny(tiny):
    a, b = tiny.dev_coeffs()
    X = tiny.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
    tiny.plan.stream_check()
    for i in range(16):
        assert _rel(X[i], tiny.o2(i)) < 2e-4, i
    for i, j in [(0, 0), (5, 9), (15, 15)]:
        assert _rel(X[i, j], tiny.o1(i, j)) < tiny.eps


def test_bf16_single_scores_tiny(tiny):
    a, b = tiny.dev_coeffs()
    X = tiny.plan.align_scores(a, b, ftk.BF16).cpu().numpy()
    tiny.plan.stream_check()
    for i, j in [(0, 0), (7, 3)]:
        assert _rel(X[i, j], tiny.o1(i, j)) < 3e-2


def test_bf16x3_scores_n64_ragged(mid):
    # 5 x 7 pairs x 192 rotations = 6720 rows: the last 128-row tile is ragged;
    # 441 shifts leave a ragged last 64-shift chunk.
    a, b = mid.dev_coeffs()
    X = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
    mid.plan.stream_check()
    for i in range(5):
        assert _rel(X[i], mid.o2(i)) < 2e-4, i
    assert _rel(X[1, 4], mid.o1(1, 4)) < 1e-3


def test_bf16x3_chunking_invariant(mid):
    a, b = mid.dev_coeffs()
    mn, _ = mid.plan.workspace_size(ftk.BF16X3, 5, 7)
    work = torch.empty(mn, dtype=torch.uint8, device="cuda")
    X1 = mid.plan.align_scores(a, b, ftk.BF16X3, work=work).cpu().numpy()
    X2 = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
    assert np.array_equal(X1, X2)


def test_bf16x3_best_matches_oracle(tiny):
    a, b = tiny.dev_coeffs()
    tpl, rot, shift, score = [t.cpu().numpy() for t in tiny.plan.align_best(a, b, ftk.BF16X3)]
    tiny.plan.stream_check()
    tol = 2e-4
    for i in range(16):
        X = tiny.o2(i)
        t, r, s, v = best_pose(X)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < tol * scale
        Xs = np.sort(X.reshape(-1))
        if Xs[-1] - Xs[-2] > 2 * tol * scale:
            assert (tpl[i], rot[i], shift[i]) == (t, r, s)
        else:
            assert X[tpl[i], shift[i], rot[i]] > v - tol * scale


def test_launch_shape_knobs_do_not_change_results(mid):
    a, b = mid.dev_coeffs()
    ref = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
    try:
        for knob, val in [("step3_group_max", 128), ("step3_a_stages", 3), ("step1_stages", 3),
                          ("step1_ctas_per_sm", 4)]:
            mid.plan.tune(knob, val)
        assert mid.plan.tuning()["step3_group"] <= 128
        X = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
        # the MMA width (shifts per group) may change the FP32 accumulation order
        # inside the tensor core: equal to FP32 rounding, not necessarily bitwise
        assert _rel(X, ref) < 1e-6
        # another FFT of Step 2 rounds Z differently in FP32, and the split Z = hi + lo keeps
        # 16 mantissa bits, so the scores move by up to the split's resolution (2^-16)
        mid.plan.tune("fft_lanes", 32)
        X32 = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
        assert _rel(X32, ref) < 5e-5
    finally:
        for knob in ("step3_group_max", "step3_a_stages", "step1_stages", "step1_ctas_per_sm", "fft_lanes"):
            mid.plan.tune(knob, 0)
    with pytest.raises(ftk.FtkError):
        mid.plan.tune("no_such_knob", 1)


def test_bf16x3_best_equals_scores_argmax(mid):
    # The Step-3 epilogue's running maximum equals the maximum of the written scores
    # (the separate Step-2 and Step-3 kernels, which align_scores also runs).
    a, b = mid.dev_coeffs()
    X = mid.plan.align_scores(a, b, ftk.BF16X3).cpu().numpy()
    mid.plan.tune("step23", 0)
    try:
        tpl, rot, shift, score = [t.cpu().numpy() for t in mid.plan.align_best(a, b, ftk.BF16X3)]
    finally:
        mid.plan.tune("step23", 1)
    for i in range(5):
        t, r, s, v = best_pose(X[i])
        assert (tpl[i], rot[i], shift[i]) == (t, r, s)
        assert score[i] == np.float32(v)
