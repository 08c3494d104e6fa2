"""FTK_FP16: one FP16 term per operand on the tcgen05 kind::f16 path (A and B both
FP16, FP32 accumulation), for Step 1, the separate Steps 2-3 and the fused Steps 2-3.

Tolerance: 5e-3 of the pair's peak vs O2. Each operand is rounded to an 11-bit
significand (relative error <= 2^-12); the plain-BF16 mode, with 8-bit significands,
measures about 2e-2 (tests/test_gpu_precision.py), and three more bits divide that
by 8. Against O1 the bound adds eps (Section 5.2).
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle.best import best_pose
from tests.test_gpu_parity import Case, _rel

pytestmark = pytest.mark.gpu

TOL = 5e-3


@pytest.fixture(scope="module")
def tiny():
    return Case("n32_tiny", 16, 16)


@pytest.fixture(scope="module")
def mid():
    return Case("n64_1k", 5, 7)


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_fp16_scores_match_oracle(name, request):
    case = request.getfixturevalue(name)
    a, b = case.dev_coeffs()
    X = case.plan.align_scores(a, b, ftk.FP16).cpu().numpy()
    case.plan.stream_check()
    worst = 0.0
    for i in range(a.shape[0]):
        worst = max(worst, _rel(X[i], case.o2(i)))
    assert worst < TOL, worst
    assert worst > 1e-6          # really rounded to FP16, not the FP32 or BF16x3 engine
    assert _rel(X[1, 2], case.o1(1, 2)) < case.eps + TOL


@pytest.mark.parametrize("fused", [True, False])
def test_fp16_best_pose(mid, fused):
    a, b = mid.dev_coeffs()
    mid.plan.tune("step23", 1 if fused else 0)
    try:
        mid.plan.profile_begin()
        tpl, rot, shift, score = [t.cpu().numpy() for t in mid.plan.align_best(a, b, ftk.FP16)]
        prof = mid.plan.profile_end()
        mid.plan.stream_check()
    finally:
        mid.plan.tune("step23", 1)
    assert ("step23_tc" in prof) == fused
    for i in range(5):
        X = mid.o2(i)
        t, r, s, v = best_pose(X)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < TOL * scale
        assert X[tpl[i], shift[i], rot[i]] > v - 2 * TOL * scale


def test_fp16_shortlist_of_all_templates_equals_full_search(tiny):
    from paper_1905_12317_gb300.proposal import align_best_shortlist
    a, b = tiny.dev_coeffs()
    sl = torch.from_numpy(np.tile(np.arange(16, dtype=np.int32)[::-1].copy(), (16, 1))).cuda()
    got = align_best_shortlist(tiny.plan, a, b, sl, precision=ftk.FP16)
    ref = tiny.plan.align_best(a, b, ftk.FP16)
    for g, r in zip(got, ref):
        assert torch.equal(g, r)

