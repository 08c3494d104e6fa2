"""Steps 2 and 3 of eq. (fbk3) fused over a cluster of CTAs, on the n = 128 grid of the
precision workload (2Q = 384, 797 shifts in 4 Step-3 shift groups of 208, K = 2 H' = 128 in
4 slices of 32): each CTA of a 4-CTA cluster holds one shift group, and the DFT over q of
every pair is computed once per cluster (slice by slice) and shared through the cluster's
shared memory. Checked through the C ABI against the FP64 oracle O2 and against the
separate Step-2 and Step-3 kernels.

Tolerances, relative to the largest |X| of the image (as for the single-CTA fused kernel):
2e-4 for BF16x3 vs O2; between the fused and the separate kernels the DFT over q is a
different factorization (radix-3 split and a 128-point FFT against a 32 x 12 split), so Z
differs by FP32 rounding before its 16-bit split: best scores agree to 5e-5, and the fused
search's pose scores within 5e-5 of the maximum of the separate kernels' all scores.
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle.best import best_pose
from paper_1905_12317_gb300.proposal import align_best_shortlist
from tests.test_gpu_parity import Case
from workloads import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n128():
    c = Case("n128_8k", 3, 5)
    assert c.wl.two_Q == 384 and c.wl.shifts_px.shape[0] == 797 and c.plan.H_half == 64
    return c


def _run(plan, fn, cluster):
    plan.tune("cluster23", 1 if cluster else 0)
    try:
        plan.profile_begin()
        out = [t.cpu().numpy() for t in fn()]
        prof = plan.profile_end()
        plan.stream_check()
    finally:
        plan.tune("cluster23", 0)
    assert ("step23c_tc" in prof) == cluster, prof
    assert ("fft_pack" in prof) != cluster, prof
    return out


def _check_vs_separate(plan, a, b, f, u, prec, tol=5e-5):
    """Best scores agree; the fused pose scores within tol of the all-scores maximum."""
    scale = np.abs(u[3]).max()
    assert np.all(np.abs(f[3] - u[3]) <= tol * scale)
    for i in range(len(f[0])):
        X = plan.align_scores(a[i:i + 1], b, prec).cpu().numpy()[0]
        plan.stream_check()
        assert X[f[0][i], f[2][i], f[1][i]] >= X.max() - tol * scale, i
    return ((f[0] == u[0]) & (f[1] == u[1]) & (f[2] == u[2])).mean()


def test_cluster_fused_best_matches_oracle(n128):
    a, b = n128.dev_coeffs()
    tpl, rot, shift, score = _run(n128.plan, lambda: n128.plan.align_best(a, b, ftk.BF16X3), True)
    tol = 2e-4
    for i in range(len(tpl)):
        X = n128.o2(i)
        t, r, s, v = best_pose(X)
        scale = np.abs(X).max()
        assert abs(score[i] - v) < tol * scale, i
        Xs = np.sort(X.reshape(-1))
        if Xs[-1] - Xs[-2] > 2 * tol * scale:
            assert (tpl[i], rot[i], shift[i]) == (t, r, s), i
        else:
            assert X[tpl[i], shift[i], rot[i]] > v - tol * scale, i


@pytest.mark.parametrize("prec", [ftk.BF16X3, ftk.BF16])
def test_cluster_fused_matches_separate_kernels_many_pairs_per_cluster(n128, prec):
    # 40 x 9 = 360 pairs over at most 38 clusters: every cluster cycles through its ring slots
    # and both accumulators many times; the pairs of the last round leave some clusters idle
    big = make_workload("n128_8k", n_images=40, n_templates=9, seed=5)
    a = n128.plan.transform(torch.from_numpy(big.images).cuda())
    b = n128.plan.transform(torch.from_numpy(big.templates).cuda())
    f = _run(n128.plan, lambda: n128.plan.align_best(a, b, prec), True)
    u = _run(n128.plan, lambda: n128.plan.align_best(a, b, prec), False)
    if prec == ftk.BF16X3:
        assert _check_vs_separate(n128.plan, a[:6], b, [x[:6] for x in f], [x[:6] for x in u], prec) > 0.5
        scale = np.abs(u[3]).max()
        assert np.all(np.abs(f[3] - u[3]) <= 5e-5 * scale)
    else:  # one bf16 term: Z rounds to 8 mantissa bits, differently where the FP32 values differ
        assert np.all(np.abs(f[3] - u[3]) <= 2e-2 * np.abs(u[3]).max())


def test_cluster_fused_zero_image_takes_the_first_pose(n128):
    a, b = n128.dev_coeffs()
    a = a.clone()
    a[1] = 0
    tpl, rot, shift, score = _run(n128.plan, lambda: n128.plan.align_best(a, b, ftk.BF16X3), True)
    assert (tpl[1], rot[1], shift[1], score[1]) == (0, 0, 0, 0.0)


def test_cluster_fused_shortlist_with_window_matches_separate(n128):
    a, b = n128.dev_coeffs()
    sl = torch.tensor([[4, 1], [0, 2], [3, 3]], dtype=torch.int32, device="cuda")
    cen = torch.tensor([[0.5, -1.0], [0.0, 0.0], [-2.0, 1.5]], dtype=torch.float32, device="cuda")
    f = _run(n128.plan, lambda: align_best_shortlist(n128.plan, a, b, sl, cen, 1.25, ftk.BF16X3), True)
    u = _run(n128.plan, lambda: align_best_shortlist(n128.plan, a, b, sl, cen, 1.25, ftk.BF16X3), False)
    scale = np.abs(u[3]).max()
    assert np.all(np.abs(f[3] - u[3]) <= 5e-5 * scale)
    shifts = n128.wl.shifts_px
    for i in range(3):
        assert f[0][i] in sl[i].tolist()
        assert np.all(np.abs(shifts[f[2][i]] - cen[i].cpu().numpy()) <= 1.25)
