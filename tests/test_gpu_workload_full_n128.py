"""Parity at the full size of the n = 128 precision workload (8192 images x 4096 templates,
2Q = 384, N = 797, eps = 1e-3), the configuration the benchmark times: the transform of every
image and template, then the best-pose search with the library's default workspace and launch
configuration.

The oracle cannot search 4096 templates per image, so the check is a chain on sampled images
(the first, one from a later chunk, one inside and the last):
  1. the search's best pose and score agree with the argmax of the same image's all-scores
     output (ftk_align_scores) over all 4096 templates, to 1e-4 of the image's largest |X|
     (the fused-vs-separate tolerance of the Steps 2-3 tests, with margin);
  2. those all-scores values match the FP64 oracle O2 from the same pixels (the oracle's own
     transform) on sampled templates: the reported one, the argmax, the planted one and one
     seeded random one, to 5e-4 (the FP32 transform's 2e-5 plus the BF16x3 bound of 2e-4,
     with margin).
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from workloads import make_workload

pytestmark = pytest.mark.gpu

SAMPLE = (0, 2500, 6143, 8191)


@pytest.fixture(scope="module")
def full():
    wl = make_workload("n128_8k")
    assert wl.images.shape[0] == 8192 and wl.templates.shape[0] == 4096 and wl.shifts_px.shape[0] == 797
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    a = plan.transform(torch.from_numpy(np.ascontiguousarray(wl.images)).cuda())
    b = plan.transform(torch.from_numpy(np.ascontiguousarray(wl.templates)).cuda())
    best = [t.cpu().numpy() for t in plan.align_best(a, b, ftk.BF16X3)]
    plan.stream_check()
    return wl, plan, a, b, best


def test_full_size_search_reports_valid_poses(full):
    wl, plan, a, b, best = full
    tpl, rot, shift, score = best
    assert np.all((tpl >= 0) & (tpl < 4096) & (rot >= 0) & (rot < 384) & (shift >= 0) & (shift < 797))
    assert np.all(np.isfinite(score))


@pytest.mark.parametrize("i", SAMPLE)
def test_full_size_best_pose_against_all_scores_and_oracle(full, i):
    wl, plan, a, b, best = full
    tpl, rot, shift, score = (x[i] for x in best)
    X = plan.align_scores(a[i:i + 1], b, ftk.BF16X3).cpu().numpy()[0]      # [4096, 797, 384]
    plan.stream_check()
    scale = float(np.abs(X).max())
    jm, sm, rm = np.unravel_index(int(np.argmax(X)), X.shape)
    xmax = float(X[jm, sm, rm])
    # 1. the search against the argmax of all scores
    assert abs(score - xmax) <= 1e-4 * scale
    assert X[tpl, shift, rot] >= xmax - 1e-4 * scale
    # 2. the all-scores values against the FP64 oracle from pixels, on sampled templates
    rng = np.random.default_rng(2000 + i)
    T = sorted({int(tpl), int(jm), int(wl.true_template[i]), int(rng.integers(0, 4096))})
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    ao = tr.fourier_bessel(wl.images[i:i + 1].astype(np.float64), k, wl.two_Q)
    bo = tr.fourier_bessel(wl.templates[T].astype(np.float64), k, wl.two_Q)
    plan_o = svd_plan.build_plan(wl.W, wl.eps, K)
    Xo = ftk_steps.ftk_scores(ao[0], bo, k, w, plan_o, brute.shift_vectors(wl.shifts_px, wl.n))
    ref = float(np.abs(Xo).max())
    for n_t, t in enumerate(T):
        assert np.abs(X[t] - Xo[n_t]).max() <= 5e-4 * ref, (i, t)
