"""Parity at the full size of the n = 64 workload (1024 images x 1024 templates, 2Q = 192,
N = 441, eps = 1e-3) in the launch configuration the benchmark times: the transform of
every image and template, then the best-pose search with the library's default workspace
(chunks of 114 images x 1024 templates, Steps 2-3 fused).

The oracle cannot search 1024 templates per image in a test's time, so the check is a chain
on sampled images (first and last of the first chunk, first of the second, one inside, the
last):
  1. the search's best pose and score agree with the argmax of the same image's all-scores
     output (ftk_align_scores, separate Step-2 and Step-3 kernels) over all templates, to the
     fused-vs-separate tolerance of tests/test_gpu_step23.py (which holds at any size);
  2. those all-scores values match the FP64 oracle O2, computed from the same pixels with
     the oracle's own transform, on sampled templates: the reported one, the argmax, the
     planted one and two seeded random ones.
Tolerances relative to the largest |X| of the image: 1e-4 for step 1; 5e-4 for step 2 (the
FP32 transform's 2e-5 plus the BF16x3 bound of 2e-4, with margin)."""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from workloads import make_workload

pytestmark = pytest.mark.gpu

SAMPLE = (0, 113, 114, 517, 1023)


@pytest.fixture(scope="module")
def full():
    wl = make_workload("n64_1k")
    assert wl.images.shape[0] == 1024 and wl.templates.shape[0] == 1024
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    a = plan.transform(torch.from_numpy(np.ascontiguousarray(wl.images)).cuda())
    b = plan.transform(torch.from_numpy(np.ascontiguousarray(wl.templates)).cuda())
    plan.profile_begin()
    best = [t.cpu().numpy() for t in plan.align_best(a, b, ftk.BF16X3)]
    prof = plan.profile_end()
    plan.stream_check()
    return wl, plan, a, b, best, prof


def test_full_size_search_runs_the_benchmarked_kernels(full):
    wl, plan, a, b, best, prof = full
    assert "step23_tc" in prof and "step1_tc" in prof
    # one fused launch per chunk of the benchmark's workspace (114 images x all 1024 templates:
    # 912 Step-1 work units, six full rounds of 152 SMs)
    assert prof["step23_tc"][1] == prof["step1_tc"][1] >= 2
    tpl, rot, shift, score = best
    assert np.all((tpl >= 0) & (tpl < 1024) & (rot >= 0) & (rot < wl.two_Q) & (shift >= 0) & (shift < 441))
    assert np.all(np.isfinite(score))


@pytest.mark.parametrize("i", SAMPLE)
def test_full_size_best_pose_against_all_scores_and_oracle(full, i):
    wl, plan, a, b, best, _ = full
    tpl, rot, shift, score = (x[i] for x in best)
    X = plan.align_scores(a[i:i + 1], b, ftk.BF16X3).cpu().numpy()[0]      # [1024, N, 2Q]
    plan.stream_check()
    scale = float(np.abs(X).max())
    jm, sm, rm = np.unravel_index(int(np.argmax(X)), X.shape)
    xmax = float(X[jm, sm, rm])
    # 1. the fused search against the argmax of all scores
    assert abs(score - xmax) <= 1e-4 * scale
    assert X[tpl, shift, rot] >= xmax - 1e-4 * scale
    # 2. the all-scores values against the FP64 oracle from pixels, on sampled templates
    rng = np.random.default_rng(1000 + i)
    T = sorted({int(tpl), int(jm), int(wl.true_template[i]), *rng.integers(0, 1024, 2).tolist()})
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    ao = tr.fourier_bessel(wl.images[i:i + 1].astype(np.float64), k, wl.two_Q)
    bo = tr.fourier_bessel(wl.templates[T].astype(np.float64), k, wl.two_Q)
    plan_o = svd_plan.build_plan(wl.W, wl.eps, K)
    Xo = ftk_steps.ftk_scores(ao[0], bo, k, w, plan_o, brute.shift_vectors(wl.shifts_px, wl.n))
    ref = float(np.abs(Xo).max())
    for n_t, t in enumerate(T):
        assert np.abs(X[t] - Xo[n_t]).max() <= 5e-4 * ref, (i, t)
