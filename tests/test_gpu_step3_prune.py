"""The best-pose epilogue of Step 3 (eq. fbk3 maximised over templates, rotations and shifts)
skips the argmax search and the atomic of a row whose maximum is below the best pose its
image already holds (read from the image's key before the tile). The search must return
exactly the pose that a full argmax over all scores returns: the all-scores output runs the
same MMAs on the same operands without any pruning, so the best poses of the two paths agree
bit for bit, ties going to the lowest pose index (template, then rotation, then shift).

Grids: n = 128 (G = 208 shifts per group: accumulator chunks of 64, 64, 64, 16 columns) and
n = 64 (G = 224: 64, 64, 64, 32). The template order is also reversed, which changes which
rows can be pruned but not the answer.
"""

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from workloads import make_workload

pytestmark = pytest.mark.gpu


def _plan(name):
    wl = make_workload(name, n_images=1, n_templates=1)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    plan.tune("step23", 0)  # the separate Step-3 kernel also where the fused one fits (n = 64)
    return plan


@pytest.fixture(scope="module")
def plans():
    return {"n128_8k": _plan("n128_8k"), "n64_1k": _plan("n64_1k")}


def _full_argmax(X):
    """Lowest pose index among the maxima of X [NI, NT, N, 2Q]: (tpl, rot, shift, score)."""
    NI, NT, N, R = X.shape
    Y = X.transpose(0, 1, 3, 2).reshape(NI, -1)  # pose index (j * 2Q + r) * N + s
    idx = Y.argmax(axis=1)  # first occurrence of the maximum
    return idx // (R * N), (idx // N) % R, idx % N, Y[np.arange(NI), idx]


@pytest.mark.parametrize("name,NI,NT", [("n128_8k", 12, 9), ("n64_1k", 20, 13)])
@pytest.mark.parametrize("prec", [ftk.BF16X3, ftk.BF16, ftk.FP16])
def test_pruned_best_equals_full_argmax(plans, name, NI, NT, prec):
    plan = plans[name]
    wl = make_workload(name, n_images=NI, n_templates=NT, seed=11)
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    X = plan.align_scores(a, b, prec).cpu().numpy()
    got = [t.cpu().numpy() for t in plan.align_best(a, b, prec)]
    plan.stream_check()
    assert plan.tuning()["step3_groups"] >= 2
    tpl, rot, shift, score = _full_argmax(X)
    assert np.array_equal(got[0], tpl) and np.array_equal(got[1], rot) and np.array_equal(got[2], shift)
    assert np.array_equal(got[3], score)

    # reversed template order: the same poses, template indices mirrored
    rev = [t.cpu().numpy() for t in plan.align_best(a, b.flip(0).contiguous(), prec)]
    plan.stream_check()
    Xr = X[:, ::-1]
    t2, r2, s2, v2 = _full_argmax(np.ascontiguousarray(Xr))
    assert np.array_equal(rev[0], t2) and np.array_equal(rev[1], r2) and np.array_equal(rev[2], s2)
    assert np.array_equal(rev[3], v2)
    assert np.array_equal(v2, score)


@pytest.mark.parametrize("name,knob,NI,NT", [("n64_1k", "step23", 20, 13), ("n128_8k", "cluster23", 6, 5)])
def test_fused_kernels_prune_without_changing_the_answer(name, knob, NI, NT):
    """The fused Steps 2-3 kernels (one CTA at n = 64, a CTA cluster at n = 128) prune the same
    way. Reversing the template order changes which tiles are pruned; every pair's scores are
    the same, so the best score is identical and the pose is the same one (mirrored)."""
    wl = make_workload(name, n_images=NI, n_templates=NT, seed=12)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    plan.tune(knob, 1)
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    plan.profile_begin()
    fwd = [t.cpu().numpy() for t in plan.align_best(a, b, ftk.BF16X3)]
    prof = plan.profile_end()
    assert ("step23_tc" if knob == "step23" else "step23c_tc") in prof, prof
    rev = [t.cpu().numpy() for t in plan.align_best(a, b.flip(0).contiguous(), ftk.BF16X3)]
    plan.stream_check()
    assert np.array_equal(fwd[3], rev[3])
    assert np.array_equal(fwd[0], NT - 1 - rev[0])
    assert np.array_equal(fwd[1], rev[1]) and np.array_equal(fwd[2], rev[2])
