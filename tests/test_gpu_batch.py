"""Uneven groups of image sizes (n = 64, 96, 128, 192) in one step.

* Each group's plan against the FP64 oracle on a 2 x 2-pair subset at the group's
  own grid (n = 96: 2Q = 288, N = 441; n = 192: 2Q = 576, N = 1793, H = 213):
  FP32 <= 2e-5 and BF16x3 <= 2e-4 of the pair's peak vs O2, and within eps of O1 on
  20 shifts (Section 5.2).
* The CUDA-graph replay of the concurrent multi-group step returns exactly the
  results of plain sequential launches.
"""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from paper_1905_12317_gb300.batch import Group, GroupedSearch
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from workloads import BATCH_GROUPS, make_workload


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("name", ["b96_1k", "b192_256"])
def test_group_grid_matches_oracle(name):
    wl = make_workload(name, n_images=2, n_templates=2)
    K = quad.nyquist_K(wl.n)
    k, w = quad.radial_rule(wl.M, K)
    Ah = tr.polar_fourier(wl.images.astype(np.float64), k, wl.two_Q)
    Bh = tr.polar_fourier(wl.templates.astype(np.float64), k, wl.two_Q)
    a, b = tr.ring_coefficients(Ah), tr.ring_coefficients(Bh)
    plan_o = svd_plan.build_plan(wl.W, wl.eps, K)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    assert plan.H == plan_o.H
    delta = brute.shift_vectors(wl.shifts_px, wl.n)
    X2 = np.stack([ftk_steps.ftk_scores(a[i], b, k, w, plan_o, delta) for i in range(2)])
    sub = np.linspace(0, len(delta) - 1, 20).astype(int)
    X1 = brute.bandlimited_inner_products(Ah[1], Bh[0], k, w, delta[sub])
    ad = torch.from_numpy(a.astype(np.complex64)).cuda()
    bd = torch.from_numpy(b.astype(np.complex64)).cuda()
    for prec, tol in [(ftk.FP32, 2e-5), (ftk.BF16X3, 2e-4)]:
        X = plan.align_scores(ad, bd, prec).cpu().numpy().astype(np.float64)
        for i in range(2):
            for j in range(2):
                assert _rel(X[i, j], X2[i, j]) < tol, (prec, i, j)
        assert _rel(X[1, 0][sub], X1) < wl.eps
    # the transform at this grid against the oracle's coefficients
    coef = plan.transform(torch.from_numpy(wl.images).cuda()).cpu().numpy()
    assert _rel(coef, a) < 2e-5


def _groups(counts, n_templates):
    out = []
    for name, ni in zip(BATCH_GROUPS, counts):
        wl = make_workload(name, n_images=ni, n_templates=n_templates)
        plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
        out.append(Group(plan=plan, images=torch.from_numpy(wl.images).cuda(),
                         templates=torch.from_numpy(wl.templates).cuda()))
    return out


def test_graph_replay_equals_sequential_launches():
    gs = GroupedSearch(_groups((16, 8, 4, 2), 40))
    gs.step_eager(concurrent=False)
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in r) for r in gs.results()]
    gs.capture()
    for r in gs.results():
        for t in r:
            t.fill_(-7)
    for _ in range(2):
        gs.replay()
    torch.cuda.synchronize()
    for g in gs.groups:
        g.plan.stream_check()
    for r, e in zip(gs.results(), ref):
        for x, y in zip(r, e):
            assert torch.equal(x, y)
    # the concurrent eager step agrees too
    gs.step_eager(concurrent=True)
    torch.cuda.synchronize()
    for r, e in zip(gs.results(), ref):
        for x, y in zip(r, e):
            assert torch.equal(x, y)


def test_c_grouped_call_equals_per_group_searches():
    # ftk_align_best_groups: the four grids (fused Steps 2-3 at 2Q = 192, separate kernels at
    # 2Q = 288, 384, 576) in one call, with the good workspace, a short one (min sizes plus a
    # share of the rest) and inside a captured CUDA graph: every group's result is that of
    # its own ftk_align_best, bit for bit
    gs = _groups((16, 8, 4, 2), 40)
    coeffs = [(g.plan, g.plan.transform(g.images), g.plan.transform(g.templates)) for g in gs]
    ref = [tuple(t.clone() for t in p.align_best(a, b, ftk.BF16X3)) for p, a, b in coeffs]
    mn, gd = ftk.groups_workspace_size(coeffs, ftk.BF16X3)
    assert 0 < mn <= gd
    for size in (gd, mn + (gd - mn) // 3):
        work = torch.empty(size, dtype=torch.uint8, device="cuda")
        outs = ftk.align_best_groups(coeffs, ftk.BF16X3, work=work)
        torch.cuda.synchronize()
        for r, e in zip(outs, ref):
            for x, y in zip(r, e):
                assert torch.equal(x, y)
    work = torch.empty(gd, dtype=torch.uint8, device="cuda")
    outs = ftk.align_best_groups(coeffs, ftk.BF16X3, work=work)   # pool streams exist before capture
    torch.cuda.synchronize()
    for r in outs:
        for t in r:
            t.fill_(-7)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            ftk.align_best_groups(coeffs, ftk.BF16X3, work=work, outs=outs, stream=side)
    graph.replay()
    torch.cuda.synchronize()
    for p, _, _ in coeffs:
        p.stream_check()
    for r, e in zip(outs, ref):
        for x, y in zip(r, e):
            assert torch.equal(x, y)
    with pytest.raises(ftk.FtkError):
        ftk.align_best_groups(coeffs, ftk.BF16X3, work=torch.empty(mn - 256, dtype=torch.uint8, device="cuda"))
