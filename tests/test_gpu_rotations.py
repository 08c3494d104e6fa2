"""Finer rotation grids by zero-padding Step 2 (Section 3.2) on the tensor-core engine.

With R = f * 2Q rotations gamma_r = 2 pi r / R the scores must match the oracle's
Step 2 evaluated on the same grid (O2, BF16x3 tolerance 2e-4 of the pair's peak),
stay within eps of the off-grid brute force (O1 with the ring's trigonometric
interpolant), and keep every f-th rotation equal to the default-grid score.
"""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from paper_1905_12317_gb300 import proposal as pr
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from oracle.best import best_pose
from workloads import make_workload


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


class _Case:
    def __init__(self, name, NI, NT):
        self.wl = wl = make_workload(name, n_images=NI, n_templates=NT)
        K = quad.nyquist_K(wl.n)
        self.k, self.w = quad.radial_rule(wl.M, K)
        self.Ah = tr.polar_fourier(wl.images, self.k, wl.two_Q)
        self.Bh = tr.polar_fourier(wl.templates, self.k, wl.two_Q)
        self.a, self.b = tr.ring_coefficients(self.Ah), tr.ring_coefficients(self.Bh)
        self.delta = brute.shift_vectors(wl.shifts_px, wl.n)
        self.plan_o = svd_plan.build_plan(wl.W, wl.eps, K)
        self.plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
        self.ad = torch.from_numpy(self.a.astype(np.complex64)).cuda()
        self.bd = torch.from_numpy(self.b.astype(np.complex64)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return _Case("n32_tiny", 4, 5)


@pytest.mark.parametrize("f", [2, 4])
def test_finer_grid_scores_match_oracle(tiny, f):
    R = f * tiny.wl.two_Q
    coarse = tiny.plan.align_scores(tiny.ad, tiny.bd, ftk.BF16X3).cpu().numpy()
    tiny.plan.set_rotations(R)
    try:
        assert tiny.plan.rotations == R
        X = tiny.plan.align_scores(tiny.ad, tiny.bd, ftk.BF16X3).cpu().numpy().astype(np.float64)
        assert X.shape == (4, 5, tiny.plan.N, R)
        for i in range(4):
            ref = ftk_steps.ftk_scores(tiny.a[i], tiny.b, tiny.k, tiny.w, tiny.plan_o, tiny.delta, n_rot=R)
            assert _rel(X[i], ref) < 2e-4, i
        assert _rel(X[..., ::f], coarse) < 2e-4
        sub = np.arange(0, tiny.plan.N, 7)
        X1 = brute.bandlimited_inner_products_rot(tiny.Ah[1], tiny.Bh[3], tiny.k, tiny.w, tiny.delta[sub],
                                                  2 * np.pi * np.arange(R) / R)
        assert _rel(X[1, 3][sub], X1) < tiny.wl.eps
        # best pose on the finer grid
        tpl, rot, shift, score = [t.cpu().numpy() for t in tiny.plan.align_best(tiny.ad, tiny.bd, ftk.BF16X3)]
        for i in range(4):
            ref = ftk_steps.ftk_scores(tiny.a[i], tiny.b, tiny.k, tiny.w, tiny.plan_o, tiny.delta, n_rot=R)
            t, r, s, v = best_pose(ref)
            scale = np.abs(ref).max()
            assert abs(score[i] - v) < 2e-4 * scale
            assert ref[tpl[i], shift[i], rot[i]] > v - 4e-4 * scale
            assert 0 <= rot[i] < R
        # the shortlist path on the finer grid: all templates = the full search, bit for bit
        sl = torch.from_numpy(np.tile(np.arange(5, dtype=np.int32)[::-1].copy(), (4, 1))).cuda()
        got = pr.align_best_shortlist(tiny.plan, tiny.ad, tiny.bd, sl, precision=ftk.BF16X3)
        full = tiny.plan.align_best(tiny.ad, tiny.bd, ftk.BF16X3)
        for g, r in zip(got, full):
            assert torch.equal(g, r)
    finally:
        tiny.plan.set_rotations(tiny.wl.two_Q)


def test_rotation_grid_arguments(tiny):
    two_Q = tiny.wl.two_Q
    with pytest.raises(ftk.FtkError):
        tiny.plan.set_rotations(two_Q + 32)          # not a multiple of 2Q
    with pytest.raises(ftk.FtkError):
        tiny.plan.set_rotations(5 * two_Q)           # 480: no register FFT of that length
    assert tiny.plan.rotations == two_Q
    tiny.plan.set_rotations(2 * two_Q)
    with pytest.raises(ftk.FtkError):
        tiny.plan.align_best(tiny.ad, tiny.bd, ftk.FP32)   # finer grids run on the tensor path
    tiny.plan.set_rotations(two_Q)
    tiny.plan.align_best(tiny.ad, tiny.bd, ftk.FP32)
    torch.cuda.synchronize()


@pytest.mark.parametrize("f", [3, 4])
def test_finer_grid_n64(f):
    c = _Case("n64_1k", 3, 4)
    R = f * c.wl.two_Q
    c.plan.set_rotations(R)
    X = c.plan.align_scores(c.ad, c.bd, ftk.BF16X3).cpu().numpy().astype(np.float64)
    for i in range(3):
        ref = ftk_steps.ftk_scores(c.a[i], c.b, c.k, c.w, c.plan_o, c.delta, n_rot=R)
        assert _rel(X[i], ref) < 2e-4, i
