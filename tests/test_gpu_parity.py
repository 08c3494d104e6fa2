"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative to the largest |X| of the compared block):
  * transform (FP32) vs oracle coefficients:                    2e-5
  * FP32 FTK vs O2 (same eps, same coefficients):                2e-5  (FP32 rounding)
  * any FTK variant vs O1 (exact inner products):                eps   (Section 5.2)
  * BF16x3 FTK vs O2:                                             2e-4
Best poses are compared only where the oracle's top-2 margin exceeds twice the
tolerance; elsewhere the GPU pose must score within tolerance of the maximum.
"""

import math

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from oracle import brute, ftk_steps, quadrature as quad, svd_plan, transform as tr
from oracle.best import best_pose
from workloads import make_workload


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


class Case:
    def __init__(self, name, NI, NT, eps=None, seed=None):
        self.wl = wl = make_workload(name, n_images=NI, n_templates=NT, seed=seed)
        self.eps = wl.eps if eps is None else eps
        self.K = quad.nyquist_K(wl.n)
        self.k, self.w = quad.radial_rule(wl.M, self.K)
        self.delta = brute.shift_vectors(wl.shifts_px, wl.n)
        self.Ah = tr.polar_fourier(wl.images, self.k, wl.two_Q)
        self.Bh = tr.polar_fourier(wl.templates, self.k, wl.two_Q)
        self.a = tr.ring_coefficients(self.Ah)
        self.b = tr.ring_coefficients(self.Bh)
        self.plan_o = svd_plan.build_plan(wl.W, self.eps, self.K)
        self.plan = ftk.Plan(wl.n, wl.W, self.eps, wl.M, wl.two_Q, wl.shifts_px)

    def o2(self, i):
        return ftk_steps.ftk_scores(self.a[i], self.b, self.k, self.w, self.plan_o, self.delta)

    def o1(self, i, j):
        return brute.bandlimited_inner_products(self.Ah[i], self.Bh[j], self.k, self.w, self.delta)

    def dev_coeffs(self):
        a = torch.from_numpy(self.a.astype(np.complex64)).cuda()
        b = torch.from_numpy(self.b.astype(np.complex64)).cuda()
        return a, b


@pytest.fixture(scope="module")
def tiny():
    return Case("n32_tiny", 16, 16)


def test_plan_matches_oracle(tiny):
    l, sig = tiny.plan.terms()
    ref = sorted((lz, s) for lz, m in tiny.plan_o.modes.items() if lz >= 0 for s in m.sigma)
    got = sorted(zip(l.tolist(), sig.tolist()))
    assert len(got) == len(ref)
    assert all(a[0] == b[0] and abs(a[1] - b[1]) < 1e-9 for a, b in zip(got, ref))
    assert tiny.plan.H == tiny.plan_o.H
    k, w = tiny.plan.radial_rule()
    assert np.allclose(k, tiny.k, rtol=1e-13) and np.allclose(w, tiny.w, rtol=1e-12)


def test_transform_matches_oracle(tiny):
    imgs = torch.from_numpy(np.ascontiguousarray(tiny.wl.images)).cuda()
    coef = tiny.plan.transform(imgs)
    torch.cuda.synchronize()
    ref = tr.fourier_bessel(tiny.wl.images.astype(np.float64), tiny.k, tiny.wl.two_Q)
    assert _rel(coef.cpu().numpy(), ref) < 2e-5


def test_transform_edge_batches(tiny):
    # B = 0 is a no-op; B not a multiple of the kernel's image block is handled.
    imgs = torch.from_numpy(np.ascontiguousarray(tiny.wl.images[:5])).cuda()
    coef = tiny.plan.transform(imgs)
    ref = tr.fourier_bessel(tiny.wl.images[:5].astype(np.float64), tiny.k, tiny.wl.two_Q)
    assert _rel(coef.cpu().numpy(), ref) < 2e-5
    empty = torch.empty((0, tiny.wl.n, tiny.wl.n), dtype=torch.float32, device="cuda")
    assert tiny.plan.transform(empty).shape[0] == 0


def test_fp32_scores_match_o2_and_o1(tiny):
    a, b = tiny.dev_coeffs()
    X = tiny.plan.align_scores(a, b, ftk.FP32).cpu().numpy()
    for i in range(16):
        ref2 = tiny.o2(i)
        assert _rel(X[i], ref2) < 2e-5, i
    for i, j in [(0, 0), (3, 7), (15, 2)]:
        assert _rel(X[i, j], tiny.o1(i, j)) < tiny.eps


def test_fp32_scores_small_workspace_chunks(tiny):
    # A workspace for one pair at a time must give identical results.
    a, b = tiny.dev_coeffs()
    mn, _ = tiny.plan.workspace_size(ftk.FP32, 16, 16)
    work = torch.empty(mn, dtype=torch.uint8, device="cuda")
    X1 = tiny.plan.align_scores(a[:3], b[:5], ftk.FP32, work=work).cpu().numpy()
    X2 = tiny.plan.align_scores(a[:3], b[:5], ftk.FP32).cpu().numpy()
    assert np.array_equal(X1, X2)


def test_fp32_best_matches_oracle(tiny):
    a, b = tiny.dev_coeffs()
    tpl, rot, shift, score = [t.cpu().numpy() for t in tiny.plan.align_best(a, b, ftk.FP32)]
    tol = 2e-5
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


def test_end_to_end_from_pixels_recovers_planted_poses(tiny):
    imgs = torch.from_numpy(np.ascontiguousarray(tiny.wl.images)).cuda()
    tpls = torch.from_numpy(np.ascontiguousarray(tiny.wl.templates)).cuda()
    a, b = tiny.plan.transform(imgs), tiny.plan.transform(tpls)
    tpl, rot, shift, score = [t.cpu().numpy() for t in tiny.plan.align_best(a, b, ftk.FP32)]
    two_Q = tiny.wl.two_Q
    hits = 0
    for i in range(16):
        gam = -tiny.wl.true_theta[i] % (2 * math.pi)
        r_true = gam / (2 * math.pi / two_Q)
        dr = min(abs(rot[i] - r_true), two_Q - abs(rot[i] - r_true))
        ds = np.hypot(*(tiny.wl.shifts_px[shift[i]] + tiny.wl.true_shift_px[i]))
        hits += tpl[i] == tiny.wl.true_template[i] and dr <= 1.5 and ds <= 0.75
    assert hits >= 14


def test_search_host_matches_device_path(tiny):
    imgs = torch.from_numpy(np.ascontiguousarray(tiny.wl.images)).pin_memory()
    tpls = torch.from_numpy(np.ascontiguousarray(tiny.wl.templates)).pin_memory()
    _, gd = tiny.plan.search_workspace_size(ftk.FP32, 16, 16)
    work = torch.empty(gd, dtype=torch.uint8, device="cuda")
    out = tuple(torch.empty(16, dtype=d).pin_memory() for d in (torch.int32, torch.int32, torch.int32, torch.float32))
    tiny.plan.search_host(imgs, tpls, ftk.FP32, work, out)
    a, b = tiny.plan.transform(imgs.cuda()), tiny.plan.transform(tpls.cuda())
    dev = [t.cpu().numpy() for t in tiny.plan.align_best(a, b, ftk.FP32)]
    for x, y in zip(out, dev):
        assert np.array_equal(x.numpy(), y)


@pytest.fixture(scope="module")
def mid():
    # n = 64 grid of the 1024 x 1024 workload (eps = 1e-3), ragged pair counts
    return Case("n64_1k", 5, 7)


def test_fp32_n64_scores_match_o2_and_o1(mid):
    a, b = mid.dev_coeffs()
    X = mid.plan.align_scores(a, b, ftk.FP32).cpu().numpy()
    for i in range(5):
        assert _rel(X[i], mid.o2(i)) < 2e-5, i
    assert _rel(X[2, 3], mid.o1(2, 3)) < 1e-3
