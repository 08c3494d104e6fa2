"""The polar transform on tensor cores (eq. Ahattrap + aqkcalc) against the FP64
oracle and against the FP32 CUDA-core form of the same sum.

Tolerances, max-relative to the batch's peak coefficient: 2e-5 vs the oracle
(as for the FP32 form), 1e-5 between the two GPU forms (split-bf16 products keep
16 mantissa bits per operand; the sums are FP32).
"""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from oracle import quadrature as quad, transform as tr
from workloads import make_workload


def _rel(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


def _plan(wl):
    return ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)


@pytest.mark.parametrize("name,B", [("n32_tiny", 5), ("n64_1k", 7)])
def test_tensor_core_transform_matches_oracle(name, B):
    wl = make_workload(name, n_images=B, n_templates=1)
    plan = _plan(wl)
    coef = plan.transform(torch.from_numpy(wl.images).cuda()).cpu().numpy()
    k, _ = quad.radial_rule(wl.M, quad.nyquist_K(wl.n))
    ref = tr.fourier_bessel(wl.images.astype(np.float64), k, wl.two_Q)
    assert _rel(coef, ref) < 2e-5


@pytest.mark.parametrize("name,B", [("n64_1k", 33), ("b96_1k", 9), ("n128_8k", 5), ("b192_256", 460)])
def test_tensor_core_transform_matches_cuda_core_form(name, B):
    # b192_256 with 460 images runs the tensor-core form in two launches (455 images of scratch)
    wl = make_workload(name, n_images=B, n_templates=1)
    plan = _plan(wl)
    imgs = torch.from_numpy(wl.images).cuda()
    tc = plan.transform(imgs).cpu().numpy()
    plan.tune("transform", 1)
    simt = plan.transform(imgs).cpu().numpy()
    plan.tune("transform", 0)
    assert _rel(tc, simt) < 1e-5
    # real images: a(k; -q) = (-1)^q conj a(k; q)
    q = np.arange(wl.two_Q)
    neg = (-q) % wl.two_Q
    sign = np.where(q % 2 == 0, 1.0, -1.0)
    assert _rel(tc[:, :, neg], sign * np.conj(tc)) < 1e-5
