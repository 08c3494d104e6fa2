"""Failure detection without a GPU fault: a bounded device wait that nothing
completes gives up, the host reads FTK_ERR_TIMEOUT from ftk_stream_check, the
latch clears, and the same context keeps producing correct results."""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from workloads import make_workload


def test_bounded_wait_times_out_and_the_context_survives():
    wl = make_workload("n32_tiny", n_images=4, n_templates=5)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    before = [t.clone() for t in plan.align_best(a, b, ftk.BF16X3)]
    plan.stream_check()
    plan.selftest_timeout(20000)          # 20 ms
    with pytest.raises(ftk.FtkError) as e:
        plan.stream_check()
    assert e.value.status == 5            # FTK_ERR_TIMEOUT
    plan.stream_check()                   # the latch was cleared
    after = plan.align_best(a, b, ftk.BF16X3)
    plan.stream_check()
    for x, y in zip(before, after):
        assert torch.equal(x, y)
    with pytest.raises(ftk.FtkError):
        plan.selftest_timeout(0)          # argument check, nothing launched
