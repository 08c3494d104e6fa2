"""A plan's device tables live on the device that was current when it was created; calls
that launch work on the plan with another device current are refused with FTK_ERR_ARG
before any launch (include/ftk.h, ftk_align_best)."""

import ctypes

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk

pytestmark = pytest.mark.gpu


def _plan():
    return ftk.Plan(32, 1.0, 1e-2, 16, 96, np.zeros((1, 2)))


def test_calls_on_the_plans_device_run():
    torch.cuda.set_device(0)
    plan = _plan()
    a = plan.transform(torch.zeros((2, 32, 32), device="cuda"))
    plan.align_best(a, a, ftk.FP32)
    plan.stream_check()


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second GPU to make another device current")
def test_calls_with_another_device_current_are_refused():
    torch.cuda.set_device(0)
    plan = _plan()
    x = torch.zeros((2, 32, 32), device="cuda:0")
    a = plan.transform(x)
    outs = [torch.empty(2, dtype=t, device="cuda:0") for t in (torch.int32, torch.int32, torch.int32, torch.float32)]
    lib = ftk.load_library()
    try:
        torch.cuda.set_device(1)
        st = lib.ftk_transform(plan._h, ctypes.c_void_p(x.data_ptr()), 2, ctypes.c_void_p(a.data_ptr()), None)
        assert st == 1
        st = lib.ftk_align_best_static(plan._h, ftk.FP32, ctypes.c_void_p(a.data_ptr()), 2,
                                       ctypes.c_void_p(a.data_ptr()), 2,
                                       *[ctypes.c_void_p(o.data_ptr()) for o in outs], None)
        assert st == 1
    finally:
        torch.cuda.set_device(0)
