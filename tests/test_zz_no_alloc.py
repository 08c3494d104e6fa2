"""The no-allocation entry point ftk_align_best_static, called through the C ABI.

It exists for callers that cannot call cudaMalloc when they use the library
(their device memory belongs to another allocator, or an allocation at call
time could block, synchronize the device or fail late). It must give the same
best poses as ftk_align_best, call after call, although its scratch lives in
one static device array that every call reuses.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

import paper_1905_12317_gb300 as ftk
from workloads import make_workload

pytestmark = pytest.mark.gpu

_vp = ctypes.c_void_p


def _entry(lib):
    fn = lib.ftk_align_best_static
    fn.restype = ctypes.c_int
    fn.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
    return fn


def _outs(n):
    return (torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("precision", [ftk.FP32, ftk.BF16X3])
def test_static_scratch_matches_align_best_on_consecutive_calls(precision):
    lib = ftk.load_library()
    fn = _entry(lib)
    wl = make_workload("n32_tiny")
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    imgs = torch.from_numpy(np.ascontiguousarray(wl.images)).cuda()
    tpls = torch.from_numpy(np.ascontiguousarray(wl.templates)).cuda()
    a, b = plan.transform(imgs), plan.transform(tpls)
    NI, NT = a.shape[0], b.shape[0]
    ref = [t.cpu().numpy() for t in plan.align_best(a, b, precision)]
    stream = _vp(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = _outs(NI)
        st = fn(plan._h, precision, _vp(a.data_ptr()), NI, _vp(b.data_ptr()), NT, *[_vp(t.data_ptr()) for t in out],
                stream)
        assert st == 0, lib.ftk_status_string(st)
        plan.stream_check()
        got = [t.cpu().numpy() for t in out]
        scale = np.abs(ref[3]).max()
        assert np.all(np.abs(got[3] - ref[3]) <= 2e-5 * scale), call
        for k in range(3):
            assert np.array_equal(got[k], ref[k]), (call, k)


def test_static_scratch_rejects_problems_beyond_its_size():
    lib = ftk.load_library()
    fn = _entry(lib)
    wl = make_workload("n32_tiny", n_images=1, n_templates=1)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    dummy = torch.empty(16, dtype=torch.float32, device="cuda")
    p = _vp(dummy.data_ptr())
    # 8 bytes of per-image state for 3 million images exceed the 16 MiB array;
    # the call must refuse before touching any pointer.
    st = fn(plan._h, ftk.FP32, p, 3_000_000, p, 1, p, p, p, p, _vp(torch.cuda.current_stream().cuda_stream))
    assert st == 8
    assert b"static" in lib.ftk_status_string(st)
