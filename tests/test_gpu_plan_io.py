"""ftk_plan_save / ftk_plan_load: a plan read back from its file holds the same
precomputation (Section 4.5: rule, terms, factors) and gives bit-identical results
through every entry point, for plain and CTF (Section 7.1) plans, with a finer
rotation grid (Section 3.2) and a tuned Step 3 carried over."""

import numpy as np
import pytest

import torch

pytestmark = pytest.mark.gpu

import paper_1905_12317_gb300 as ftk
from workloads import make_workload


def _inputs(plan, wl):
    a = plan.transform(torch.from_numpy(wl.images).cuda())
    b = plan.transform(torch.from_numpy(wl.templates).cuda())
    return a, b


def _same(x, y):
    return all(torch.equal(u, v) for u, v in zip(x, y))


@pytest.mark.parametrize("kind", ["plain", "ctf", "rotations", "tuned"])
def test_loaded_plan_reproduces_results(tmp_path, kind):
    wl = make_workload("n32_tiny", n_images=5, n_templates=7)
    kw = dict(defocus=(0.5, 2.0), phase=0.07) if kind == "ctf" else {}
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px, **kw)
    if kind == "rotations":
        plan.set_rotations(2 * wl.two_Q)
    if kind == "tuned":
        plan.tune("step3_group_max", 16)
        plan.tune("fft_lanes", 32)
    path = str(tmp_path / "plan.ftk")
    plan.save(path)
    back = ftk.Plan.load(path)
    for attr in ("H", "H_half", "L", "M", "two_Q", "N", "n", "n_defocus", "N_shift", "W", "eps"):
        assert getattr(back, attr) == getattr(plan, attr), attr
    assert back.rotations == plan.rotations
    assert back.tuning() == plan.tuning()
    for x, y in zip(plan.terms() + plan.radial_rule(), back.terms() + back.radial_rule()):
        assert np.array_equal(x, y)
    a, b = _inputs(plan, wl)
    assert torch.equal(back.transform(torch.from_numpy(wl.images).cuda()), a)
    for prec in (ftk.FP32, ftk.BF16X3):
        if prec == ftk.FP32 and kind == "rotations":
            continue   # the FP32 engine evaluates the 2Q grid only
        assert torch.equal(plan.align_scores(a, b, prec), back.align_scores(a, b, prec))
        assert _same(plan.align_best(a, b, prec), back.align_best(a, b, prec))
    torch.cuda.synchronize()
    plan.stream_check()
    back.stream_check()


def test_save_load_round_trip_is_stable(tmp_path):
    wl = make_workload("n32_tiny", n_images=1, n_templates=1)
    plan = ftk.Plan(wl.n, wl.W, wl.eps, wl.M, wl.two_Q, wl.shifts_px)
    p1, p2 = tmp_path / "a.ftk", tmp_path / "b.ftk"
    plan.save(str(p1))
    ftk.Plan.load(str(p1)).save(str(p2))
    assert p1.read_bytes() == p2.read_bytes()
