"""Launch-shape autotuner for the tensor-core pair engine.

Coordinate descent over the plan's knobs (ftk_plan_tune): each knob in turn is
set to each of its candidate values, the search is timed on the caller's inputs
with the library's launch profiler (CUDA events on the launch stream), and the
fastest value is kept. Knobs only change launch shapes, never results.
"""

from __future__ import annotations

import time

KNOBS = {
    # knob: (candidates, kernel whose time decides)
    "step3_group_max": ([256, 224, 192, 160, 128], "step3_tc"),
    "step3_a_stages": ([2, 4, 8], "step3_tc"),
    "step1_ctas_per_sm": ([1, 2, 4], "step1_tc"),
    "step1_stages": ([3, 4, 6], "step1_tc"),
    "fft_lanes": ([8, 32], "fft_pack"),
}


def _time(plan, a, b, precision, work, out, reps, kernel):
    import torch
    plan.align_best(a, b, precision, work=work, out=out)  # warm
    torch.cuda.synchronize()
    plan.profile_begin()
    for _ in range(reps):
        plan.align_best(a, b, precision, work=work, out=out)
    prof = plan.profile_end()
    return prof.get(kernel, (float("inf"), 1))[0] / reps


def autotune(plan, a, b, precision, work=None, reps: int = 2, knobs=None, log=None) -> dict:
    """Tunes `plan` in place for inputs a [NI, M, 2Q], b [NT, M, 2Q]; returns the chosen knobs."""
    import torch
    NI = a.shape[0]
    if work is None:
        _, gd = plan.workspace_size(precision, NI, b.shape[0])
        work = torch.empty(gd, dtype=torch.uint8, device=a.device)
    out = tuple(torch.empty(NI, dtype=d, device=a.device)
                for d in (torch.int32, torch.int32, torch.int32, torch.float32))
    chosen = {}
    t0 = time.perf_counter()
    for knob, (cands, kernel) in (knobs or KNOBS).items():
        best_v, best_t = 0, _time(plan, a, b, precision, work, out, reps, kernel)
        for v in cands:
            try:
                plan.tune(knob, v)
            except Exception:
                continue
            t = _time(plan, a, b, precision, work, out, reps, kernel)
            if log is not None:
                log.append((knob, v, t, dict(plan.tuning())))
            if t < best_t:
                best_v, best_t = v, t
        plan.tune(knob, best_v)
        chosen[knob] = best_v
    chosen["seconds"] = time.perf_counter() - t0
    chosen.update(plan.tuning())
    return chosen
