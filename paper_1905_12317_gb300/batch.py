"""Uneven groups of image sizes searched together under one CUDA graph.

Each group has its own plan (image size n, polar grid, shift set, eps), images
and templates. One step transforms every group's images and templates and runs
the per-image best-pose search of every group. Groups run on their own streams
(forked from and joined to the caller's stream), so small groups overlap large
ones; the whole multi-stream step is captured once as a CUDA graph and then
replayed with a single launch, which removes the per-kernel launch cost of the
many short launches of the small groups. Every kernel is the library's; this
module only allocates buffers, orders the calls and drives the capture.
"""

from __future__ import annotations

from dataclasses import dataclass, field

from .binding import BF16X3


@dataclass
class Group:
    plan: object
    images: object            # device float32 [NI, n, n]
    templates: object         # device float32 [NT, n, n]
    precision: int = BF16X3
    a: object = None
    b: object = None
    work: object = None
    out: tuple = field(default_factory=tuple)
    stream: object = None


class GroupedSearch:
    """Best pose per image for several (plan, images, templates) groups in one step."""

    def __init__(self, groups, device="cuda"):
        import torch
        self.device = torch.device(device)
        self.groups = []
        for g in groups:
            plan = g.plan
            NI, NT = g.images.shape[0], g.templates.shape[0]
            g.a = torch.empty((NI, plan.M, plan.two_Q), dtype=torch.complex64, device=self.device)
            g.b = torch.empty((NT, plan.M, plan.two_Q), dtype=torch.complex64, device=self.device)
            g.work = torch.empty(plan.workspace_size(g.precision, NI, NT)[1], dtype=torch.uint8, device=self.device)
            g.out = (torch.empty(NI, dtype=torch.int32, device=self.device),
                     torch.empty(NI, dtype=torch.int32, device=self.device),
                     torch.empty(NI, dtype=torch.int32, device=self.device),
                     torch.empty(NI, dtype=torch.float32, device=self.device))
            g.stream = torch.cuda.Stream(device=self.device)
            self.groups.append(g)
        self.graph = None

    def poses_per_step(self) -> int:
        return sum(g.images.shape[0] * g.templates.shape[0] * g.plan.two_Q * g.plan.N for g in self.groups)

    def _group_step(self, g, stream):
        g.plan.transform(g.images, out=g.a, stream=stream)
        g.plan.transform(g.templates, out=g.b, stream=stream)
        g.plan.align_best(g.a, g.b, g.precision, work=g.work, out=g.out, stream=stream)

    def step_eager(self, concurrent: bool = True):
        """One step with ordinary launches (groups on their own streams if ``concurrent``)."""
        import torch
        main = torch.cuda.current_stream(self.device)
        if not concurrent:
            for g in self.groups:
                self._group_step(g, main)
            return
        for g in self.groups:
            g.stream.wait_stream(main)
        for g in self.groups:
            with torch.cuda.stream(g.stream):
                self._group_step(g, g.stream)
        for g in self.groups:
            main.wait_stream(g.stream)

    def capture(self):
        """Captures one concurrent step as a CUDA graph (after a warm-up step)."""
        import torch
        self.step_eager()
        torch.cuda.synchronize(self.device)
        cap = torch.cuda.Stream(device=self.device)
        cap.wait_stream(torch.cuda.current_stream(self.device))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                self.step_eager()
        torch.cuda.synchronize(self.device)
        self.graph = graph
        return graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def results(self):
        """Per group: (template, rotation, shift, score) device tensors."""
        return [g.out for g in self.groups]
