"""Ragged batches in the default split mode.

A batch whose templates carry their own FFT length (``fstat_template.n_fft``)
and output offset (``out_off``) can run in one persistent launch
(``MODE_PERSISTENT``), or, as here, grouped by FFT length: every group runs
on its own plan (one FFT shape per plan, so the batched split kernels apply)
in slices of at most ``slice_templates`` templates, and every template's 2F
lands at its ``out_off`` of one output buffer.  All calls go on one stream and
can be captured in one CUDA graph.  Grouping is host work on the template
records the caller already holds; every step of the computation is the
library's kernels.
"""
from __future__ import annotations

import numpy as np

__all__ = ["RaggedBatch"]


class RaggedBatch:
    def __init__(self, desc, x_h, templates_np, gaps=None, twoF=None, device=None,
                 slice_templates: int = 256, graph: bool = False):
        import torch
        from . import Plan, TEMPLATE_DTYPE, pack_templates
        self.device = torch.device("cuda" if device is None else device)
        tm = np.ascontiguousarray(templates_np).astype(TEMPLATE_DTYPE)
        if np.any(tm["n_fft"] <= 0) or np.any(tm["out_off"] < 0):
            raise ValueError("every template needs its n_fft and out_off")
        self.x_h, self.gaps = x_h, gaps
        total = int(np.max(tm["out_off"] + tm["n_fft"]))
        self.twoF = twoF if twoF is not None else torch.empty(total, dtype=torch.float32,
                                                              device=self.device)
        self.calls = []                       # (plan, device templates)
        self.plans = {}
        for nf in sorted(set(tm["n_fft"].tolist())):
            idx = np.nonzero(tm["n_fft"] == nf)[0]
            mt = int(min(len(idx), slice_templates))
            plan = Plan(desc.replace(n_fft=int(nf), max_templates=mt), device=self.device)
            self.plans[int(nf)] = plan
            for s0 in range(0, len(idx), mt):
                self.calls.append((plan, pack_templates(tm[idx[s0:s0 + mt]], device=self.device)))
        self.stream = torch.cuda.Stream(device=self.device)
        self.graph = None
        if graph:
            self.run()                        # first calls set kernel attributes outside the capture
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._launch()

    def _launch(self):
        from . import fstat_compute
        for plan, td in self.calls:
            fstat_compute(plan, self.x_h, td, self.gaps, self.twoF, stream=self.stream)

    def run(self):
        """Enqueue every group on the batch's stream (or replay the graph)."""
        import torch
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._launch()
        return self.twoF

    def status(self) -> int:
        """First non-zero device status of the groups' plans (0 if none)."""
        from . import fstat_status
        self.stream.synchronize()
        for plan in self.plans.values():
            rc = fstat_status(plan, self.stream, raise_error=False)
            if rc:
                return rc
        return 0

    def close(self):
        for plan in self.plans.values():
            plan.close()
        self.plans = {}
