"""Single-patch periodic driver: one step = ghost fill (periodic images) ->
CFL dt (device scalar) -> patch advance of the interior.  Two library calls
(the fill, then mhd_patch_step_cfl, whose primitive pass also reduces the
CFL dt), or three with the separate mhd_cfl_dt (cfl_in_step = False); no
host synchronisation: the dt never leaves the device, so the step can be
captured once as a CUDA graph and replayed.
"""
from __future__ import annotations

import torch

from . import capi
from .patch import Patch, periodic_copies


class PeriodicRunner:
    def __init__(self, patch: Patch, ctx, stream: torch.cuda.Stream | None = None, cfl_in_step: bool = True):
        self.patch = patch
        self.cfl_in_step = cfl_in_step
        self.ctx = ctx
        self.stream = stream or torch.cuda.current_stream(patch.state.device)
        self.descs = [patch.desc()]
        self.copies = periodic_copies(patch.n, patch.g, patch.lo)
        self.d_dt = torch.zeros(1, dtype=torch.float64, device=patch.state.device)

    @property
    def sp(self) -> int:
        return self.stream.cuda_stream

    def fill(self) -> None:
        capi.mhd_ghost_fill(self.ctx, self.descs, self.copies, self.sp)

    def step(self, dt: float | None = None) -> None:
        self.fill()
        if dt is None and self.cfl_in_step:
            capi.mhd_patch_step_cfl(self.ctx, self.descs, self.d_dt.data_ptr(), self.sp)
            return
        if dt is None:
            capi.mhd_cfl_dt(self.ctx, self.descs, self.d_dt.data_ptr(), self.sp)
        else:
            with torch.cuda.stream(self.stream):
                self.d_dt.fill_(float(dt))
        capi.mhd_patch_advance(self.ctx, self.descs, self.d_dt.data_ptr(), self.sp)

    def capture_graph(self):
        """Captures one step (fill, CFL dt, advance) as a CUDA graph; one eager
        step first puts every descriptor table on the device and sizes the
        scratch arena, so the capture uploads and allocates nothing."""
        self.step()
        torch.cuda.synchronize(self.patch.state.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.step()
        self.graph = g
        return g

    def replay(self) -> None:
        # CUDAGraph.replay launches on the current stream
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def run(self, steps: int, dt: float | None = None, record_dt: bool = False):
        dts = []
        for _ in range(steps):
            self.step(dt)
            if record_dt:
                dts.append(float(self.d_dt.item()))
        self.fill()
        return dts
