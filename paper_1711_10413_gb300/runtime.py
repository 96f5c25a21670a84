"""Convenience wrapper: a context plus torch-owned device buffers.

Argument marshalling only: every call goes straight to the C ABI.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import (TEAM_STATUS_DTYPE, dsr_create, dsr_destroy, dsr_launch_region,
               dsr_region_extent, dsr_stack_init)


class Runtime:
    """A dsr context on one GPU with its stack configuration.

    slab_bytes: shared-memory slab per team (the in-smem part of the stack).
    overflow_bytes_per_team / max_teams: global overflow slab per team; the
    pool is a torch uint8 tensor owned by this object.
    """

    def __init__(self, device: int = 0, slab_bytes: int = 16384,
                 overflow_bytes_per_team: int = 0, max_teams: int = 0,
                 wait_timeout_ns: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = dsr_create(device, wait_timeout_ns)
        self.pool = None
        self.configure(slab_bytes, overflow_bytes_per_team, max_teams)

    def configure(self, slab_bytes: int, overflow_bytes_per_team: int = 0, max_teams: int = 0):
        torch = self.torch
        pool_bytes = overflow_bytes_per_team * max_teams
        if pool_bytes:
            if self.pool is None or self.pool.numel() < pool_bytes:
                self.pool = torch.empty(pool_bytes, dtype=torch.uint8,
                                        device="cuda:%d" % self.device)
        dsr_stack_init(self.ctx, slab_bytes, overflow_bytes_per_team, max_teams,
                       self.pool if pool_bytes else None, pool_bytes)
        self.slab_bytes = slab_bytes
        self.overflow_bytes_per_team = overflow_bytes_per_team
        self.max_teams = max_teams

    def close(self):
        if self.ctx:
            dsr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers ------------------------------------------------------------
    def device_buffers(self, workload):
        """Device copies of a workload's images, output and statuses."""
        torch = self.torch
        dev = "cuda:%d" % self.device
        images = torch.from_numpy(np.ascontiguousarray(workload.images)).to(dev)
        out = torch.zeros(max(workload.out_bytes, 16) // 4, dtype=torch.int32, device=dev)
        if workload.out_init is not None:
            out[: workload.out_init.size] = torch.from_numpy(workload.out_init).to(dev)
        status = torch.zeros(workload.n_status * 8, dtype=torch.int32, device=dev)
        return images, out, status

    def launch(self, region, images, out, status, stream=None):
        dsr_launch_region(self.ctx, region, images, out, status, stream)

    def run_workload(self, workload, stream=None):
        """Launch every region of a workload (plain form) and return the
        output (int32 or float32 numpy) and team statuses."""
        images, out, status = self.device_buffers(workload)
        for r in workload.regions:
            self.launch(r, images, out, status, stream)
        self.torch.cuda.synchronize(self.device)
        o = out.cpu().numpy()
        if workload.out_dtype == "float32":
            o = o.view(np.float32)
        return o, status.cpu().numpy().view(TEAM_STATUS_DTYPE)

    @staticmethod
    def extent(region):
        return dsr_region_extent(region)
