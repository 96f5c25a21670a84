"""Convenience wrapper: a context plus torch-owned device buffers.

Argument marshalling only: every call goes straight to the C ABI.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import (TEAM_STATUS_DTYPE, dsr_autotune, dsr_batch_count, dsr_batch_errors,
               dsr_batch_workspace_bytes, dsr_create, dsr_destroy, dsr_launch_batch,
               dsr_launch_region, dsr_launch_regions, dsr_region_extent,
               dsr_region_occupancy, dsr_serve_start,
               dsr_serve_stop, dsr_serve_workspace_bytes, dsr_stack_init, pack_descs)


def batch_class(descs: np.ndarray) -> str:
    """Shape class of a batch, the autotuner cache's key: its programs, the
    power of two below its instance count, and the rounded log2 of its mean
    team count, mean threads per team and mean total frame bytes per team,
    with its mean depth rounded. Batches drawn from one distribution get the
    same class (a batch near a rounding edge may not: the tuner then runs
    again); the images and outputs play no part."""
    n = max(len(descs), 1)

    def lg(v):
        return int(round(float(np.log2(max(float(np.mean(v)), 1.0)))))

    key = dict(program=sorted(set(int(p) for p in descs["program"])),
               instances=int(np.floor(np.log2(n))),
               teams=lg(descs["teams"]), threads=lg(descs["threads"]),
               frames=lg(descs["frame_bytes"].sum(axis=1)),
               depth=int(round(float(np.mean(descs["depth"])))))
    return hashlib.sha256(json.dumps(key, sort_keys=True).encode()).hexdigest()[:16]


def _load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


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

    def occupancy(self, region):
        return dsr_region_occupancy(self.ctx, region)

    @staticmethod
    def extent(region):
        return dsr_region_extent(region)

    # -- batched form ---------------------------------------------------------
    def batch_buffers(self, workload):
        """Device buffers of a batch: descriptors, images, output, statuses
        and the workspace, plus the host descriptor array and team total."""
        torch = self.torch
        dev = "cuda:%d" % self.device
        descs = pack_descs(workload.regions)
        images, out, status = self.device_buffers(workload)
        total = dsr_batch_count(descs, images.numel(), out.numel() * 4, status.numel() // 8)
        ws = torch.empty(dsr_batch_workspace_bytes(len(descs), total), dtype=torch.uint8,
                         device=dev)
        descs_dev = torch.from_numpy(descs.view(np.uint8)).to(dev)
        return dict(descs=descs, descs_dev=descs_dev, images=images, out=out, status=status,
                    ws=ws, total=total, program=int(descs["program"][0]))

    def launch_batch(self, b, tuning=None, stream=None, use_graph=False):
        dsr_launch_batch(self.ctx, b["descs_dev"], len(b["descs"]), b["program"], b["total"],
                         b["images"], b["out"], b["status"], b["ws"], tuning, stream, use_graph)

    def autotune(self, b, stream=None):
        return dsr_autotune(self.ctx, b["descs_dev"], len(b["descs"]), b["program"], b["total"],
                            b["images"], b["out"], b["status"], b["ws"], stream)

    def device_key(self) -> str:
        p = self.torch.cuda.get_device_properties(self.device)
        return "%s/%d SMs" % (p.name, p.multi_processor_count)

    def autotune_cached(self, b, path: str, stream=None, device_key=None):
        """The autotuner's choice for this batch's device and shape class
        (batch_class), from the JSON file at `path` when it holds one;
        otherwise the autotuner runs (leaving the batch's outputs computed)
        and its choice is added to the file. Returns (tuning, ms, hit); on a
        hit nothing runs and ms is the time stored with the choice."""
        key = "%s|%s" % (device_key or self.device_key(), batch_class(b["descs"]))
        entry = _load_cache(path).get(key)
        if entry:
            t = entry["tuning"]
            return (dict(threads=int(t["threads"]), slab_bytes=int(t["slab_bytes"]),
                         ctas_per_sm=int(t["ctas_per_sm"])), float(entry["ms"]), True)
        tuning, ms = self.autotune(b, stream)
        cache = _load_cache(path)
        cache[key] = dict(tuning=tuning, ms=ms)
        tmp = "%s.%d.tmp" % (path, os.getpid())
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
        return tuning, ms, False

    def launch_regions(self, b, stream=None):
        dsr_launch_regions(self.ctx, b["descs"], b["images"], b["out"], b["status"], stream)

    def batch_errors(self, b, stream=None):
        return dsr_batch_errors(self.ctx, b["ws"], stream)

    def run_batch(self, workload, tuning=None, use_graph=False):
        """Run a workload's regions as one batch; returns (out, statuses)."""
        b = self.batch_buffers(workload)
        self.launch_batch(b, tuning, use_graph=use_graph)
        self.torch.cuda.synchronize(self.device)
        return self.fetch(b, workload)

    def fetch(self, b, workload):
        o = b["out"].cpu().numpy()
        if workload.out_dtype == "float32":
            o = o.view(np.float32)
        return o, b["status"].cpu().numpy().view(TEAM_STATUS_DTYPE)

    # -- served form ----------------------------------------------------------
    def serve_start(self, workload, threads=128, slab_bytes=16384, capacity=4096,
                    idle_timeout_ns=0):
        """Start a server over a workload's buffers; returns the buffer dict
        (allocated before the server occupies the SMs)."""
        torch = self.torch
        dev = "cuda:%d" % self.device
        images, out, status = self.device_buffers(workload)
        ws = torch.empty(dsr_serve_workspace_bytes(capacity), dtype=torch.uint8, device=dev)
        torch.cuda.synchronize(self.device)
        program = workload.regions[0].program
        dsr_serve_start(self.ctx, program, images, out, status, ws, threads, slab_bytes,
                        capacity, 0, idle_timeout_ns)
        return dict(images=images, out=out, status=status, ws=ws, descs=pack_descs(workload.regions))

    def serve_stop(self):
        dsr_serve_stop(self.ctx)
