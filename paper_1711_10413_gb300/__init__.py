"""GB300 data-sharing runtime for OpenMP-style generic-mode regions.

Thin ctypes binding of libdsr.so (the C ABI declared in include/dsr.h).
The functions keep the C names and only marshal arguments; every step of a
region runs in the library's CUDA kernels. PyTorch supplies device memory
(tensor data pointers) and streams. There is no CPU fallback: loading fails
loudly when libdsr.so has not been built (see `build()`).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdsr.so")

DSR_OK, DSR_ERR_INVALID, DSR_ERR_OVERFLOW, DSR_ERR_LIFO = 0, 1, 2, 3
DSR_ERR_BUDGET, DSR_ERR_TIMEOUT, DSR_ERR_CUDA = 4, 5, 6
DSR_MAX_DEPTH = 4
DSR_MAX_FRAMES = 8
DSR_PENDING = -1
DSR_SLAB_AUTO = 0xFFFFFFFF
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OVERFLOW", 3: "LIFO", 4: "BUDGET", 5: "TIMEOUT",
                6: "CUDA"}

DSR_PROG_PAPER_SCALARS = 1
DSR_PROG_PAPER_ARRAYS = 2
DSR_PROG_SCALARS = 3
DSR_PROG_NESTED = 4
DSR_PROG_SWEEP = 5
DSR_PROG_HETERO = 6
DSR_PROG_WORKERS = 7
DSR_PROG_USER = 256


class dsr_region_desc(ctypes.Structure):
    _fields_ = [("program", ctypes.c_uint32), ("teams", ctypes.c_uint32),
                ("threads", ctypes.c_uint32), ("depth", ctypes.c_uint32),
                ("frame_bytes", ctypes.c_uint32 * DSR_MAX_DEPTH), ("width", ctypes.c_uint32),
                ("param", ctypes.c_uint32), ("salt", ctypes.c_uint32),
                ("status_index", ctypes.c_uint32), ("image_offset", ctypes.c_uint64),
                ("out_offset", ctypes.c_uint64)]


class dsr_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("wait_timeout_ns", ctypes.c_uint64)]


class dsr_batch_tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("slab_bytes", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class dsr_region_buffers(ctypes.Structure):
    _fields_ = [("images_dev", ctypes.c_void_p), ("image_bytes", ctypes.c_uint64),
                ("out_dev", ctypes.c_void_p), ("out_bytes", ctypes.c_uint64),
                ("status_dev", ctypes.c_void_p), ("n_status", ctypes.c_uint64)]


class dsr_serve_program(ctypes.Structure):
    """Hooks of a user-written program's server (filled in by the device
    API's dsr_serve_user_start in the program's own library)."""
    _fields_ = [("program", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("validate", ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64,
                                              ctypes.c_uint64, ctypes.c_uint64)),
                ("prepare", ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.POINTER(ctypes.c_int32))),
                ("launch", ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p))]


class dsr_serve_cfg(ctypes.Structure):
    _fields_ = [("program", ctypes.c_uint32), ("threads", ctypes.c_uint32),
                ("slab_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("capacity", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("idle_timeout_ns", ctypes.c_uint64), ("images_dev", ctypes.c_void_p),
                ("image_bytes", ctypes.c_uint64), ("out_dev", ctypes.c_void_p),
                ("out_bytes", ctypes.c_uint64), ("status_dev", ctypes.c_void_p),
                ("n_status", ctypes.c_uint64)]


class dsr_plain_config(ctypes.Structure):
    _fields_ = [("pool_dev", ctypes.c_void_p), ("ovf_per_team", ctypes.c_uint64),
                ("timeout_ns", ctypes.c_uint64), ("slab_bytes", ctypes.c_uint32),
                ("ctrl_bytes", ctypes.c_uint32), ("device", ctypes.c_int32),
                ("max_smem", ctypes.c_uint32)]


class dsr_batch_plan(ctypes.Structure):
    _fields_ = [("descs", ctypes.c_void_p), ("tasks", ctypes.c_void_p), ("hdr", ctypes.c_void_p),
                ("images", ctypes.c_void_p), ("out", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("pool", ctypes.c_void_p), ("capacity", ctypes.c_uint64),
                ("image_bytes", ctypes.c_uint64), ("out_bytes", ctypes.c_uint64),
                ("n_status", ctypes.c_uint64), ("ovf_per_cta", ctypes.c_uint64),
                ("timeout_ns", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("slab_bytes", ctypes.c_uint32), ("grid", ctypes.c_uint32),
                ("threads", ctypes.c_uint32)]


class dsr_smem_probe(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint64), ("ms", ctypes.c_double), ("gbs", ctypes.c_double),
                ("sm_mhz", ctypes.c_double), ("bytes_per_clk_sm", ctypes.c_double),
                ("ctas", ctypes.c_uint32), ("threads", ctypes.c_uint32)]


class dsr_footprint(ctypes.Structure):
    _fields_ = [("smem_per_team", ctypes.c_uint32), ("ctrl_bytes", ctypes.c_uint32),
                ("slab_bytes", ctypes.c_uint32), ("teams_per_sm", ctypes.c_uint32),
                ("limit", ctypes.c_uint32), ("spill_bytes", ctypes.c_uint32)]


class dsr_occupancy(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_uint32), ("regs_per_thread", ctypes.c_uint32),
                ("smem_per_team", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("sm_count", ctypes.c_uint32), ("spill_bytes", ctypes.c_uint32)]


TEAM_STATUS_DTYPE = np.dtype([("status", "<i4"), ("depth_final", "<u4"), ("hwm_bytes", "<u4"),
                              ("spill_bytes", "<u4"), ("chk", "<u4", (DSR_MAX_DEPTH,))])
assert ctypes.sizeof(dsr_region_desc) == 64 and TEAM_STATUS_DTYPE.itemsize == 32

DESC_DTYPE = np.dtype([("program", "<u4"), ("teams", "<u4"), ("threads", "<u4"),
                       ("depth", "<u4"), ("frame_bytes", "<u4", (DSR_MAX_DEPTH,)),
                       ("width", "<u4"), ("param", "<u4"), ("salt", "<u4"),
                       ("status_index", "<u4"), ("image_offset", "<u8"),
                       ("out_offset", "<u8")])
assert DESC_DTYPE.itemsize == 64


class DsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


_lib = None
_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32


def _declare(L):
    P = ctypes.POINTER
    sig = {
        "dsr_create": (_i32, [P(_vp), P(dsr_config)]),
        "dsr_destroy": (_i32, [_vp]),
        "dsr_last_error_string": (ctypes.c_char_p, [_vp]),
        "dsr_stack_init": (_i32, [_vp, _u32, _u64, _u32, _vp, _u64]),
        "dsr_validate_region": (_i32, [P(dsr_region_desc), _u64, _u64, _u64]),
        "dsr_region_extent": (_i32, [P(dsr_region_desc), P(_u64), P(_u64), P(_u64)]),
        "dsr_footprint_model": (_i32, [P(dsr_region_desc), _u32, _u32, P(dsr_footprint)]),
        "dsr_region_occupancy": (_i32, [_vp, P(dsr_region_desc), P(dsr_occupancy)]),
        "dsr_region_footprint": (_i32, [P(dsr_region_desc), P(_u64), P(_u64)]),
        "dsr_launch_region": (_i32, [_vp, P(dsr_region_desc), _vp, _u64, _vp, _u64, _vp, _u64,
                                     _vp]),
        "dsr_run_region_host": (_i32, [_vp, P(dsr_region_desc), _vp, _u64, _vp, _u64, _vp,
                                       _vp, _vp, _vp, _vp]),
        "dsr_enqueue_region_host": (_i32, [_vp, P(dsr_region_desc), _vp, _u64, _vp, _u64, _vp,
                                           _vp, _vp, _vp, _vp]),
        "dsr_check_bounded_wait": (_i32, [_vp, _u64, _vp, _vp]),
        "dsr_check_stack": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp]),
        "dsr_probe_smem_bandwidth": (_i32, [_vp, _u32, _vp, _vp, P(dsr_smem_probe)]),
        "dsr_batch_workspace_bytes": (_u64, [_u32, _u64]),
        "dsr_batch_count": (_i32, [_vp, _u32, _u64, _u64, _u64, P(_u64)]),
        "dsr_launch_batch": (_i32, [_vp, _vp, _u32, _u32, _u64, _vp, _u64, _vp, _u64, _vp, _u64,
                                    _vp, _u64, P(dsr_batch_tuning), _vp, ctypes.c_int]),
        "dsr_batch_errors": (_i32, [_vp, _vp, P(_u32), P(_u64), _vp]),
        "dsr_autotune": (_i32, [_vp, _vp, _u32, _u32, _u64, _vp, _u64, _vp, _u64, _vp, _u64, _vp,
                                _u64, _vp, P(dsr_batch_tuning), P(ctypes.c_float)]),
        "dsr_launch_regions": (_i32, [_vp, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _u64, _vp]),
        "dsr_launch_batch_static": (_i32, [_vp, _vp, _u32, _u32, _u64, _vp, _u64, _vp, _u64,
                                           _vp, _u64, P(dsr_batch_tuning), _vp]),
        "dsr_batch_static_capacity": (_u64, []),
        "dsr_batch_static_errors": (_i32, [_vp, P(_u32), P(_u64), _vp]),
        "dsr_batch_abort": (_i32, [_vp, _vp]),
        "dsr_batch_progress": (_i32, [_vp, _vp, P(_u64), P(_u64), _vp]),
        "dsr_report_error": (_i32, [_vp, _i32, ctypes.c_char_p]),
        "dsr_user_plain_config": (_i32, [_vp, P(dsr_region_desc), _u64, _u64, _u64, _u64, _u64,
                                         _vp, _vp, P(dsr_plain_config)]),
        "dsr_batch_prepare": (_i32, [_vp, _vp, _u32, _u32, _u64, _vp, _u64, _vp, _u64, _vp,
                                     _u64, _vp, _u64, _u32, _u32, _u32, _vp,
                                     P(dsr_batch_plan)]),
        "dsr_serve_workspace_bytes": (_u64, [_u32]),
        "dsr_graph_capture_regions": (_i32, [_vp, P(dsr_region_desc), P(dsr_region_buffers), _u32,
                                              P(_vp)]),
        "dsr_graph_launch": (_i32, [_vp, _vp, _vp]),
        "dsr_graph_destroy": (_i32, [_vp]),
        "dsr_serve_start": (_i32, [_vp, P(dsr_serve_cfg), _vp, _u64]),
        "dsr_serve_start_user": (_i32, [_vp, P(dsr_serve_cfg), _vp, _u64, P(dsr_serve_program)]),
        "dsr_serve_submit": (_i32, [_vp, P(dsr_region_desc), P(_u64)]),
        "dsr_serve_poll": (_i32, [_vp, _u64, P(_i32)]),
        "dsr_serve_stop": (_i32, [_vp]),
        "dsr_serve_stats": (_i32, [_vp, P(_u64), P(_u64), P(_u32), P(_u32)]),
        "dsr_serve_bench": (_i32, [_vp, _vp, _u32, _vp, _vp, P(ctypes.c_int64)]),
        "dsr_launch_bench": (_i32, [_vp, _vp, _u32, _vp, _vp, P(ctypes.c_int64), _vp, _u64, _vp,
                                    _u64, _vp, _u64, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    return L


def lib():
    """The loaded libdsr.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdsr.so is missing: build it with "
                              "paper_1711_10413_gb300.build() (nvcc, sm_103a)")
        _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def build(force: bool = False) -> str:
    from . import builder
    return builder.build(force=force)


def exported_symbols():
    return ["dsr_create", "dsr_destroy", "dsr_last_error_string", "dsr_stack_init",
            "dsr_validate_region", "dsr_region_extent", "dsr_footprint_model",
            "dsr_region_occupancy", "dsr_region_footprint",
            "dsr_launch_region", "dsr_run_region_host", "dsr_enqueue_region_host",
            "dsr_batch_workspace_bytes",
            "dsr_batch_count", "dsr_launch_batch", "dsr_batch_errors", "dsr_autotune",
            "dsr_launch_regions", "dsr_launch_batch_static", "dsr_batch_static_capacity",
            "dsr_batch_static_errors", "dsr_batch_abort", "dsr_batch_progress",
            "dsr_report_error", "dsr_user_plain_config",
            "dsr_batch_prepare",
            "dsr_graph_capture_regions", "dsr_graph_launch", "dsr_graph_destroy",
            "dsr_serve_workspace_bytes", "dsr_serve_start", "dsr_serve_start_user",
            "dsr_serve_submit", "dsr_serve_poll", "dsr_serve_stop", "dsr_serve_stats",
            "dsr_serve_bench", "dsr_launch_bench", "dsr_check_bounded_wait",
            "dsr_check_stack", "dsr_probe_smem_bandwidth"]


# ---------------------------------------------------------------------------
# Marshalling helpers
# ---------------------------------------------------------------------------
def pack_desc(r) -> dsr_region_desc:
    """A dsr_region_desc from a dict or an object with as_dict()."""
    d = r.as_dict() if hasattr(r, "as_dict") else dict(r)
    fb = list(d["frame_bytes"]) + [0] * DSR_MAX_DEPTH
    return dsr_region_desc(d["program"], d["teams"], d["threads"], d["depth"],
                           (ctypes.c_uint32 * DSR_MAX_DEPTH)(*fb[:DSR_MAX_DEPTH]),
                           d.get("width", 0), d.get("param", 0), d.get("salt", 0),
                           d.get("status_index", 0), d.get("image_offset", 0),
                           d.get("out_offset", 0))


def pack_descs(regions) -> np.ndarray:
    """A DESC_DTYPE array (bytes identical to dsr_region_desc[])."""
    a = np.zeros(len(regions), dtype=DESC_DTYPE)
    for i, r in enumerate(regions):
        d = r.as_dict() if hasattr(r, "as_dict") else dict(r)
        fb = list(d["frame_bytes"]) + [0] * DSR_MAX_DEPTH
        a[i] = (d["program"], d["teams"], d["threads"], d["depth"], fb[:DSR_MAX_DEPTH],
                d.get("width", 0), d.get("param", 0), d.get("salt", 0),
                d.get("status_index", 0), d.get("image_offset", 0), d.get("out_offset", 0))
    return a


def _ptr(x) -> Optional[int]:
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _check(rc: int, ctx=None):
    if rc != DSR_OK:
        msg = lib().dsr_last_error_string(ctx)
        raise DsrError(rc, msg.decode() if msg else "")
    return rc


# ---------------------------------------------------------------------------
# The C ABI, name for name
# ---------------------------------------------------------------------------
def dsr_create(device: int = 0, wait_timeout_ns: int = 0) -> int:
    h = ctypes.c_void_p()
    cfg = dsr_config(device, 0, wait_timeout_ns)
    _check(lib().dsr_create(ctypes.byref(h), ctypes.byref(cfg)))
    return h.value


def dsr_destroy(ctx: int) -> None:
    lib().dsr_destroy(ctx)


def dsr_last_error_string(ctx: Optional[int] = None) -> str:
    s = lib().dsr_last_error_string(ctx)
    return s.decode() if s else ""


def dsr_stack_init(ctx: int, smem_slab_bytes: int, overflow_bytes_per_team: int = 0,
                   max_teams: int = 0, overflow_pool=None, pool_bytes: int = 0) -> None:
    _check(lib().dsr_stack_init(ctx, smem_slab_bytes, overflow_bytes_per_team, max_teams,
                                _ptr(overflow_pool), pool_bytes), ctx)


def dsr_validate_region(region, image_bytes: int, out_bytes: int, n_status: int) -> int:
    d = pack_desc(region)
    return int(lib().dsr_validate_region(ctypes.byref(d), image_bytes, out_bytes, n_status))


def dsr_region_extent(region):
    d = pack_desc(region)
    a, b, c = _u64(), _u64(), _u64()
    _check(lib().dsr_region_extent(ctypes.byref(d), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(c)))
    return a.value, b.value, c.value


def dsr_footprint_model(region, slab_bytes: int, regs: int = 0) -> dict:
    d = pack_desc(region)
    f = dsr_footprint()
    _check(lib().dsr_footprint_model(ctypes.byref(d), slab_bytes, regs, ctypes.byref(f)))
    return {k: getattr(f, k) for k, _ in dsr_footprint._fields_}


def dsr_region_footprint(region):
    """(peak stack bytes, slab bytes that hold every frame) of a region."""
    d = pack_desc(region)
    a, b = _u64(), _u64()
    _check(lib().dsr_region_footprint(ctypes.byref(d), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def dsr_region_occupancy(ctx: int, region) -> dict:
    """Registers, shared memory per team and resident teams per SM of the
    plain launch of `region` with the ctx's stack configuration."""
    d = pack_desc(region)
    o = dsr_occupancy()
    _check(lib().dsr_region_occupancy(ctx, ctypes.byref(d), ctypes.byref(o)), ctx)
    return {k: getattr(o, k) for k, _ in dsr_occupancy._fields_}


def _nbytes(x) -> int:
    if hasattr(x, "element_size"):
        return x.numel() * x.element_size()
    return int(x.nbytes)


def dsr_launch_region(ctx: int, region, images, out, status, stream=None) -> None:
    """images / out / status: device tensors (their sizes are passed on)."""
    d = pack_desc(region)
    _check(lib().dsr_launch_region(ctx, ctypes.byref(d), _ptr(images),
                                   _nbytes(images) if images is not None else 0, _ptr(out),
                                   _nbytes(out), _ptr(status), _nbytes(status) // 32,
                                   _stream(stream)), ctx)


def dsr_graph_capture_regions(ctx: int, regions, buffers) -> int:
    """A launch graph of len(regions) plain launches, region i on buffers[i]
    = (images, out, status) device tensors; returns the graph handle
    (dsr_graph_destroy frees it)."""
    n = len(regions)
    descs = (dsr_region_desc * n)(*[pack_desc(r) for r in regions])
    bufs = (dsr_region_buffers * n)()
    for i, (images, out, status) in enumerate(buffers):
        bufs[i] = dsr_region_buffers(_ptr(images), _nbytes(images) if images is not None else 0,
                                     _ptr(out), _nbytes(out), _ptr(status), _nbytes(status) // 32)
    g = ctypes.c_void_p()
    _check(lib().dsr_graph_capture_regions(ctx, descs, bufs, n, ctypes.byref(g)), ctx)
    return g.value


def dsr_graph_launch(ctx: int, graph: int, stream=None) -> None:
    _check(lib().dsr_graph_launch(ctx, graph, _stream(stream)), ctx)


def dsr_graph_destroy(graph: int) -> None:
    lib().dsr_graph_destroy(graph)


def dsr_run_region_host(ctx: int, region, images_host, image_bytes: int, out_host,
                        out_bytes: int, status_host, images_dev, out_dev, status_dev,
                        stream=None) -> None:
    d = pack_desc(region)
    _check(lib().dsr_run_region_host(ctx, ctypes.byref(d), _ptr(images_host), image_bytes,
                                     _ptr(out_host), out_bytes, _ptr(status_host),
                                     _ptr(images_dev), _ptr(out_dev), _ptr(status_dev),
                                     _stream(stream)), ctx)


def dsr_enqueue_region_host(ctx: int, region, images_host, image_bytes: int, out_host,
                            out_bytes: int, status_host, images_dev, out_dev, status_dev,
                            stream=None) -> None:
    """dsr_run_region_host without the synchronisation (pinned host buffers)."""
    d = pack_desc(region)
    _check(lib().dsr_enqueue_region_host(ctx, ctypes.byref(d), _ptr(images_host), image_bytes,
                                         _ptr(out_host), out_bytes, _ptr(status_host),
                                         _ptr(images_dev), _ptr(out_dev), _ptr(status_dev),
                                         _stream(stream)), ctx)


def dsr_check_bounded_wait(ctx: int, timeout_ns: int, result, stream=None) -> None:
    """result: a device tensor of two int64 (or more bytes): receives
    {status, elapsed ns} of a device wait that nothing completes."""
    if result is None or _nbytes(result) < 16:
        raise ValueError("result must hold two 64-bit words")
    _check(lib().dsr_check_bounded_wait(ctx, timeout_ns, _ptr(result), _stream(stream)), ctx)


def dsr_check_stack(ctx: int, result, scratch, stream=None) -> None:
    """result: a device tensor of at least 25 int64; scratch: at least 64
    device bytes (the check's overflow slab)."""
    _check(lib().dsr_check_stack(ctx, _ptr(result), _nbytes(result) // 8, _ptr(scratch),
                                 _nbytes(scratch), _stream(stream)), ctx)


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, dsr_batch_tuning):
        return ctypes.byref(t)
    d = dict(t)
    return ctypes.byref(dsr_batch_tuning(d.get("threads", 256), d.get("slab_bytes", 16384),
                                         d.get("ctas_per_sm", 0), 0))


def dsr_batch_workspace_bytes(n: int, total_teams: int) -> int:
    return int(lib().dsr_batch_workspace_bytes(n, total_teams))


def dsr_batch_count(descs: np.ndarray, image_bytes: int, out_bytes: int, n_status: int) -> int:
    """descs: DESC_DTYPE host array. Returns the total team count."""
    t = _u64()
    _check(lib().dsr_batch_count(descs.ctypes.data, len(descs), image_bytes, out_bytes,
                                 n_status, ctypes.byref(t)))
    return t.value


def dsr_launch_batch(ctx: int, descs_dev, n: int, program: int, total_teams: int, images, out,
                     status, workspace, tuning=None, stream=None, use_graph: bool = False):
    """descs_dev / images / out / status / workspace: device tensors."""
    _check(lib().dsr_launch_batch(ctx, _ptr(descs_dev), n, program, total_teams, _ptr(images),
                                  _nbytes(images) if images is not None else 0, _ptr(out),
                                  _nbytes(out), _ptr(status), _nbytes(status) // 32,
                                  _ptr(workspace), _nbytes(workspace), _tuning(tuning),
                                  _stream(stream), 1 if use_graph else 0), ctx)


def dsr_launch_batch_static(ctx: int, descs_dev, n: int, program: int, total_teams: int,
                            images, out, status, tuning=None, stream=None):
    """The batched launch with its workspace in the library's fixed device
    array (no workspace argument, nothing allocated)."""
    _check(lib().dsr_launch_batch_static(ctx, _ptr(descs_dev), n, program, total_teams,
                                         _ptr(images),
                                         _nbytes(images) if images is not None else 0,
                                         _ptr(out), _nbytes(out), _ptr(status),
                                         _nbytes(status) // 32, _tuning(tuning),
                                         _stream(stream)), ctx)


def dsr_batch_static_capacity() -> int:
    return int(lib().dsr_batch_static_capacity())


def dsr_batch_static_errors(ctx: int, stream=None):
    """(tasks rejected on the device, tasks counted) of the last
    dsr_launch_batch_static on the ctx's device (synchronises `stream`)."""
    e, t = _u32(), _u64()
    _check(lib().dsr_batch_static_errors(ctx, ctypes.byref(e), ctypes.byref(t),
                                         _stream(stream)), ctx)
    return int(e.value), int(t.value)


def dsr_probe_smem_bandwidth(ctx: int, reps: int, scratch, stream=None) -> dict:
    """Measured shared-memory bandwidth (scratch: device tensor of at least
    32 bytes); synchronises `stream`."""
    r = dsr_smem_probe()
    _check(lib().dsr_probe_smem_bandwidth(ctx, reps, _ptr(scratch), _stream(stream),
                                          ctypes.byref(r)), ctx)
    return {f: getattr(r, f) for f, _ in dsr_smem_probe._fields_}


def dsr_batch_abort(ctx: int, workspace=None) -> None:
    """Ask the batch running on `workspace` (None: the static workspace) to
    stop after its CTAs' next grabs; does not wait."""
    _check(lib().dsr_batch_abort(ctx, _ptr(workspace)), ctx)


def dsr_batch_progress(ctx: int, workspace=None, stream=None):
    """(tasks taken, tasks counted) of the last batch on `workspace`."""
    t, c = _u64(), _u64()
    _check(lib().dsr_batch_progress(ctx, _ptr(workspace), ctypes.byref(t), ctypes.byref(c),
                                    _stream(stream)), ctx)
    return int(t.value), int(c.value)


def dsr_report_error(ctx: int, code: int, msg: str) -> int:
    return int(lib().dsr_report_error(ctx, code, msg.encode()))


def dsr_user_plain_config(ctx: int, region, image_need: int, out_need: int, image_bytes: int,
                          out_bytes: int, n_status: int, out, status) -> dict:
    """The checks and stack configuration of a plain launch of a user-written
    program (what dsr_launch_user_region passes to its kernel)."""
    c = dsr_plain_config()
    _check(lib().dsr_user_plain_config(ctx, ctypes.byref(pack_desc(region)), image_need,
                                       out_need, image_bytes, out_bytes, n_status, _ptr(out),
                                       _ptr(status), ctypes.byref(c)), ctx)
    return {f: getattr(c, f) for f, _ in dsr_plain_config._fields_}


def dsr_batch_errors(ctx: int, workspace, stream=None):
    e, t = _u32(), _u64()
    _check(lib().dsr_batch_errors(ctx, _ptr(workspace), ctypes.byref(e), ctypes.byref(t),
                                  _stream(stream)), ctx)
    return e.value, t.value


def dsr_autotune(ctx: int, descs_dev, n: int, program: int, total_teams: int, images, out,
                 status, workspace, stream=None):
    best = dsr_batch_tuning()
    ms = ctypes.c_float()
    _check(lib().dsr_autotune(ctx, _ptr(descs_dev), n, program, total_teams, _ptr(images),
                              _nbytes(images) if images is not None else 0, _ptr(out),
                              _nbytes(out), _ptr(status), _nbytes(status) // 32,
                              _ptr(workspace), _nbytes(workspace), _stream(stream),
                              ctypes.byref(best), ctypes.byref(ms)), ctx)
    return dict(threads=best.threads, slab_bytes=best.slab_bytes,
                ctas_per_sm=best.ctas_per_sm), ms.value


def dsr_launch_regions(ctx: int, descs: np.ndarray, images, out, status, stream=None):
    """descs: DESC_DTYPE host array; one plain launch per region."""
    _check(lib().dsr_launch_regions(ctx, descs.ctypes.data, len(descs), _ptr(images),
                                    _nbytes(images) if images is not None else 0, _ptr(out),
                                    _nbytes(out), _ptr(status), _nbytes(status) // 32,
                                    _stream(stream)), ctx)


def dsr_serve_workspace_bytes(capacity: int) -> int:
    return int(lib().dsr_serve_workspace_bytes(capacity))


def dsr_serve_start(ctx: int, program: int, images, out, status, workspace, threads: int = 128,
                    slab_bytes: int = 16384, capacity: int = 4096, ctas_per_sm: int = 0,
                    idle_timeout_ns: int = 0) -> None:
    cfg = serve_cfg(program, images, out, status, threads, slab_bytes, capacity, ctas_per_sm,
                    idle_timeout_ns)
    _check(lib().dsr_serve_start(ctx, ctypes.byref(cfg), _ptr(workspace), _nbytes(workspace)),
           ctx)


def serve_cfg(program: int, images, out, status, threads: int = 128, slab_bytes: int = 16384,
              capacity: int = 4096, ctas_per_sm: int = 0, idle_timeout_ns: int = 0):
    """A dsr_serve_cfg over the given device buffers."""
    return dsr_serve_cfg(program, threads, slab_bytes, ctas_per_sm, capacity, 0, idle_timeout_ns,
                         _ptr(images), _nbytes(images) if images is not None else 0, _ptr(out),
                         _nbytes(out), _ptr(status), _nbytes(status) // 32)


def dsr_serve_start_user(ctx: int, cfg, workspace, prog) -> None:
    """Serve a user-written program: `prog` a dsr_serve_program (its hooks
    from the program's library)."""
    _check(lib().dsr_serve_start_user(ctx, ctypes.byref(cfg), _ptr(workspace),
                                      _nbytes(workspace), ctypes.byref(prog)), ctx)


def dsr_serve_submit(ctx: int, region):
    """Returns the ticket, or None when admission must wait (DSR_ERR_BUDGET)."""
    d = pack_desc(region)
    t = _u64()
    rc = lib().dsr_serve_submit(ctx, ctypes.byref(d), ctypes.byref(t))
    if rc == DSR_ERR_BUDGET:
        return None
    _check(rc, ctx)
    return t.value


def dsr_serve_poll(ctx: int, ticket: int) -> int:
    st = _i32()
    _check(lib().dsr_serve_poll(ctx, ticket, ctypes.byref(st)), ctx)
    return st.value


def dsr_serve_stop(ctx: int) -> None:
    _check(lib().dsr_serve_stop(ctx), ctx)


def dsr_serve_stats(ctx: int) -> dict:
    a, b, c, d = _u64(), _u64(), _u32(), _u32()
    _check(lib().dsr_serve_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                 ctypes.byref(d)), ctx)
    return dict(submitted=a.value, completed=b.value, idle_exits=c.value, errors=d.value)


def dsr_serve_bench(ctx: int, descs: np.ndarray, arrival_ns: np.ndarray):
    """Open-loop run on a started server; returns (latency_ns[], elapsed_ns)."""
    arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    lat = np.zeros(len(descs), dtype=np.int64)
    el = ctypes.c_int64()
    _check(lib().dsr_serve_bench(ctx, descs.ctypes.data, len(descs), arr.ctypes.data,
                                 lat.ctypes.data, ctypes.byref(el)), ctx)
    return lat, el.value


def dsr_launch_bench(ctx: int, descs: np.ndarray, arrival_ns: np.ndarray, images, out, status,
                     stream=None):
    arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
    lat = np.zeros(len(descs), dtype=np.int64)
    el = ctypes.c_int64()
    _check(lib().dsr_launch_bench(ctx, descs.ctypes.data, len(descs), arr.ctypes.data,
                                  lat.ctypes.data, ctypes.byref(el), _ptr(images),
                                  _nbytes(images) if images is not None else 0, _ptr(out),
                                  _nbytes(out), _ptr(status), _nbytes(status) // 32,
                                  _stream(stream)), ctx)
    return lat, el.value


from .runtime import Runtime  # noqa: E402  (convenience wrapper over the calls above)
