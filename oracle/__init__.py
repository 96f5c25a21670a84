"""CPU oracle for the generic-mode data-sharing runtime.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the product path may not.

`dsr_oracle.c` is a plain sequential interpreter of the region programs
under OpenMP "parallel nested in target" sharing semantics (Sec. 3.2, 4,
5.1). This module compiles it with gcc and calls it through ctypes; it
shares no code with the CUDA library (its own descriptor struct, its own
build).

`footprint.py` restates the paper's static shared-memory footprint and
occupancy arithmetic (Sec. 6.2, Tables 1-6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OVERFLOW, ERR_LIFO = 0, 1, 2, 3
MAX_LEVELS = 4


class Region(ctypes.Structure):
    _fields_ = [
        ("program", ctypes.c_uint32),
        ("teams", ctypes.c_uint32),
        ("threads", ctypes.c_uint32),
        ("depth", ctypes.c_uint32),
        ("frame_bytes", ctypes.c_uint32 * MAX_LEVELS),
        ("width", ctypes.c_uint32),
        ("param", ctypes.c_uint32),
        ("salt", ctypes.c_uint32),
        ("status_index", ctypes.c_uint32),
        ("image_offset", ctypes.c_uint64),
        ("out_offset", ctypes.c_uint64),
    ]


STATUS_DTYPE = np.dtype([("status", "<i4"), ("depth_final", "<u4"), ("hwm_bytes", "<u4"),
                         ("spill_bytes", "<u4"), ("chk", "<u4", (MAX_LEVELS,))])
assert STATUS_DTYPE.itemsize == 32 and ctypes.sizeof(Region) == 64


def _foreign(path: str) -> bool:
    """True when `path` was built for another CPU architecture."""
    import sys

    def machine(p):
        with open(p, "rb") as f:
            h = f.read(20)
        return int.from_bytes(h[18:20], "little") if h[:4] == b"\x7fELF" else -1
    return machine(path) != machine(sys.executable)


def build(force: bool = False) -> str:
    """Compile dsr_oracle.c into liboracle.so (plain gcc, -O2, no floating-point
    contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or _foreign(_LIB)
                 or os.path.getmtime(_LIB) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-Wall",
                                   "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_mix32.restype = ctypes.c_uint32
        L.orc_mix32.argtypes = [ctypes.c_uint32]
        L.orc_run.restype = ctypes.c_int
        L.orc_run.argtypes = [ctypes.POINTER(Region), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_uint32]
        L.orc_stack_new.restype = ctypes.c_void_p
        L.orc_stack_new.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_stack_free.argtypes = [ctypes.c_void_p]
        L.orc_stack_push.restype = ctypes.c_int
        L.orc_stack_push.argtypes = [ctypes.c_void_p, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_int)]
        L.orc_stack_pop.restype = ctypes.c_int
        L.orc_stack_pop.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_stack_state.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
        _lib = L
    return _lib


def mix32(x: int) -> int:
    return int(lib().orc_mix32(x & 0xFFFFFFFF))


def pack(r) -> Region:
    """Pack a region given as a dict (or an object with as_dict())."""
    d = r.as_dict() if hasattr(r, "as_dict") else dict(r)
    fb = list(d["frame_bytes"]) + [0] * MAX_LEVELS
    return Region(d["program"], d["teams"], d["threads"], d["depth"],
                  (ctypes.c_uint32 * MAX_LEVELS)(*fb[:MAX_LEVELS]), d.get("width", 0),
                  d.get("param", 0), d.get("salt", 0), d.get("status_index", 0),
                  d.get("image_offset", 0), d.get("out_offset", 0))


def run_region(region, images: np.ndarray, out: np.ndarray, status: np.ndarray,
               slab_bytes: int = 1 << 62, overflow_bytes: int = 0,
               team_begin: int = 0, team_end: Optional[int] = None) -> int:
    """Run teams [team_begin, team_end) of one region instance in place."""
    rg = pack(region)
    if team_end is None:
        team_end = rg.teams
    assert images.flags.c_contiguous and out.flags.c_contiguous
    assert status.dtype == STATUS_DTYPE
    return int(lib().orc_run(ctypes.byref(rg), images.ctypes.data, out.ctypes.data,
                             status.ctypes.data, slab_bytes, overflow_bytes,
                             team_begin, team_end))


def run_workload(wl, slab_bytes: int = 1 << 62, overflow_bytes: int = 0,
                 regions: Optional[Sequence[int]] = None):
    """Run every (or the selected) region of a workload; returns (out, status).

    The sweep program's output comes back as float64 triples per output slot
    (fp64 sum, fp64 sum of magnitudes, fp32 sum); `sweep_fields` splits them.
    """
    if wl.out_dtype == "float32":
        out = np.zeros(wl.out_bytes // 4 * 3, dtype=np.float64)
    else:
        out = np.zeros(wl.out_bytes // 4, dtype=np.int32)
        if wl.out_init is not None:
            out[: wl.out_init.size] = wl.out_init
    status = np.zeros(wl.n_status, dtype=STATUS_DTYPE)
    sel = range(len(wl.regions)) if regions is None else regions
    for i in sel:
        rc = run_region(wl.regions[i], wl.images, out, status, slab_bytes, overflow_bytes)
        if rc != OK:
            raise ValueError("oracle rejected region %d (rc=%d)" % (i, rc))
    return out, status


def sweep_fields(out: np.ndarray):
    """Split the sweep program's oracle output into its three per-slot
    values: the fp64 sum, the fp64 sum of magnitudes (for the error bound)
    and the fp32 sum in index order (float32, the program's own result)."""
    t = out.reshape(-1, 3)
    return t[:, 0], t[:, 1], t[:, 2].astype(np.float32)


class Stack:
    """The oracle's team stack, for allocator tests on the CPU."""

    def __init__(self, slab_bytes: int, overflow_bytes: int):
        self._h = lib().orc_stack_new(slab_bytes, overflow_bytes)

    def push(self, nbytes: int):
        flag = ctypes.c_int(0)
        idx = lib().orc_stack_push(self._h, nbytes, ctypes.byref(flag))
        return idx, bool(flag.value)

    def pop(self, idx: int) -> int:
        return int(lib().orc_stack_pop(self._h, idx))

    def state(self) -> dict:
        a = (ctypes.c_uint64 * 6)()
        lib().orc_stack_state(self._h, a)
        st = ctypes.c_int64(a[5]).value
        return dict(depth=a[0], slab_used=a[1], overflow_used=a[2], hwm=a[3],
                    spill_hwm=a[4], status=st)

    def close(self):
        if self._h:
            lib().orc_stack_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
