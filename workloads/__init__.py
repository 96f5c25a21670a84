"""Seeded synthetic workloads for the generic-mode data-sharing runtime.

This module is the ONE piece shared by the CPU oracle and the CUDA path. It
holds only random-number generation and buffer layout (where each instance's
init image and output live); it contains none of the method's arithmetic
(no stack allocation, no frame fills, no region bodies, no hashing of frame
data). Every random value a region program consumes is drawn here, on the
host, and handed to both sides as plain integers and numpy arrays.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). The i-th output (1-based) of
a stream with state s is mix64(s + i * GAMMA); that closed form lets numpy
draw a whole stream at once.

Region programs (see the oracle for their semantics):
  PX1 "paper scalars"  - the paper's program that shares n scalars and the
                         array reference (Sec. 6.1, Fig. "8 variables").
  PX2 "paper arrays"   - the paper's program that shares k int[W] arrays
                         (Sec. 6.1, Fig. "arrays").
  P1  "scalars"        - 1 team x 128 threads, many sequential regions, a
                         4 x int32 frame drawn U[0, 2^20).
  P2  "nested"         - 1024 teams x 256 threads, 3 nested levels, frames
                         of 16 int32 scalars + int32[256].
  P3  "sweep"          - 512 teams x 128 threads, one FP32 frame of S bytes
                         with N(0,1) values.
  P4  "hetero"         - heterogeneous instances (log-uniform teams and
                         frame sizes, uniform threads and depth).
  P5  "workers"        - worker-level sharing: every worker pushes its own
                         frame of S bytes for a nested region on its warp.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

DEFAULT_SEED = 171110413

# Program identifiers; both sides use these numbers on the wire.
PROG_PAPER_SCALARS = 1
PROG_PAPER_ARRAYS = 2
PROG_SCALARS = 3
PROG_NESTED = 4
PROG_SWEEP = 5
PROG_HETERO = 6
PROG_WORKERS = 7

MAX_DEPTH = 4
NESTED_FRAME_WORDS = 16 + 256  # int32 s[16]; int32 arr[256]
NESTED_FRAME_BYTES = 4 * NESTED_FRAME_WORDS

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


# ----------------------------------------------------------------------------
# SplitMix64
# ----------------------------------------------------------------------------
def _mix64_scalar(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_outputs(state: int, n: int) -> np.ndarray:
    """First n outputs of the SplitMix64 stream whose state is `state`."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & _M64) + i * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def derive(seed: int, *keys: int) -> int:
    """Stream state for a (config, instance, team, level, ...) key path."""
    h = seed & _M64
    for k in keys:
        h = _mix64_scalar((h ^ (k & _M64)) + _GAMMA)
    return h


def uniform_u32(state: int, n: int, bits: int = 32) -> np.ndarray:
    """n integers uniform in [0, 2^bits), from the high bits of each output."""
    x = splitmix64_outputs(state, n) >> np.uint64(64 - bits)
    return x.astype(np.uint32)


def uniform_f64(state: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1) with 53 random bits."""
    x = splitmix64_outputs(state, n) >> np.uint64(11)
    return x.astype(np.float64) * (1.0 / (1 << 53))


def normal_f32(state: int, n: int) -> np.ndarray:
    """n N(0,1) values: Box-Muller in double, rounded once to float32."""
    m = (n + 1) // 2
    u = splitmix64_outputs(state, 2 * m) >> np.uint64(11)
    u1 = (u[0::2].astype(np.float64) + 1.0) * (1.0 / (1 << 53))  # (0, 1]
    u2 = u[1::2].astype(np.float64) * (1.0 / (1 << 53))
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n].astype(np.float32)


def log_uniform_int(state: int, n: int, lo: int, hi: int) -> np.ndarray:
    """floor(exp(U(ln lo, ln(hi+1)))) clamped to [lo, hi]."""
    u = uniform_f64(state, n)
    x = np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo))))
    return np.clip(x, lo, hi).astype(np.int64)


# ----------------------------------------------------------------------------
# Region descriptors (plain data; each side packs its own struct)
# ----------------------------------------------------------------------------
@dataclass
class Region:
    program: int
    teams: int
    threads: int
    depth: int
    frame_bytes: List[int]
    width: int = 0          # threads of each parallel region; 0 = every worker
    param: int = 0
    salt: int = 0
    status_index: int = 0
    image_offset: int = 0
    out_offset: int = 0

    @property
    def workers(self) -> int:
        """W = threads - 32 (the last warp is the master warp)."""
        return self.threads - 32

    @property
    def team_width(self) -> int:
        """Threads that run each parallel region: `width` when set, else W
        (or 1 when W == 0: the region runs as a team of one)."""
        return self.width if self.width else max(self.threads - 32, 1)

    def as_dict(self) -> dict:
        fb = list(self.frame_bytes) + [0] * (MAX_DEPTH - len(self.frame_bytes))
        return dict(program=self.program, teams=self.teams, threads=self.threads,
                    depth=self.depth, frame_bytes=fb, width=self.width,
                    param=self.param, salt=self.salt, status_index=self.status_index,
                    image_offset=self.image_offset, out_offset=self.out_offset)


@dataclass
class Workload:
    """Regions plus the buffers they read and write.

    images:  bytes read by the masters' sequential code (uint8 view).
    out_init: initial output contents (programs PX1/PX2 update in place);
              None means the output starts zeroed.
    out_bytes / n_status: sizes of the output and team-status arrays.
    """
    name: str
    regions: List[Region]
    images: np.ndarray
    out_bytes: int
    n_status: int
    out_dtype: str = "int32"
    out_init: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)


def _pad16(n: int) -> int:
    return (n + 15) & ~15


def _as_bytes(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a).view(np.uint8).reshape(-1)


# ----------------------------------------------------------------------------
# Paper programs (Sec. 6.1)
# ----------------------------------------------------------------------------
def paper_scalars(n_vars: int = 7, teams: int = 4, threads: int = 128,
                  seed: int = DEFAULT_SEED) -> Workload:
    """The paper's scalar-sharing program: n shared ints plus the array ref.

    Frame layout: int32 c[n], padded to 8 bytes, then one 8-byte pointer.
    The initial array contents are random so the update is observable.
    """
    w = max(threads - 32, 1)
    fb = ((4 * n_vars + 7) & ~7) + 8
    r = Region(PROG_PAPER_SCALARS, teams, threads, 1, [fb], param=n_vars)
    a0 = uniform_u32(derive(seed, 0xA1, n_vars), teams * w).view(np.int32)
    return Workload("paper_scalars", [r], np.zeros(16, np.uint8), 4 * teams * w,
                    teams, out_init=a0.copy())


def paper_arrays(n_arrays: int = 1, teams: int = 4, threads: int = 128,
                 seed: int = DEFAULT_SEED) -> Workload:
    """The paper's array-sharing program: k arrays int d[W] shared."""
    w = max(threads - 32, 1)
    r = Region(PROG_PAPER_ARRAYS, teams, threads, 1, [4 * n_arrays * w], param=n_arrays)
    a0 = uniform_u32(derive(seed, 0xA2, n_arrays), teams * w).view(np.int32)
    return Workload("paper_arrays", [r], np.zeros(16, np.uint8), 4 * teams * w,
                    teams, out_init=a0.copy())


# ----------------------------------------------------------------------------
# Scalars: many tiny sequential regions
# ----------------------------------------------------------------------------
def scalars(n_regions: int = 1000, teams: int = 1, threads: int = 128,
            seed: int = DEFAULT_SEED) -> Workload:
    """R sequential regions (param = R); region r's frame is 4 int32 drawn
    U[0, 2^20)."""
    w = max(threads - 32, 1)
    img = uniform_u32(derive(seed, 1), 4 * n_regions, bits=20)
    r = Region(PROG_SCALARS, teams, threads, 1, [16], param=n_regions)
    return Workload("scalars", [r], _as_bytes(img), 4 * n_regions * teams * w, teams)


# ----------------------------------------------------------------------------
# Nested: wide regions with nested levels
# ----------------------------------------------------------------------------
def nested(teams: int = 1024, threads: int = 256, depth: int = 3,
           elems_per_team: int = 4096, seed: int = DEFAULT_SEED) -> Workload:
    """Per (team, level) an init image of 16 + 256 uniform int32 words."""
    img = uniform_u32(derive(seed, 2), teams * depth * NESTED_FRAME_WORDS)
    r = Region(PROG_NESTED, teams, threads, depth, [NESTED_FRAME_BYTES] * depth,
               param=elems_per_team)
    return Workload("nested", [r], _as_bytes(img), 4 * teams * elems_per_team, teams)


# ----------------------------------------------------------------------------
# Sweep: one fp32 frame per team, in the slab or spilled
# ----------------------------------------------------------------------------
SWEEP_SIZES = (64, 1024, 8192, 32768, 98304, 196608)


def sweep(frame_bytes: int, teams: int = 512, threads: int = 128,
          seed: int = DEFAULT_SEED) -> Workload:
    """One FP32 frame of `frame_bytes` per team, N(0,1) per-team images."""
    assert frame_bytes % 4 == 0 and frame_bytes > 0
    w = max(threads - 32, 1)
    img = normal_f32(derive(seed, 3, frame_bytes), teams * (frame_bytes // 4))
    r = Region(PROG_SWEEP, teams, threads, 1, [frame_bytes])
    return Workload("sweep", [r], _as_bytes(img), 4 * teams * w, teams, out_dtype="float32")


# ----------------------------------------------------------------------------
# Hetero: heterogeneous instances (batched / served)
# ----------------------------------------------------------------------------
def hetero_shapes(n_instances: int, seed: int = DEFAULT_SEED,
                  max_teams: int = 512, max_frame: int = 32768):
    """Draw (teams, threads, depth, frame_bytes[3], salt) per instance.

    teams: log-uniform in [1, max_teams]; threads: uniform over the multiples
    of 32 in [32, 1024]; depth: uniform in {1, 2, 3}; frame bytes per level:
    log-uniform in [16, max_frame], rounded down to a multiple of 4.
    """
    s = derive(seed, 4)
    teams = log_uniform_int(derive(s, 1), n_instances, 1, max_teams)
    threads = 32 * (1 + (uniform_u32(derive(s, 2), n_instances).astype(np.uint64) * 32
                         >> np.uint64(32)).astype(np.int64))
    depth = 1 + (uniform_u32(derive(s, 3), n_instances).astype(np.uint64) * 3
                 >> np.uint64(32)).astype(np.int64)
    fb = log_uniform_int(derive(s, 4), 3 * n_instances, 16, max_frame).reshape(n_instances, 3)
    fb = (fb // 4) * 4
    salt = uniform_u32(derive(s, 5), n_instances)
    return teams, threads, depth, fb, salt


def hetero(n_instances: int = 10000, seed: int = DEFAULT_SEED,
           max_teams: int = 512, max_frame: int = 32768,
           instances: Optional[np.ndarray] = None) -> Workload:
    """Heterogeneous region instances with packed images and outputs.

    Instance i's images sit at image_offset (16-byte aligned), level k after
    levels < k (each level padded to 16 bytes); its output int32[T][W'] sits
    at out_offset (16-byte aligned); its team-status entries start at
    status_index. `instances` optionally selects a subset (by index) of the
    same draw, keeping each instance's random content.
    """
    teams, threads, depth, fb, salt = hetero_shapes(n_instances, seed, max_teams, max_frame)
    sel = np.arange(n_instances) if instances is None else np.asarray(instances)
    regions = []
    img_off = out_off = st_idx = 0
    chunks = []
    for i in sel.tolist():
        d = int(depth[i])
        fbs = [int(x) for x in fb[i, :d]]
        w = max(int(threads[i]) - 32, 1)
        r = Region(PROG_HETERO, int(teams[i]), int(threads[i]), d, fbs,
                   salt=int(salt[i]), status_index=st_idx,
                   image_offset=img_off, out_offset=out_off)
        regions.append(r)
        for k, b in enumerate(fbs):
            words = uniform_u32(derive(seed, 5, i, k), b // 4)
            pad = _pad16(b) - b
            chunks.append(_as_bytes(words))
            if pad:
                chunks.append(np.zeros(pad, np.uint8))
            img_off += _pad16(b)
        out_off += _pad16(4 * int(teams[i]) * w)
        st_idx += int(teams[i])
    images = np.concatenate(chunks) if chunks else np.zeros(16, np.uint8)
    return Workload("hetero", regions, images, max(out_off, 16), st_idx,
                    meta=dict(n_instances=len(regions)))


# ----------------------------------------------------------------------------
# Worker-level sharing (the paper's future work, Sec. 7)
# ----------------------------------------------------------------------------
def workers(teams: int = 1024, threads: int = 256, frame_bytes: int = 256, width: int = 0,
            seed: int = DEFAULT_SEED, share: int = 0) -> Workload:
    """Per team an image of int32 s[4] then int32 base[S/4], the pair padded
    to 16 bytes; uniform int32 words. `share` is the descriptor's param: how
    the nested teams get their workers' keys and frame offsets on the GPU
    (0: warp shuffles, 1: a shared-memory table); results do not depend on
    it."""
    assert frame_bytes % 4 == 0 and frame_bytes > 0 and threads >= 64
    stride = 16 + _pad16(frame_bytes)
    img = uniform_u32(derive(seed, 7, frame_bytes), teams * stride // 4)
    r = Region(PROG_WORKERS, teams, threads, 2, [16, frame_bytes], width=width, param=share)
    return Workload("workers", [r], _as_bytes(img), 4 * teams * r.team_width, teams)


def poisson_arrivals(n: int, rate_per_s: float, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Open-loop arrival times (ns from start) of a Poisson process."""
    u = uniform_f64(derive(seed, 6, int(rate_per_s)), n)
    gaps = -np.log1p(-u) / rate_per_s
    return np.round(np.cumsum(gaps) * 1e9).astype(np.int64)
