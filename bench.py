"""Benchmark of the generic-mode data-sharing runtime on one GB300 (or N,
one process per GPU, each running its own independent regions).

Default workload: the wide plain-launch configuration -- 1024 teams x 256
threads, 3 nested levels each pushing a 1088-byte frame (16 int32 scalars
+ int32[256]), 4M int32 output -- one region instance per step, launched
through the C ABI. Metric: regions/s, with push+pop/s beside it. The steps
run back to back between one pair of CUDA events, each on the next of a
rotating set of copies of the region's buffers that together exceed twice
the L2; one launch timed alone after an L2 flush is reported beside it. The
end-to-end figure runs the same steps from pinned host buffers, alternating
over two streams (upload, kernel and download of every step inside the
timed region).

The same JSON line also carries the other configurations and launch forms
(`--forms none` skips them):
  sweep    - 512 teams x 128 threads, one fp32 frame of 64 B .. 192 KiB per
             team, in the shared-memory slab and in the overflow slab: time,
             HBM GB/s, occupancy and shared memory per team for each (frames
             of 8 KiB and up over rotating copies, back to back);
  scalars  - 1 team x 128 threads, 1000 sequential regions: one launch that
             runs them all against 1000 launches of one region each;
  batched  - 10,000 heterogeneous instances (log-uniform teams and frame
             sizes) in one persistent launch replayed from a CUDA graph,
             against one plain launch per instance;
  served   - the same instance distribution submitted open-loop (Poisson)
             to the device-resident server at several rates: p50/p99
             latency and sustained requests/s, against one plain launch per
             request under the same arrivals;
  workers  - worker-level sharing, 1024 teams x 256 threads: every worker
             pushes a 256-byte frame on its warp's stack for a nested region
             on its warp, with the warp stacks in the slab and on the global
             stack.

Prints ONE JSON line (rank 0), with the CPU oracle timed beside it on a
bounded sample (every host core, and one thread). `--impl reference` times
the oracle alone on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
ROTATE_BYTES = 264 << 20    # > twice the 129 MB L2: the headline's rotating input sets

# CTA shapes of the device-resident server (threads per CTA, shared slab
# bytes), from sweeps of 64 to 256 threads and 4 to 24 KiB slabs on the
# hetero distribution: 256 threads gives the lowest latency, 128 threads
# with 24 KiB slabs the highest capacity (above a million requests/s) with
# latency close behind.
SERVE_SHAPES = [dict(threads=256, slab_bytes=16384), dict(threads=128, slab_bytes=24576)]

# DRAM traffic per launch of the plain nested kernel in the headline's steady
# state (launches back to back over the rotating input sets, so each launch
# also writes back the output lines an earlier launch left dirty in L2):
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture
# (profiles/nested_1024x256_d3_traffic.md), keyed by a hash of the code of
# the sources that kernel is built from (comments and white space left
# out); any change to that code makes it null.
TRAFFIC_BY_SOURCE = {"7fee0faf7817506d": 18553318}
KERNEL_SOURCES = ["include/dsr_runtime.cuh", "include/dsr_check.cuh", "include/dsr_kernels.cuh",
                  "include/dsr.h", "paper_1711_10413_gb300/csrc/dsr_programs.cuh",
                  "paper_1711_10413_gb300/csrc/dsr_capi.cu"]


def _code_only(text: str) -> str:
    """C/C++/CUDA source without comments and white space."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return "".join(text.split())


def source_key() -> str:
    """Hash of the code of the headline kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic():
    return TRAFFIC_BY_SOURCE.get(source_key())


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6800.0, source="fallback")


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def rotating_sets(work):
    """(bytes of one copy of a region's buffers, copies whose total exceeds
    twice the L2): the headline's inputs larger than L2."""
    set_bytes = (work.images.nbytes + 4 * (max(work.out_bytes, 16) // 4) + 32 * work.n_status)
    return set_bytes, 1 + -(-ROTATE_BYTES // set_bytes)


def bench_config(cfg, work, world: int) -> dict:
    """The `config` both arms print (the same dict for the same workload)."""
    set_bytes, n_sets = rotating_sets(work)
    return dict(cfg, parallelism="independent regions per GPU" if world > 1 else "1 GPU",
                l2="inputs larger than L2: %d rotating sets of the region's buffers "
                   "(%.1f MB each, %.0f MB in all), launched back to back"
                   % (n_sets, set_bytes / 1e6, n_sets * set_bytes / 1e6))


def make_workload(name: str, rank: int = 0):
    seed = wl.DEFAULT_SEED + 7919 * rank
    if name == "nested":
        work = wl.nested(teams=1024, threads=256, depth=3, elems_per_team=4096, seed=seed)
        r = work.regions[0]
        algo_bytes = (r.teams * r.depth * 1088          # images read
                      + 4 * r.teams * r.param           # output written
                      + 32 * r.teams)                   # team statuses written
        cfg = dict(workload="nested_1024x256_d3", teams=1024, threads=256, depth=3,
                   frame_bytes=1088, out_elems=1024 * 4096, slab_bytes=3264)
        return work, 3264, 0, algo_bytes, cfg
    raise SystemExit("unknown workload %r" % name)


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part codes, 0x41/0xd4f being Neoverse V2, Grace's core)."""
    import platform
    name, impl, part = "", "", ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k == "model name" and not name:
                    name = v
                elif k == "CPU implementer" and not impl:
                    impl = v
                elif k == "CPU part" and not part:
                    part = v
    except OSError:
        pass
    if name:
        return name
    if impl or part:
        known = {("0x41", "0xd4f"): "Arm Neoverse V2"}
        return "%s (implementer %s, part %s)" % (known.get((impl, part), platform.machine()),
                                                impl, part)
    return platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(work, slab, ovf, budget_s: float = 10.0, threads: int = 1):
    """Regions/s of the oracle on `threads` host threads, each running its own
    contiguous slice of the teams in chunks until the budget runs out. The
    oracle keeps no global state and its ctypes call releases the GIL, so the
    threads run in parallel; their team slices, output rows and status words
    are disjoint."""
    import threading
    import oracle
    oracle.build()
    r = work.regions[0]
    out = np.zeros(work.out_bytes // 4, dtype=np.int32)
    st = np.zeros(work.n_status, dtype=oracle.STATUS_DTYPE)
    threads = max(1, min(threads, r.teams))
    done = [0] * threads
    chunk = 64 if threads == 1 else 8
    start = threading.Barrier(threads + 1)
    t_end = [0.0]

    def worker(i):
        lo, hi = i * r.teams // threads, (i + 1) * r.teams // threads
        b = lo
        start.wait()
        while time.perf_counter() < t_end[0]:
            e = min(b + chunk, hi)
            oracle.run_region(r, work.images, out, st, slab, ovf, b, e)
            done[i] += e - b
            b = lo if e == hi else e

    pool = [threading.Thread(target=worker, args=(i,)) for i in range(threads)]
    for t in pool:
        t.start()
    t0 = time.perf_counter()
    t_end[0] = t0 + budget_s
    start.wait()
    for t in pool:
        t.join()
    dt = time.perf_counter() - t0
    teams_done = sum(done)
    regions = teams_done / r.teams
    return dict(value=regions / dt, unit="regions/s", cores=threads, kind="oracle",
                cpu=cpu_model(),
                sample="%d teams of the workload (%.2f regions) in %.1f s, %d thread%s"
                       % (teams_done, regions, dt, threads, "" if threads == 1 else "s"))


def cpu_baseline(work, slab, ovf, budget_s: float):
    """The oracle on every host core, with the one-thread figure beside it."""
    one = time_oracle(work, slab, ovf, budget_s / 2, threads=1)
    n = host_cores()
    if n <= 1:
        return one
    line = time_oracle(work, slab, ovf, budget_s / 2, threads=n)
    line["single_thread"] = dict(value=one["value"], sample=one["sample"])
    return line


# ---------------------------------------------------------------------------
# The other launch forms
# ---------------------------------------------------------------------------
def _event_ms(torch, fn, reps, flush=None):
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    out = []
    for i in range(reps):
        if flush is not None:
            flush.fill_(i)
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        z.record(s)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(z))
    return float(np.median(out))


def _rotating_ms(torch, launch, n_sets, reps):
    """Per-launch time of `reps` launches back to back between one pair of
    events, launch i on input set i % n_sets (sets larger than L2 together,
    so no launch finds its inputs in L2 from the set's last use)."""
    s = torch.cuda.current_stream()
    for i in range(n_sets):
        launch(i)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    torch.cuda._sleep(int(2.1e9 * (1e-3 + 50e-6 * reps)))  # the host queues ahead
    a.record(s)
    for i in range(reps):
        launch(i)
    z.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(z) / reps


def smem_footprint(torch, rt, region, device):
    """Shared memory the headline's resident teams hold on one SM, as a
    share of the SM's shared memory, beside the paper's K40 figure for its
    scalars program (context only: other hardware, another program)."""
    occ = rt.occupancy(region)
    props = torch.cuda.get_device_properties(device)
    sm_bytes = getattr(props, "shared_memory_per_multiprocessor", 0) or 233472
    held = occ["ctas_per_sm"] * occ["smem_per_team"]
    return dict(per_team=occ["smem_per_team"], ctas_per_sm=occ["ctas_per_sm"],
                bytes_per_sm=held, sm_bytes=sm_bytes, frac_of_sm=held / sm_bytes,
                paper_context="K40, scalars program: at most 4332 bytes per SM, about 26 % "
                              "of the 16 KB default shared memory (Sec. 6.3)")


def smem_derived_gbs(sm_count: int, sm_mhz: float = 2070.0) -> float:
    """Shared-memory bandwidth from the unit counts: 128 bytes per clock per
    SM (32 banks of 4 bytes) at the maximum SM clock."""
    return sm_count * 128.0 * sm_mhz * 1e6 / 1e9


_SMEM_PEAK = {}


def smem_peak(dsr=None, torch=None, device: int = 0, sm_count: int = 152) -> dict:
    """The shared-memory roofline: measured once per run by the library's
    probe (conflict-free 16-byte loads streaming on every SM, CUDA-event
    timed), with the figure derived from the unit counts beside it."""
    if "gbs" not in _SMEM_PEAK:
        derived = smem_derived_gbs(sm_count)
        try:
            rt = dsr.Runtime(device, slab_bytes=0)
            scratch = torch.zeros(4, dtype=torch.int64, device="cuda:%d" % device)
            p = dsr.dsr_probe_smem_bandwidth(rt.ctx, 4096, scratch)
            rt.close()
            _SMEM_PEAK.update(gbs=p["gbs"], source="measured", probe=p, derived_gbs=derived)
        except Exception as e:   # noqa: BLE001 - a probe failure must not hide the bench
            _SMEM_PEAK.update(gbs=derived, source="derived (probe failed: %s)" % e,
                              derived_gbs=derived)
    return _SMEM_PEAK


def smem_peak_gbs(sm_count: int) -> float:
    return smem_peak(sm_count=sm_count)["gbs"] if _SMEM_PEAK else smem_derived_gbs(sm_count)


def hetero_stack_bytes(regions) -> int:
    """Stack bytes the hetero program moves by its definition, summed over
    teams: each level's frame is written once by its push, read and written
    once by a non-innermost region, read once by the master's sum after
    that region, and read once by the innermost region."""
    total = 0
    for r in regions:
        fb = list(r.frame_bytes)[: r.depth]
        total += r.teams * (2 * sum(fb) + 3 * sum(fb[:-1]))
    return total


SWEEP_MAX_SETS = 80


def measure_sweep(dsr, torch, device, flush, hbm_gbs, sizes=None):
    """The sweep: one fp32 frame per team, 512 teams x 128 threads, for each
    frame size placed in the shared-memory slab (when one CTA can hold it)
    and in the global overflow slab; HBM bytes per launch = images read +
    outputs + statuses. Like the headline, a frame size whose buffers fit
    SWEEP_MAX_SETS copies into more than twice the L2 is timed over rotating
    copies launched back to back; smaller ones one launch at a time after
    an L2 flush."""
    teams, threads = 512, 128
    smem_bound = smem_peak_gbs(torch.cuda.get_device_properties(device).multi_processor_count)
    rt = dsr.Runtime(device, slab_bytes=0, overflow_bytes_per_team=max(wl.SWEEP_SIZES),
                     max_teams=teams)
    res = []
    for S in sizes or wl.SWEEP_SIZES:
        work = wl.sweep(S, teams=teams, threads=threads)
        region = work.regions[0]
        images, out, status = rt.device_buffers(work)
        set_bytes = images.numel() + 4 * (out.numel() + status.numel())
        n_sets = 1 + -(-ROTATE_BYTES // set_bytes)
        sets = [(images, out, status)]
        if n_sets <= SWEEP_MAX_SETS:
            sets += [(images.clone(), torch.empty_like(out), torch.zeros_like(status))
                     for _ in range(n_sets - 1)]
        for where in ("smem", "overflow"):
            if where == "smem":
                if S + 384 > 232448:
                    continue
                rt.configure(S, 0, 0)
            else:
                rt.configure(0, S, teams)
            occ = rt.occupancy(region)

            def launch(i=0):
                im, o, st_d = sets[i % len(sets)]
                dsr.dsr_launch_region(rt.ctx, region, im, o, st_d)

            if len(sets) > 1:
                ms = _rotating_ms(torch, launch, len(sets), max(20, 2 * len(sets)))
                timing = "%d rotating sets (%.0f MB), back to back" % (
                    len(sets), len(sets) * set_bytes / 1e6)
            else:
                ms = _event_ms(torch, launch, 10, flush)
                timing = "one launch per event pair after an L2 flush"
            st = np.concatenate([x[2].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
                                 for x in sets])
            hbm = teams * S + teams * (threads - 32) * 4 + teams * 32
            gbs = hbm / (ms * 1e-3) / 1e9
            # a frame in the slab: the fill writes S bytes of shared memory per
            # team and the workers read them back
            smem = 2 * teams * S if where == "smem" else 0
            smem_gbs = smem / (ms * 1e-3) / 1e9
            res.append(dict(frame_bytes=S, placement=where, us=ms * 1e3,
                            regions_per_s=1.0 / (ms * 1e-3), hbm_bytes=hbm, hbm_gbs=gbs,
                            hbm_frac=gbs / hbm_gbs, smem_bytes=smem, smem_gbs=smem_gbs,
                            smem_frac=smem_gbs / smem_bound,
                            overflow_bytes=2 * teams * S if where == "overflow" else 0,
                            smem_per_team=occ["smem_per_team"], ctas_per_sm=occ["ctas_per_sm"],
                            regs_per_thread=occ["regs_per_thread"],
                            spill_bytes_per_team=int(st["spill_bytes"].max()),
                            bad_team_status=int((st["status"] != 0).sum()), timing=timing))
        del images, out, status, sets
    rt.close()
    return dict(workload="sweep_512x128", teams=teams, threads=threads, runs=res)


FORMS = ("sweep", "scalars", "batched", "served", "workers")


def measure_host_link(torch, nbytes=16 << 20, reps=10):
    """Copy bandwidth of the host link, each direction alone: 16 MiB between
    pinned host memory and the device by cudaMemcpyAsync (torch's
    non-blocking copy), CUDA events on the copying stream, best of three
    rounds after a warm-up. The host-buffer path can move its bytes no
    faster, so it bounds the e2e figure."""
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream()
    res = {}
    for name, dst, src in (("d2h_gbs", h, d), ("h2d_gbs", d, h)):
        best = None
        with torch.cuda.stream(s):
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            for _ in range(3):
                a = torch.cuda.Event(enable_timing=True)
                z = torch.cuda.Event(enable_timing=True)
                a.record(s)
                for _ in range(reps):
                    dst.copy_(src, non_blocking=True)
                z.record(s)
                z.synchronize()
                ms = a.elapsed_time(z)
                best = ms if best is None else min(best, ms)
        res[name] = nbytes * reps / (best * 1e-3) / 1e9
    return res


def measure_workers(dsr, torch, device, flush, sm_count):
    """Worker-level sharing: 1024 teams x 256 threads, each of the 224
    workers pushes a 256-byte frame on its warp's stack and runs a nested
    region on its warp. Warp stacks in the slab, then all on the global
    (overflow) stack. Stack bytes per worker frame: written by the fill,
    read and written by the nested region, read by the worker's sum.

    Beside it, the two ways a worker's nested team (its warp's lanes) gets
    the worker's key and frame offset, in the slab: warp shuffles (param 0)
    against a per-warp table in shared memory (param 1), for 256-byte frames
    (whole rows of 32 words: keys only) and 100-byte frames (the general
    walk: keys and slot offsets at every step)."""
    teams, threads, S = 1024, 256, 256
    W = threads - 32
    rt = dsr.Runtime(device, slab_bytes=0, overflow_bytes_per_team=16 + W * S, max_teams=teams)
    runs = []

    def one(work, where, slab, ovf):
        region = work.regions[0]
        images, out, status = rt.device_buffers(work)
        rt.configure(slab, ovf, teams if ovf else 0)
        occ = rt.occupancy(region)
        ms = _event_ms(torch, lambda: dsr.dsr_launch_region(rt.ctx, region, images, out, status),
                       10, flush)
        st = status.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
        fb = region.frame_bytes[1]
        stack = teams * W * 4 * ((fb + 15) // 16 * 16)
        gbs = stack / (ms * 1e-3) / 1e9
        return dict(placement=where, frame_bytes=fb, share="smem" if region.param else "shuffle",
                    us=ms * 1e3, regions_per_s=1.0 / (ms * 1e-3),
                    worker_frames_per_s=teams * W / (ms * 1e-3), stack_bytes=stack,
                    stack_gbs=gbs, smem_frac=gbs / smem_peak_gbs(sm_count),
                    smem_per_team=occ["smem_per_team"], ctas_per_sm=occ["ctas_per_sm"],
                    regs_per_thread=occ["regs_per_thread"],
                    spill_bytes_per_team=int(st["spill_bytes"].max()),
                    bad_team_status=int((st["status"] != 0).sum()))

    work = wl.workers(teams=teams, threads=threads, frame_bytes=S)
    runs.append(one(work, "slab", 16 + W * S, 0))
    runs.append(one(work, "overflow", 16, W * S))
    sharing = []
    for fb in (256, 100):
        slab = 16 + W * ((fb + 15) // 16 * 16)
        for share in (0, 1):
            sharing.append(one(wl.workers(teams=teams, threads=threads, frame_bytes=fb,
                                          share=share), "slab", slab, 0))
    rt.close()
    return dict(workload="workers_1024x256_256B", teams=teams, threads=threads,
                worker_frame_bytes=S, runs=runs, sharing_within_a_warp=sharing)


def measure_forms(dsr, torch, device, flush, hbm_gbs, which=FORMS, instances=10000,
                  sweep_sizes=None, tuning=None, dist=None):
    """The other launch forms. With several ranks (torchrun) only the batched
    and served forms run, each rank on its share of the instances or
    requests with no data-path collective; the single-instance workloads
    (sweep, scalars, workers) are measured on one GPU."""
    forms = {}
    if dist is not None:
        which = [f for f in which if f in ("batched", "served")]
    sm_count = torch.cuda.get_device_properties(device).multi_processor_count
    peak = smem_peak(dsr, torch, device, sm_count)
    forms["smem_peak"] = dict(gbs=peak["gbs"], source=peak["source"],
                              derived_gbs=peak["derived_gbs"], probe=peak.get("probe"))
    if "sweep" in which:
        forms["sweep"] = measure_sweep(dsr, torch, device, flush, hbm_gbs, sweep_sizes)
    rt = dsr.Runtime(device, slab_bytes=16384, overflow_bytes_per_team=3 * 32768, max_teams=4096)
    if "scalars" in which:
        forms.update(measure_scalars(dsr, torch, rt, flush))
    if "batched" in which:
        forms.update(measure_batched(dsr, torch, rt, flush, sm_count, instances, tuning, dist))
    if "served" in which:
        forms.update(measure_served(dsr, rt, dist))
    rt.close()
    if "workers" in which:
        forms["workers"] = measure_workers(dsr, torch, device, flush, sm_count)
    return forms


def measure_scalars(dsr, torch, rt, flush):
    forms = {}
    # scalars: 1000 sequential regions of one team
    sc = wl.scalars(n_regions=1000, teams=1, threads=128)
    one = wl.scalars(n_regions=1, teams=1, threads=128)
    rt.configure(1024, 3 * 32768, 4096)
    images, out, status = rt.device_buffers(sc)
    r_all = sc.regions[0]
    ms_all = _event_ms(torch, lambda: dsr.dsr_launch_region(rt.ctx, r_all, images, out, status),
                       10, flush)
    descs = dsr.pack_descs([dict(one.regions[0].as_dict(), image_offset=16 * i,
                                 out_offset=4 * 96 * i) for i in range(1000)])
    ms_each = _event_ms(torch, lambda: dsr.dsr_launch_regions(rt.ctx, descs, images, out, status),
                        3, flush)
    forms["scalars"] = dict(workload="scalars_1x128_r1000", regions=1000,
                            one_launch_regions_per_s=1000 / (ms_all * 1e-3),
                            per_launch_regions_per_s=1000 / (ms_each * 1e-3),
                            handoff_ns_per_region=ms_all * 1e6 / 1000)
    return forms


def batch_share(instances: int, rank: int, world: int):
    """This rank's instances of the batched form: the contiguous range of the
    `instances`-instance hetero draw that balanced_ranges gives it by team
    count (all of them on one GPU)."""
    from paper_1711_10413_gb300 import shard
    teams = wl.hetero_shapes(instances)[0]
    a, b = shard.balanced_ranges(teams, world)[rank]
    return np.arange(a, b)


def served_share(descs_teams, rank: int, world: int):
    """The requests this rank serves, by least outstanding teams
    (route_requests), in arrival order."""
    from paper_1711_10413_gb300 import shard
    return np.nonzero(shard.route_requests(descs_teams, world) == rank)[0]


def _pool_latencies(lat, dist):
    """Every rank's latencies, on rank 0 (None elsewhere)."""
    if dist is None:
        return lat
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(lat, parts, dst=0)
    return np.concatenate(parts) if parts is not None else None


def measure_batched(dsr, torch, rt, flush, sm_count, instances=10000, tuning=None, dist=None):
    """The batched form on this rank's share of the instances (all of them on
    one GPU); with several ranks every figure is the job's: instances of all
    ranks over the slowest rank's time."""
    from paper_1711_10413_gb300 import shard
    forms = {}
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    mine = batch_share(instances, rank, world)
    rt.configure(16384, 3 * 32768, 4096)
    work = wl.hetero(n_instances=instances, instances=mine)
    b = rt.batch_buffers(work)
    if tuning is None:
        tuning, _ = rt.autotune(b)
    if dist:
        dist.barrier()
    ms_batch = shard.max_over_ranks(
        _event_ms(torch, lambda: rt.launch_batch(b, tuning, use_graph=True), 5, flush), dist)
    err, counted = rt.batch_errors(b)
    ms_plain = shard.max_over_ranks(_event_ms(torch, lambda: rt.launch_regions(b), 2, flush), dist)
    st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    # the same per-instance launches with each launch's slab sized from its
    # region's footprint instead of one 16 KiB slab for all
    rt.configure(dsr.DSR_SLAB_AUTO, 3 * 32768, 4096)
    ms_auto = shard.max_over_ranks(_event_ms(torch, lambda: rt.launch_regions(b), 2, flush), dist)
    # ... and those launches replayed from one launch graph (no host call per
    # instance): the strongest one-launch-per-region baseline
    graph = dsr.dsr_graph_capture_regions(rt.ctx, work.regions,
                                          [(b["images"], b["out"], b["status"])] * len(work.regions))
    ms_graph = shard.max_over_ranks(
        _event_ms(torch, lambda: dsr.dsr_graph_launch(rt.ctx, graph), 2, flush), dist)
    dsr.dsr_graph_destroy(graph)
    rt.configure(16384, 3 * 32768, 4096)
    stack = shard.sum_over_ranks(hetero_stack_bytes(work.regions), dist)
    push_pop = shard.sum_over_ranks(sum(r.teams * r.depth for r in work.regions), dist)
    counted = int(shard.sum_over_ranks(counted, dist))
    err = int(shard.sum_over_ranks(err, dist))
    bad = int(shard.sum_over_ranks(int((st["status"] != 0).sum()), dist))
    smem_gbs = stack / (ms_batch * 1e-3) / 1e9
    forms["batched"] = dict(workload="hetero_%d_instances" % instances, instances=instances,
                            teams=counted, tuning=tuning,
                            ranks=world, scaling="strong" if world > 1 else None,
                            batched_regions_per_s=instances / (ms_batch * 1e-3),
                            per_launch_regions_per_s=instances / (ms_plain * 1e-3),
                            per_launch_auto_slab_regions_per_s=instances / (ms_auto * 1e-3),
                            per_launch_graph_regions_per_s=instances / (ms_graph * 1e-3),
                            batched_push_pop_per_s=push_pop / (ms_batch * 1e-3),
                            speedup=ms_plain / ms_batch,
                            speedup_vs_graph=ms_graph / ms_batch,
                            stack_roofline=dict(bound="smem", stack_bytes=stack,
                                                achieved=smem_gbs,
                                                peak=world * smem_peak_gbs(sm_count),
                                                unit="GB/s",
                                                frac=smem_gbs / (world * smem_peak_gbs(sm_count)),
                                                peak_source=_SMEM_PEAK.get("source", "derived"),
                                                derived_peak=world * smem_derived_gbs(sm_count)),
                            device_rejects=err, bad_team_status=bad)
    del b
    return forms


def measure_served(dsr, rt, dist=None):
    """The served form: each rank serves the requests routed to it (all of
    them on one GPU) with its own server, at the requests' arrival times;
    the job's latency percentiles pool every rank's requests and its
    sustained rate is all requests over the slowest rank's span."""
    from paper_1711_10413_gb300 import shard
    forms = {}
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    # hetero requests: served at several rates vs per-request launches. 100,000
    # requests per rate cycle over 20,000 distinct instances (a request's
    # twins rewrite the same output rows with the same values); the first
    # 10 % of each run are warm-up and not counted in the percentiles.
    distinct, n = 20000, 100000
    warm = n // 10
    sw = wl.hetero(n_instances=distinct)
    # the served form's overflow pool: 4 GiB, 1 MiB for each of 4096 CTAs
    pool_per_cta, pool_ctas = 1 << 20, 4096
    rt.configure(16384, pool_per_cta, pool_ctas)
    served = {}
    for shape in SERVE_SHAPES:
        # The server runs its own CTA shape: with requests arriving one at a
        # time, fewer and wider CTAs contend less on the claim words than the
        # many narrow CTAs that suit a whole batch known up front.
        bs = rt.serve_start(sw, threads=shape["threads"], slab_bytes=shape["slab_bytes"],
                            capacity=8192)
        descs = np.tile(bs["descs"], n // distinct)
        mine = served_share(descs["teams"], rank, world)
        is_warm = mine >= warm  # requests after the first 10 % of the stream
        res = {}
        try:
            for rate in (50000, 100000, 200000, 500000):
                arrivals = wl.poisson_arrivals(n, float(rate))[mine]
                if dist:
                    dist.barrier()
                lat, el = dsr.dsr_serve_bench(rt.ctx, descs[mine], arrivals)
                el = shard.max_over_ranks(el, dist)
                failed = int(shard.sum_over_ranks(int((lat < 0).sum()), dist))
                pooled = _pool_latencies(lat[is_warm], dist)
                if rank == 0:
                    ok = pooled[pooled >= 0]
                    res[str(rate)] = dict(p50_us=float(np.percentile(ok, 50)) / 1e3,
                                          p99_us=float(np.percentile(ok, 99)) / 1e3,
                                          sustained_regions_per_s=n / (el * 1e-9),
                                          failed=failed)
            # closed loop: every request due at once, so the ring stays full
            # and the server runs at its own capacity
            if dist:
                dist.barrier()
            lat, el = dsr.dsr_serve_bench(rt.ctx, descs[mine], np.zeros(len(mine), dtype=np.int64))
            el = shard.max_over_ranks(el, dist)
            failed = int(shard.sum_over_ranks(int((lat < 0).sum()), dist))
            res["capacity"] = dict(regions_per_s=n / (el * 1e-9), failed=failed)
        finally:
            rt.serve_stop()
        served["%d_threads_%d_slab" % (shape["threads"], shape["slab_bytes"])] = res
    launched = {}
    for rate in (50000, 100000):
        m = 5000
        sel = served_share(bs["descs"]["teams"][:m], rank, world)
        if dist:
            dist.barrier()
        lat, el = dsr.dsr_launch_bench(rt.ctx, bs["descs"][:m][sel],
                                       wl.poisson_arrivals(m, float(rate))[sel],
                                       bs["images"], bs["out"], bs["status"])
        el = shard.max_over_ranks(el, dist)
        pooled = _pool_latencies(lat, dist)
        if rank == 0:
            launched[str(rate)] = dict(p50_us=float(np.percentile(pooled, 50)) / 1e3,
                                       p99_us=float(np.percentile(pooled, 99)) / 1e3,
                                       sustained_regions_per_s=m / (el * 1e-9))
    forms["served"] = dict(workload="hetero_poisson_%d_requests_%d_distinct" % (n, distinct),
                           ranks=world, warmup_dropped=warm,
                           overflow_pool_bytes=pool_per_cta * pool_ctas,
                           server=served, per_request_launch=launched)
    return forms


# ---------------------------------------------------------------------------
# Main
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="dsr", choices=["dsr", "reference"])
    ap.add_argument("--workload", default="nested")
    ap.add_argument("--cpu-budget", type=float, default=16.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="all",
                    help="all, none, or a comma-separated list of " + ", ".join(FORMS))
    ap.add_argument("--instances", type=int, default=10000,
                    help="instances of the batched form")
    ap.add_argument("--tuning", default="",
                    help="threads,slab_bytes of the batched form (default: autotuned)")
    ap.add_argument("--sweep-sizes", default="",
                    help="comma-separated frame sizes of the sweep form (default: all six)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        work, slab, ovf, algo_bytes, cfg = make_workload(args.workload, 0)
        for _ in range(args.warmup):
            pass
        per_step = []
        budget = max(0.25, 60.0 / max(args.steps, 1))  # about a minute in all
        samples = []
        cores = host_cores()
        for _ in range(args.steps):
            s = time_oracle(work, slab, ovf, budget_s=budget, threads=cores)
            samples.append(s)
            per_step.append(s["value"])
        v = float(statistics.median(per_step))
        line = dict(impl="reference", metric="regions/s", value=v, unit="regions/s",
                    n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                    ms_per_step=1000.0 / v, higher_is_better=True, scaling="weak",
                    vs_baseline=None, dtype="int32", data="synthetic",
                    config=bench_config(cfg, work, args.gpus),
                    e2e=dict(value=v, unit="regions/s", h2d_bytes_per_step=0,
                             d2h_bytes_per_step=0),
                    cpu_baseline=dict(value=v, unit="regions/s", cores=samples[-1]["cores"],
                                      kind="oracle", cpu=samples[-1]["cpu"],
                                      sample=samples[-1]["sample"]))
        print(json.dumps(line))
        return

    import torch
    import paper_1711_10413_gb300 as dsr
    from paper_1711_10413_gb300 import shard

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dsr.build()

    work, slab, ovf, algo_bytes, cfg = make_workload(args.workload, rank)
    region = work.regions[0]
    rt = dsr.Runtime(local, slab_bytes=slab, overflow_bytes_per_team=ovf,
                     max_teams=region.teams if ovf else 0)
    images, out, status = rt.device_buffers(work)
    stream = torch.cuda.current_stream()

    # Inputs larger than L2: the region's buffers (images, output, statuses)
    # in n_sets copies, launched in turn. Between two uses of a set the other
    # sets, more than twice the L2, pass through it, so no launch finds its
    # images or output lines in L2 from the last time, and the timed launches
    # run back to back with no flush between them.
    set_bytes, n_sets = rotating_sets(work)
    assert set_bytes == images.numel() * images.element_size() + 4 * (out.numel() + status.numel())
    sets = [(images, out, status)] + [
        (images.clone(), torch.empty_like(out), torch.zeros_like(status))
        for _ in range(n_sets - 1)]

    def step(i=0, s=None):
        im, o, st = sets[i % n_sets]
        dsr.dsr_launch_region(rt.ctx, region, im, o, st, stream if s is None else s)

    warmup_launches = max(args.warmup, n_sets)  # every set used once before timing
    for i in range(warmup_launches):
        step(i)
    torch.cuda.synchronize()

    # The timed steps are the same K launches (set i mod n_sets for step i),
    # issued by replaying the library's launch graph of them
    # (dsr_graph_capture_regions): consecutive launches keep their
    # programmatic dependence as graph edges, and the GPU takes the K kernel
    # nodes without a host call each. Issued one call at a time they are timed
    # as well (direct_launches).
    graph = dsr.dsr_graph_capture_regions(rt.ctx, [region] * args.steps,
                                          [sets[i % n_sets] for i in range(args.steps)])
    dsr.dsr_graph_launch(rt.ctx, graph, stream)  # untimed: one more pass over every set
    torch.cuda.synchronize()

    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # hold the stream for a moment so the host queues every step before the
    # GPU reaches it: the events then time the GPU alone, never a GPU that
    # waits for the host to launch the next kernel
    torch.cuda._sleep(int(2.1e9 * 2e-3))
    t_start.record(stream)
    dsr.dsr_graph_launch(rt.ctx, graph, stream)
    t_stop.record(stream)
    torch.cuda.synchronize()
    bracket_s = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2.1e9 * (2e-3 + 30e-6 * args.steps)))
    d_start = torch.cuda.Event(enable_timing=True)
    d_stop = torch.cuda.Event(enable_timing=True)
    d_start.record(stream)
    for i in range(args.steps):
        step(i)
    d_stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_step = t_start.elapsed_time(t_stop) / args.steps
    ms_step = shard.max_over_ranks(ms_step, dist)   # the slowest rank's step
    ms_direct = shard.max_over_ranks(d_start.elapsed_time(d_stop) / args.steps, dist)
    dsr.dsr_graph_destroy(graph)
    regions_done = shard.sum_over_ranks(1.0, dist)  # one region per rank per step

    # every team of every set must have ended OK with its stack empty, and
    # every set must hold the same output (the same images, the same region)
    bad_status = 0
    for _, o, st in sets:
        st_np = st.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
        bad_status += int((st_np["status"] != 0).sum() + (st_np["depth_final"] != 0).sum())
    sets_agree = all(torch.equal(o, out) for _, o, _ in sets[1:])

    # For comparison: one launch at a time, timed by its own pair of events,
    # after a 256 MiB write that flushes L2 (outside the events).
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2.1e9 * (2e-3 + 60e-6 * args.steps)))
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        step()
        stops[i].record(stream)
    torch.cuda.synchronize()
    ms_flushed = float(np.mean([a.elapsed_time(b) for a, b in zip(starts, stops)]))
    ms_flushed = shard.max_over_ranks(ms_flushed, dist)
    del sets

    # e2e through the C ABI from pinned host memory: every step uploads its
    # images, runs the region, downloads its output and statuses, and the
    # host checks that step's statuses before the slot is used again. Steps
    # alternate between two streams, each with its own device and host
    # buffers, so one step's download overlaps the next step's upload and
    # kernel (dsr_enqueue_region_host). The one-step-at-a-time call
    # (dsr_run_region_host, synchronised every step) is timed beside it.
    ib, ob, _ = dsr.dsr_region_extent(region)
    img_h = torch.from_numpy(np.ascontiguousarray(work.images)).pin_memory()
    e2e_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_dev = [(images, out, status), rt.device_buffers(work)]
    e2e_host = [(torch.empty(out.numel(), dtype=torch.int32).pin_memory(),
                 torch.empty(status.numel(), dtype=torch.int32).pin_memory()) for _ in range(2)]
    e2e_done = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_bad = [0]
    torch.cuda.synchronize()

    def e2e_run(n):
        for i in range(n + 2):
            k = i % 2
            if i >= 2:   # step i - 2 used this slot: wait for it and read its statuses
                e2e_done[k].synchronize()
                st = e2e_host[k][1].numpy().view(dsr.TEAM_STATUS_DTYPE)
                e2e_bad[0] += int((st["status"] != 0).sum())
            if i < n:
                im, o, st_d = e2e_dev[k]
                oh, sh = e2e_host[k]
                dsr.dsr_enqueue_region_host(rt.ctx, region, img_h, ib, oh, ob, sh, im, o, st_d,
                                            e2e_streams[k])
                e2e_done[k].record(e2e_streams[k])

    e2e_run(args.warmup)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    e2e_run(args.steps)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t1) / args.steps
    e2e_s = shard.max_over_ranks(e2e_s, dist)
    e2e_agree = bool(np.array_equal(e2e_host[0][0].numpy(), out.cpu().numpy()))

    out_h, st_h = e2e_host[0]

    def e2e_step():
        dsr.dsr_run_region_host(rt.ctx, region, img_h, ib, out_h, ob, st_h, images, out,
                                status, stream)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_serial_s = shard.max_over_ranks((time.perf_counter() - t1) / args.steps, dist)
    link = measure_host_link(torch)
    e2e_bound = regions_done * link["d2h_gbs"] * 1e9 / (ob + 32 * region.teams)

    # the other launch forms (every rank takes part: with several ranks the
    # batched and served forms run on each rank's share)
    peaks = _peaks()
    which = FORMS if args.forms == "all" else [f for f in args.forms.split(",")
                                               if f and f != "none"]
    forms = None
    if which:
        sizes = [int(x) for x in args.sweep_sizes.split(",") if x]
        tuning = None
        if args.tuning:
            th, sl = (int(x) for x in args.tuning.split(","))
            tuning = dict(threads=th, slab_bytes=sl, ctas_per_sm=0)
        forms = measure_forms(dsr, torch, local, flush, peaks["hbm_gbs"], which,
                              args.instances, sizes or None, tuning, dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    regions_per_s = regions_done * 1000.0 / ms_step
    achieved = algo_bytes / (ms_step * 1e-3) / 1e9
    line = dict(
        metric="regions/s", value=regions_per_s, unit="regions/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="int32", data="synthetic",
        config=bench_config(cfg, work, world),
        warmup_launches=warmup_launches,
        push_pop_per_s=regions_per_s * region.teams * region.depth,
        roofline=dict(bound="hbm", achieved=achieved, peak=peaks["hbm_gbs"], unit="GB/s",
                      frac=achieved / peaks["hbm_gbs"], traffic=_traffic(),
                      peak_source=peaks["source"], algorithmic_bytes=algo_bytes),
        e2e=dict(value=regions_done / e2e_s, unit="regions/s", h2d_bytes_per_step=int(ib),
                 d2h_bytes_per_step=int(ob + 32 * region.teams),
                 how="dsr_enqueue_region_host, steps alternating over two streams",
                 bad_team_status=e2e_bad[0], output_agrees=e2e_agree,
                 one_step_at_a_time=regions_done / e2e_serial_s,
                 link=dict(link, bound_regions_per_s=e2e_bound,
                           frac=(regions_done / e2e_s) / e2e_bound,
                           how="each rank's step download at the measured "
                               "device-to-host copy bandwidth (16 MiB, pinned, alone)")),
        gpu_launches=args.steps,
        bracket_ms_per_step=1000.0 * bracket_s / args.steps,
        bad_team_status=bad_status,
        sets_agree=sets_agree,
        direct_launches=dict(
            ms_per_step=ms_direct, regions_per_s=regions_done * 1000.0 / ms_direct,
            frac=algo_bytes / (ms_direct * 1e-3) / 1e9 / peaks["hbm_gbs"],
            how="the same K launches, one dsr_launch_region call each"),
        issue="the K timed launches replayed from one launch graph "
              "(dsr_graph_capture_regions, dsr_graph_launch)",
        per_launch_flushed=dict(
            ms=ms_flushed, regions_per_s=regions_done * 1000.0 / ms_flushed,
            frac=algo_bytes / (ms_flushed * 1e-3) / 1e9 / peaks["hbm_gbs"],
            how="one launch between its own pair of events after a 256 MiB L2 flush"),
        smem_footprint=smem_footprint(torch, rt, region, local),
        clocks=clk,
    )
    if forms is not None:
        line["forms"] = forms
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(work, slab, ovf, args.cpu_budget)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
