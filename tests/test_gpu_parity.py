"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs. Integer programs must match bit for bit. The FP32
sweep must equal the oracle's own fp32 index-order sum bit for bit (both
sides add in the program's order, rounding every step to fp32), and, as a
second check, lie within 1e-6 relative plus the recursive-summation error
bound of the oracle's fp64 sum."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # unit roundoff of fp32


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    dsr.build()
    r = dsr.Runtime(0, slab_bytes=16384)
    yield r
    r.close()


def _configure(rt, slab, ovf=0, teams=0):
    rt.configure(slab, ovf, teams if ovf else 0)


def _run_both(rt, work, slab=1 << 16, ovf=0, max_teams=0):
    _configure(rt, slab, ovf, max_teams or work.n_status)
    gpu_out, gpu_st = rt.run_workload(work)
    ref_out, ref_st = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=ovf)
    return gpu_out, gpu_st, ref_out, ref_st


def _assert_status_equal(gst, rst):
    for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(gst[f], rst[f]), f


# ---------------------------------------------------------------------------
# The paper's programs (Sec. 6.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_vars", [1, 7, 20, 21, 64])
@pytest.mark.parametrize("threads", [32, 128, 1024])
def test_paper_scalars(rt, n_vars, threads):
    work = wl.paper_scalars(n_vars=n_vars, teams=37, threads=threads)
    g, gs, r, rs = _run_both(rt, work, slab=1024)
    assert np.array_equal(g, r)
    expect = (work.out_init.astype(np.int64) + n_vars * (n_vars + 1) // 2) & 0xFFFFFFFF
    assert np.array_equal(g.view(np.uint32).astype(np.int64), expect)
    _assert_status_equal(gs, rs)


@pytest.mark.parametrize("n_arrays", [1, 2, 3, 4])
def test_paper_arrays(rt, n_arrays):
    work = wl.paper_arrays(n_arrays=n_arrays, teams=100, threads=128)
    g, gs, r, rs = _run_both(rt, work, slab=2048)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Scalars: 1 team x 128 threads, 1000 sequential regions
# ---------------------------------------------------------------------------
def test_scalars_1000_regions_full(rt):
    work = wl.scalars(n_regions=1000, teams=1, threads=128)
    g, gs, r, rs = _run_both(rt, work, slab=1024)
    assert np.array_equal(g, r)
    assert gs["depth_final"][0] == 0 and gs["hwm_bytes"][0] == 16 and gs["status"][0] == 0


@pytest.mark.parametrize("teams,threads,width", [(5, 256, 0), (3, 1024, 0), (4, 32, 0),
                                                 (2, 128, 17), (3, 64, 1)])
def test_scalars_shapes(rt, teams, threads, width):
    work = wl.scalars(n_regions=33, teams=teams, threads=threads)
    work.regions[0].width = width
    w = work.regions[0].team_width
    work.out_bytes = 4 * 33 * teams * w
    g, gs, r, rs = _run_both(rt, work, slab=1024)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Nested: 1024 teams x 256 threads, 3 nested levels, 4M int32 output
# ---------------------------------------------------------------------------
def test_nested_1024x256_full(rt):
    work = wl.nested(teams=1024, threads=256, depth=3, elems_per_team=4096)
    g, gs, r, rs = _run_both(rt, work, slab=3264)
    assert g.size == 4 * 1024 * 1024
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)
    assert (gs["depth_final"] == 0).all() and (gs["hwm_bytes"] == 3264).all()


@pytest.mark.parametrize("slab,spill", [(0, 3264), (1088, 2176), (2176, 1088), (3264, 0)])
def test_nested_smem_overflow_equivalence(rt, slab, spill):
    work = wl.nested(teams=61, threads=256, depth=3, elems_per_team=4096)
    g, gs, r, rs = _run_both(rt, work, slab=slab, ovf=4096, max_teams=61)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)
    assert (gs["spill_bytes"] == spill).all()


@pytest.mark.parametrize("teams,threads,depth,E,width", [
    (1, 64, 1, 7, 0), (3, 1024, 4, 5000, 0), (9, 96, 2, 333, 0), (4, 256, 3, 4096, 100),
    (2, 32, 3, 64, 0),
    # the innermost region by classes of j & 255: n = 64 exactly, n not a
    # multiple of 64, more threads than periods (some threads write nothing)
    (2, 96, 1, 256, 64), (5, 128, 2, 1280, 0), (3, 1024, 3, 2048, 0), (2, 1024, 4, 256, 0)])
def test_nested_shapes(rt, teams, threads, depth, E, width):
    work = wl.nested(teams=teams, threads=threads, depth=depth, elems_per_team=E)
    work.regions[0].width = width
    g, gs, r, rs = _run_both(rt, work, slab=4352)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)


def test_nested_overflow_failure_reports(rt):
    work = wl.nested(teams=8, threads=256, depth=3)
    g, gs, r, rs = _run_both(rt, work, slab=1088, ovf=1088, max_teams=8)
    assert (gs["status"] == 2).all() and (gs["depth_final"] == 0).all()
    assert np.array_equal(g, r) and not g.any()
    _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Sweep: FP32, 512 teams x 128 threads, frames 64 B .. 192 KiB
# ---------------------------------------------------------------------------
def _check_sweep(work, g, ref):
    r = work.regions[0]
    W, T, L = r.team_width, r.teams, r.frame_bytes[0] // 4
    s64, mag, s32 = oracle.sweep_fields(ref)
    g32 = np.ascontiguousarray(g[: T * W]).view(np.float32).reshape(T, W)
    # the oracle's fp32 sum, bit for bit
    assert np.array_equal(g32.view(np.uint32), s32[: T * W].reshape(T, W).view(np.uint32))
    # and within the tolerance of its fp64 sum
    s = s64[: T * W].reshape(T, W)
    mag = mag[: T * W].reshape(T, W)
    n = np.array([max(0, (L - t + W - 1) // W) for t in range(W)], dtype=np.float64)
    gamma = (n - 1).clip(0) * U / (1 - (n - 1).clip(0) * U)
    tol = 1e-6 * np.abs(s) + gamma[None, :] * mag
    assert (np.abs(g32.astype(np.float64) - s) <= tol).all()


@pytest.mark.parametrize("S", list(wl.SWEEP_SIZES))
@pytest.mark.parametrize("where", ["smem", "overflow"])
def test_sweep_512x128(rt, S, where):
    work = wl.sweep(S, teams=512, threads=128)
    if where == "smem":
        if S + 384 > 232448:
            pytest.skip("frame larger than one CTA's shared memory")
        g, gs, r, rs = _run_both(rt, work, slab=S)
        assert (gs["spill_bytes"] == 0).all()
    else:
        g, gs, r, rs = _run_both(rt, work, slab=0, ovf=S, max_teams=512)
        assert (gs["spill_bytes"] == S).all()
    _check_sweep(work, g, r)
    assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()


@pytest.mark.parametrize("S", [4, 20, 1092, 4000, 65540])
def test_sweep_ragged(rt, S):
    work = wl.sweep(S, teams=7, threads=160)
    g, gs, r, rs = _run_both(rt, work, slab=(S + 15) // 16 * 16)
    _check_sweep(work, g, r)
    g2, gs2, r2, rs2 = _run_both(rt, work, slab=0, ovf=(S + 15) // 16 * 16, max_teams=7)
    _check_sweep(work, g2, r2)


# ---------------------------------------------------------------------------
# Hetero program, one instance per plain launch
# ---------------------------------------------------------------------------
def test_hetero_plain_instances(rt):
    work = wl.hetero(n_instances=60, max_teams=40)
    g, gs, r, rs = _run_both(rt, work, slab=3 * 32768)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)


def test_hetero_plain_spill(rt):
    work = wl.hetero(n_instances=30, max_teams=16)
    g, gs, r, rs = _run_both(rt, work, slab=8192, ovf=3 * 32768, max_teams=512)
    assert np.array_equal(g, r)
    _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Occupancy of the plain launch, read from the compiled kernel
# ---------------------------------------------------------------------------
def test_region_occupancy_matches_model_limits(rt):
    import paper_1711_10413_gb300 as dsr
    # nested program, 256 threads: the kernel is held to 32 registers, so
    # the 64-warp limit (8 CTAs of 8 warps) binds, not registers or smem
    r = wl.nested(teams=8, threads=256, depth=3).regions[0]
    _configure(rt, 3264)
    occ = rt.occupancy(r)
    assert occ["threads"] == 256 and occ["smem_per_team"] == 384 + 3264
    assert occ["regs_per_thread"] <= 32 and occ["ctas_per_sm"] == 8
    assert occ["sm_count"] >= 1 and occ["spill_bytes"] == 0
    # a 192 KiB sweep frame in the slab leaves room for one CTA per SM
    s = wl.sweep(196608, teams=2, threads=128).regions[0]
    _configure(rt, 196608)
    occ = rt.occupancy(s)
    assert occ["ctas_per_sm"] == 1 and occ["smem_per_team"] == 384 + 196608
    model = dsr.dsr_footprint_model(s, 196608, occ["regs_per_thread"])
    assert model["teams_per_sm"] == occ["ctas_per_sm"] and model["limit"] == 2
    # the same frame with no slab spills whole to the overflow slab
    _configure(rt, 0, 196608, 2)
    occ = rt.occupancy(s)
    assert occ["spill_bytes"] == 196608 and occ["smem_per_team"] == 384


def test_balanced_residency_caps_ctas_per_sm(rt):
    """A plain launch of more teams than SMs holds at most ceil(teams / SMs)
    of them on an SM (its dynamic shared memory padded past what the
    program uses), when that is below the kernel's occupancy; the results
    are the oracle's either way. Up to the SM count, and at or above the
    occupancy, nothing changes."""
    probe = wl.nested(teams=8, threads=256, depth=3).regions[0]
    _configure(rt, 3264)
    occ8 = rt.occupancy(probe)
    sms, full = occ8["sm_count"], occ8["ctas_per_sm"]
    assert full == 8 and occ8["smem_per_team"] == 384 + 3264
    for teams in (sms + 1, 2 * sms + 1, 5 * sms, 7 * sms, 9 * sms):
        work = wl.nested(teams=teams, threads=256, depth=3, elems_per_team=256, seed=teams)
        occ = rt.occupancy(work.regions[0])
        cap = -(-teams // sms)
        assert occ["ctas_per_sm"] == (cap if cap < full else full), (teams, occ)
        assert occ["smem_per_team"] == 384 + 3264   # what the program uses
        g, gs, r, rs = _run_both(rt, work, slab=3264)
        assert _same_out(g, r)
        _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Worker-level sharing (Sec. 7): per-warp stacks, nested regions on warps
# ---------------------------------------------------------------------------
def _same_out(g, r):
    """The device output buffer is padded to 16 bytes; the rest is zero."""
    return np.array_equal(g[: r.size], r) and not g[r.size:].any()


def _workers_slab(threads, S, frames_per_warp=32):
    fp = (S + 15) // 16 * 16
    return 16 + (threads - 32) // 32 * frames_per_warp * fp


@pytest.mark.parametrize("teams,threads,S,width", [
    (3, 64, 64, 0),       # one worker warp
    (5, 256, 256, 0),     # seven worker warps
    (4, 160, 100, 45),    # ragged width: warps of 32 and 13 workers, one idle
    (2, 1024, 36, 0),     # 31 worker warps, frames of 9 words
    (7, 96, 1028, 33),    # frames of 257 words, a warp with one worker
    (1, 128, 4, 1),       # one worker, one word
    (3, 192, 384, 70),    # frames of 96 words (rows of 32), warps of 32, 32 and 6 workers
    (2, 256, 128, 0),     # frames of one row of 32 words
])
def test_workers_parity(rt, teams, threads, S, width):
    work = wl.workers(teams=teams, threads=threads, frame_bytes=S, width=width)
    g, gs, r, rs = _run_both(rt, work, slab=_workers_slab(threads, S))
    assert _same_out(g, r)
    _assert_status_equal(gs, rs)
    assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()


@pytest.mark.parametrize("teams,threads,S,width,slab_frames", [
    (4, 160, 100, 45, 32),   # the general walk (keys and offsets per step)
    (2, 1024, 36, 0, 32),    # 31 worker warps
    (5, 256, 256, 0, 32),    # rows of 32 words (keys only)
    (3, 192, 200, 70, 9),    # part of each warp's frames on the overflow share
])
def test_workers_smem_table_sharing_equals_shuffles(rt, teams, threads, S, width, slab_frames):
    """The worker program with the nested teams' keys and frame offsets read
    from a shared-memory table (param 1) against the oracle and against the
    shuffle variant (param 0): the same outputs and team records."""
    slab = _workers_slab(threads, S, slab_frames)
    ovf = (threads - 32) * ((S + 15) // 16 * 16)
    outs = []
    for share in (0, 1):
        work = wl.workers(teams=teams, threads=threads, frame_bytes=S, width=width, share=share)
        g, gs, r, rs = _run_both(rt, work, slab=slab, ovf=ovf, max_teams=teams)
        assert _same_out(g, r)
        _assert_status_equal(gs, rs)
        outs.append((g, gs))
    assert np.array_equal(outs[0][0], outs[1][0])
    for f in ("status", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(outs[0][1][f], outs[1][1][f]), f


@pytest.mark.parametrize("S", [200, 256])  # frames of 50 words; of two rows of 32
def test_workers_spill_to_overflow_shares(rt, S):
    fp = (S + 15) // 16 * 16
    work = wl.workers(teams=6, threads=96, frame_bytes=S, width=40)
    # slab shares of 10 frames, overflow shares of 22; then all in overflow
    for slab, ovf in [(16 + 2 * 10 * fp, 2 * 22 * fp), (0, 16 + 2 * 32 * fp)]:
        g, gs, r, rs = _run_both(rt, work, slab=slab, ovf=ovf, max_teams=6)
        assert _same_out(g, r)
        _assert_status_equal(gs, rs)
        assert (gs["spill_bytes"] > 0).all()


def test_workers_overflow_reports_like_the_oracle(rt):
    S, fp = 200, 208
    work = wl.workers(teams=3, threads=96, frame_bytes=S, width=40)
    g, gs, r, rs = _run_both(rt, work, slab=16 + 2 * 10 * fp, ovf=2 * 10 * fp, max_teams=3)
    assert _same_out(g, r)  # the workers whose frames fitted, and zeros
    _assert_status_equal(gs, rs)
    assert (gs["status"] == 2).all()


def test_workers_full_size(rt):
    """The bench's workload: 1024 teams x 256 threads, 256-byte worker frames
    (224 frames of 256 bytes per team, 56 KiB of warp stacks)."""
    work = wl.workers(teams=1024, threads=256, frame_bytes=256)
    g, gs, r, rs = _run_both(rt, work, slab=_workers_slab(256, 256))
    assert _same_out(g, r)
    _assert_status_equal(gs, rs)


# ---------------------------------------------------------------------------
# Shared memory sized per launch from the footprint estimate (DSR_SLAB_AUTO)
# ---------------------------------------------------------------------------
def test_auto_slab_holds_every_frame(rt):
    import paper_1711_10413_gb300 as dsr
    works = [wl.nested(teams=16, threads=256, depth=3), wl.sweep(98304, teams=8),
             wl.workers(teams=6, threads=160, frame_bytes=100, width=45),
             wl.hetero(30, max_teams=8, max_frame=8192), wl.paper_arrays(2, teams=3)]
    for work in works:
        rt.configure(dsr.DSR_SLAB_AUTO, 0, 0)
        for region in work.regions:
            occ = rt.occupancy(region)
            assert occ["smem_per_team"] == 384 + dsr.dsr_region_footprint(region)[1]
            assert occ["spill_bytes"] == 0
        g, gs = rt.run_workload(work)
        r, rs = oracle.run_workload(work, slab_bytes=1 << 40, overflow_bytes=0)
        if work.out_dtype == "float32":
            _check_sweep(work, g, r)
        else:
            assert _same_out(g, r)
        _assert_status_equal(gs, rs)
        assert (gs["spill_bytes"] == 0).all() and (gs["status"] == 0).all()


# ---------------------------------------------------------------------------
# The host-buffer path (images in and results out through pinned memory)
# ---------------------------------------------------------------------------
def test_run_region_host_matches_oracle(rt):
    import torch

    import paper_1711_10413_gb300 as dsr
    cases = [(wl.nested(teams=12, threads=256, depth=3), 3264),
             (wl.paper_scalars(9, teams=5), 4096),       # output updated in place
             (wl.sweep(8192, teams=6), 8192)]
    for work, slab in cases:
        rt.configure(slab, 0, 0)
        region = work.regions[0]
        ib, ob, ns = dsr.dsr_region_extent(region)
        images, out, status = rt.device_buffers(work)
        img_h = torch.from_numpy(np.ascontiguousarray(work.images)).pin_memory()
        out_h = torch.zeros(out.numel(), dtype=torch.int32).pin_memory()
        if work.out_init is not None:
            out_h[: work.out_init.size] = torch.from_numpy(work.out_init)
        out.fill_(-1)  # stale device contents must not reach the host
        st_h = torch.zeros(status.numel(), dtype=torch.int32).pin_memory()
        dsr.dsr_run_region_host(rt.ctx, region, img_h, ib, out_h, ob, st_h, images, out, status)
        g = out_h.numpy()
        gs = st_h.numpy().view(dsr.TEAM_STATUS_DTYPE)
        r, rs = oracle.run_workload(work, slab_bytes=slab)
        if work.out_dtype == "float32":
            _check_sweep(work, g.view(np.float32), r)
        else:
            assert _same_out(g[: ob // 4], r[: ob // 4])
        _assert_status_equal(gs, rs)
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_run_region_host(rt.ctx, region, img_h, ib, None, ob, st_h, images, out, status)
    assert ei.value.code == dsr.DSR_ERR_INVALID


def test_enqueue_region_host_pipelines_on_two_streams(rt):
    """Eight steps enqueued on two streams without synchronisation, each
    step with its own input images (a different seed), device buffers and
    pinned host outputs; a slot's device buffers are reused two steps later
    on the same stream. After one synchronisation every host output and
    status record equals the oracle's for that step's inputs."""
    import torch

    import paper_1711_10413_gb300 as dsr
    T, slab = 256, 3264
    rt.configure(slab, 0, 0)
    works = [wl.nested(teams=T, threads=256, depth=3, seed=100 + i) for i in range(8)]
    region = works[0].regions[0]
    ib, ob, _ = dsr.dsr_region_extent(region)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    slots = [rt.device_buffers(works[0]) for _ in streams]
    torch.cuda.synchronize()  # the slots' set-up ran on the default stream
    host = []
    for i, work in enumerate(works):
        img_h = torch.from_numpy(np.ascontiguousarray(work.images)).pin_memory()
        out_h = torch.full((ob // 4,), -1, dtype=torch.int32).pin_memory()
        st_h = torch.zeros(T * 8, dtype=torch.int32).pin_memory()
        images, out, status = slots[i % 2]
        dsr.dsr_enqueue_region_host(rt.ctx, region, img_h, ib, out_h, ob, st_h, images, out,
                                    status, streams[i % 2].cuda_stream)
        host.append((img_h, out_h, st_h))
    torch.cuda.synchronize()
    for work, (_, out_h, st_h) in zip(works, host):
        r, rs = oracle.run_workload(work, slab_bytes=slab)
        assert np.array_equal(out_h.numpy(), r[: ob // 4])
        _assert_status_equal(st_h.numpy().view(dsr.TEAM_STATUS_DTYPE), rs)


def test_region_reads_the_previous_regions_output(rt):
    """Back to back in one stream with no synchronisation between them, region
    B's init images are region A's output. The plain launch lets B's CTAs be
    placed while A still runs (A's 512 teams leave most of the GPU's CTA
    slots free), so B is right only if none of B's threads reads global
    memory before A has completed. Six pairs on fresh buffers, all launched
    before one synchronisation; both regions checked against the oracle."""
    import torch
    import paper_1711_10413_gb300 as dsr
    T = 512
    a = wl.nested(teams=T, threads=256, depth=3, elems_per_team=4096, seed=11)
    ref_a, ref_as = oracle.run_workload(a, slab_bytes=3264)
    b = wl.nested(teams=T, threads=256, depth=3, elems_per_team=4096, seed=12)
    assert a.out_bytes >= len(b.images)
    b_on_a = wl.Workload("nested_on_a", b.regions, np.ascontiguousarray(ref_a.view(np.uint8)),
                         b.out_bytes, b.n_status)
    ref_b, ref_bs = oracle.run_workload(b_on_a, slab_bytes=3264)
    _configure(rt, 3264)
    img_a, _, _ = rt.device_buffers(a)
    pairs = []
    for _ in range(6):
        out_a = torch.empty(a.out_bytes // 4, dtype=torch.int32, device="cuda")
        st_a = torch.zeros(a.n_status * 8, dtype=torch.int32, device="cuda")
        out_b = torch.empty(b.out_bytes // 4, dtype=torch.int32, device="cuda")
        st_b = torch.zeros(b.n_status * 8, dtype=torch.int32, device="cuda")
        rt.launch(a.regions[0], img_a, out_a, st_a)
        rt.launch(b.regions[0], out_a.view(torch.uint8), out_b, st_b)
        pairs.append((out_a, st_a, out_b, st_b))
    torch.cuda.synchronize()
    for out_a, st_a, out_b, st_b in pairs:
        assert np.array_equal(out_a.cpu().numpy(), ref_a)
        _assert_status_equal(st_a.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE), ref_as)
        assert np.array_equal(out_b.cpu().numpy(), ref_b)
        _assert_status_equal(st_b.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE), ref_bs)
