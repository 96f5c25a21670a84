"""Region programs written against the public device API (include/
dsr_device.cuh), outside the library, run through its plain and batched
launches and compared with the CPU oracle running the same definitions:
the paper's "8 variables" program (Sec. 6.1, the oracle's PX1) and the
heterogeneous-instance program (the oracle's P4). Outputs and team records
(status, depth left, peak stack bytes, peak overflow bytes, check words)
must agree bit for bit, with frames in the slab and spilled."""
import copy
import ctypes
import os

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "user_program", "user_programs.cu")
LIB = os.path.join(ROOT, "tests", "user_program", "libuser_programs.so")


@pytest.fixture(scope="module")
def user():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    from paper_1711_10413_gb300 import builder
    builder.build_user([SRC], LIB)
    L = ctypes.CDLL(LIB)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    for name in ("user_paper_scalars", "user_hetero"):
        f = getattr(L, name + "_launch")
        f.restype = i32
        f.argtypes = [vp, ctypes.POINTER(dsr.dsr_region_desc), vp, u64, vp, u64, vp, u64, vp]
        f = getattr(L, name + "_launch_batch")
        f.restype = i32
        f.argtypes = [vp, vp, u32, u64, vp, u64, vp, u64, vp, u64, vp, u64,
                      ctypes.POINTER(dsr.dsr_batch_tuning), vp]
        f = getattr(L, name + "_program")
        f.restype = u32
    rt = dsr.Runtime(0, slab_bytes=16384, overflow_bytes_per_team=3 * 32768, max_teams=4096)
    yield L, rt
    rt.close()


def _as_user(work, program):
    """The same workload with its descriptors naming a user program id."""
    w = copy.copy(work)
    w.regions = [copy.copy(r) for r in work.regions]
    for r in w.regions:
        r.program = program
    return w


def _check(rc, rt):
    import paper_1711_10413_gb300 as dsr
    if rc != 0:
        raise dsr.DsrError(rc, dsr.lib().dsr_last_error_string(rt.ctx).decode())


def _plain(L, rt, name, work):
    """Every region of `work` through <name>_launch; (output, statuses)."""
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    images, out, status = rt.device_buffers(work)
    launch = getattr(L, name + "_launch")
    s = torch.cuda.current_stream().cuda_stream
    for r in work.regions:
        d = dsr.pack_desc(r)
        _check(launch(rt.ctx, ctypes.byref(d), images.data_ptr(), images.numel(),
                      out.data_ptr(), out.numel() * 4, status.data_ptr(), status.numel() // 8,
                      s), rt)
    torch.cuda.synchronize()
    return out.cpu().numpy(), status.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)


def _batch(L, rt, name, work, tuning):
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    b = rt.batch_buffers(work)
    t = dsr.dsr_batch_tuning(tuning["threads"], tuning["slab_bytes"], 0, 0)
    launch = getattr(L, name + "_launch_batch")
    _check(launch(rt.ctx, b["descs_dev"].data_ptr(), len(b["descs"]), b["total"],
                  b["images"].data_ptr(), b["images"].numel(), b["out"].data_ptr(),
                  b["out"].numel() * 4, b["status"].data_ptr(), b["status"].numel() // 8,
                  b["ws"].data_ptr(), b["ws"].numel(), ctypes.byref(t),
                  torch.cuda.current_stream().cuda_stream), rt)
    torch.cuda.synchronize()
    errors, counted = rt.batch_errors(b)
    return (b["out"].cpu().numpy(), b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE),
            errors, counted, b["total"])


def _same_status(g, r):
    for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(g[f], r[f]), f


@pytest.mark.parametrize("n_vars,threads,teams", [(7, 128, 4), (1, 64, 3), (20, 96, 5),
                                                  (64, 1024, 2), (7, 32, 3)])
def test_user_paper_scalars_plain(user, n_vars, threads, teams):
    L, rt = user
    work = wl.paper_scalars(n_vars, teams=teams, threads=threads)
    uw = _as_user(work, L.user_paper_scalars_program())
    rt.configure(4096, 0, 0)
    g, gs = _plain(L, rt, "user_paper_scalars", uw)
    r, rs = oracle.run_workload(work, slab_bytes=4096)
    n = work.out_bytes // 4
    assert np.array_equal(g[:n], r[:n])
    _same_status(gs, rs)
    # the closed form: a + n(n+1)/2 in every slot
    a0 = work.out_init.astype(np.int64)
    assert np.array_equal(g[:n].astype(np.int64), (a0 + n_vars * (n_vars + 1) // 2 + 2 ** 31)
                          % 2 ** 32 - 2 ** 31)


def test_user_paper_scalars_spilled(user):
    """The frame in the overflow slab: the same results."""
    L, rt = user
    work = wl.paper_scalars(30, teams=6)
    uw = _as_user(work, L.user_paper_scalars_program())
    rt.configure(0, 256, 64)
    g, gs = _plain(L, rt, "user_paper_scalars", uw)
    r, rs = oracle.run_workload(work, slab_bytes=0, overflow_bytes=256)
    assert np.array_equal(g[: r.size], r)
    _same_status(gs, rs)
    assert (gs["spill_bytes"] > 0).all()


@pytest.mark.parametrize("slab,ovf", [(16384, 3 * 32768), (1024, 3 * 32768), (0, 3 * 32768)])
def test_user_hetero_plain(user, slab, ovf):
    L, rt = user
    work = wl.hetero(n_instances=40, max_teams=16, max_frame=8192, seed=11)
    uw = _as_user(work, L.user_hetero_program())
    rt.configure(slab, ovf, 64)
    g, gs = _plain(L, rt, "user_hetero", uw)
    r, rs = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=ovf)
    assert np.array_equal(g[: r.size], r)
    _same_status(gs, rs)
    assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()


def test_user_hetero_matches_builtin_program(user):
    """The user-written program and the built-in one agree on the GPU too."""
    L, rt = user
    work = wl.hetero(n_instances=30, max_teams=8, max_frame=4096, seed=5)
    rt.configure(4096, 3 * 32768, 64)
    g_user, s_user = _plain(L, rt, "user_hetero", _as_user(work, L.user_hetero_program()))
    g_lib, s_lib = rt.run_workload(work)
    assert np.array_equal(g_user, g_lib)
    _same_status(s_user, s_lib)


@pytest.mark.parametrize("threads,slab", [(128, 8192), (256, 16384), (1024, 4096)])
def test_user_hetero_batch(user, threads, slab):
    L, rt = user
    work = wl.hetero(n_instances=300, max_teams=32, max_frame=16384, seed=3)
    uw = _as_user(work, L.user_hetero_program())
    rt.configure(16384, 3 * 32768, 4096)
    g, gs, errors, counted, total = _batch(L, rt, "user_hetero", uw,
                                           dict(threads=threads, slab_bytes=slab))
    r, rs = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=3 * 32768)
    assert errors == 0 and counted == total
    assert np.array_equal(g[: r.size], r)
    # the batched form's placement is per CTA: compare what is placement-free
    for f in ("status", "depth_final", "hwm_bytes", "chk"):
        assert np.array_equal(gs[f], rs[f]), f


def test_user_paper_scalars_batch(user):
    L, rt = user
    regions, out_off, st = [], 0, 0
    init = []
    for i, (n, teams, threads) in enumerate([(7, 4, 128), (3, 9, 64), (12, 2, 512), (1, 5, 32)]):
        w = wl.paper_scalars(n, teams=teams, threads=threads, seed=100 + i)
        r = copy.copy(w.regions[0])
        r.out_offset, r.status_index = out_off, st
        regions.append(r)
        init.append(w.out_init)
        pad = (-w.out_init.size) % 4
        init.append(np.zeros(pad, np.int32))
        out_off += 4 * (w.out_init.size + pad)
        st += teams
    a0 = np.concatenate(init)
    work = wl.Workload("paper_scalars_batch", regions, np.zeros(16, np.uint8), out_off, st,
                       out_init=a0)
    uw = _as_user(work, L.user_paper_scalars_program())
    rt.configure(4096, 0, 0)
    g, gs, errors, counted, total = _batch(L, rt, "user_paper_scalars", uw,
                                           dict(threads=128, slab_bytes=4096))
    r, rs = oracle.run_workload(work)
    assert errors == 0 and counted == total
    assert np.array_equal(g[: r.size], r)
    _same_status(gs, rs)


def test_user_batch_rejects_other_programs(user):
    """A descriptor naming another program is rejected on the device (its
    teams report INVALID), the others run."""
    import paper_1711_10413_gb300 as dsr
    L, rt = user
    work = wl.hetero(n_instances=20, max_teams=4, max_frame=1024, seed=9)
    uw = _as_user(work, L.user_hetero_program())
    uw.regions[3].program = dsr.DSR_PROG_HETERO  # a built-in id in a user batch
    rt.configure(16384, 3 * 32768, 4096)
    g, gs, errors, counted, total = _batch(L, rt, "user_hetero", uw,
                                           dict(threads=128, slab_bytes=8192))
    bad = uw.regions[3]
    assert errors == bad.teams
    assert (gs["status"][bad.status_index: bad.status_index + bad.teams] == 1).all()
    others = np.ones(len(gs), bool)
    others[bad.status_index: bad.status_index + bad.teams] = False
    assert (gs["status"][others] == 0).all()


def test_user_plain_refusals(user):
    """Host-side refusals, nothing launched: a descriptor naming another
    program, a built-in launch of a user id, and outputs too small."""
    import paper_1711_10413_gb300 as dsr
    L, rt = user
    work = wl.hetero(n_instances=2, max_teams=4, max_frame=1024, seed=2)
    rt.configure(4096, 0, 0)
    images, out, status = rt.device_buffers(work)
    d = dsr.pack_desc(work.regions[0])  # built-in id through the user launch
    rc = L.user_hetero_launch(rt.ctx, ctypes.byref(d), images.data_ptr(), images.numel(),
                              out.data_ptr(), out.numel() * 4, status.data_ptr(),
                              status.numel() // 8, None)
    assert rc == dsr.DSR_ERR_INVALID
    uw = _as_user(work, L.user_hetero_program())
    with pytest.raises(dsr.DsrError) as ei:   # user id through the built-in launch
        dsr.dsr_launch_region(rt.ctx, uw.regions[0], images, out, status)
    assert "user-written" in str(ei.value)
    d = dsr.pack_desc(uw.regions[0])
    rc = L.user_hetero_launch(rt.ctx, ctypes.byref(d), images.data_ptr(), images.numel(),
                              out.data_ptr(), 4, status.data_ptr(), status.numel() // 8, None)
    assert rc == dsr.DSR_ERR_INVALID
    assert "outputs" in dsr.lib().dsr_last_error_string(rt.ctx).decode()
    cfg = dsr.dsr_user_plain_config(rt.ctx, uw.regions[0], 0, 16, 0, out.numel() * 4,
                                    status.numel() // 8, out, status)
    assert cfg["slab_bytes"] == 4096 and cfg["ctrl_bytes"] == 384


def _serve_user(L, rt, name, work, threads, slab, capacity=64):
    """Every region of `work` (naming the user program) through a server of
    <name>'s program started with dsr_serve_user_start; (output, statuses,
    completion statuses)."""
    import time
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    images, out, status = rt.device_buffers(work)
    ws = torch.empty(dsr.dsr_serve_workspace_bytes(capacity), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    start = getattr(L, name + "_serve_start")
    start.restype = ctypes.c_int32
    start.argtypes = [ctypes.c_void_p, ctypes.POINTER(dsr.dsr_serve_cfg), ctypes.c_void_p,
                      ctypes.c_uint64]
    cfg = dsr.serve_cfg(work.regions[0].program, images, out, status, threads, slab, capacity)
    _check(start(rt.ctx, ctypes.byref(cfg), ws.data_ptr(), ws.numel()), rt)
    done = {}
    try:
        tickets, pending, t0 = [], list(work.regions), time.time()
        while pending:
            assert time.time() - t0 < 30
            tk = dsr.dsr_serve_submit(rt.ctx, pending[0])
            if tk is None:      # admission waits for completions
                dsr.dsr_serve_poll(rt.ctx, 1 << 62)
                continue
            tickets.append(tk)
            pending.pop(0)
        left = set(tickets)
        while left:
            assert time.time() - t0 < 30, "requests did not complete"
            for tk in list(left):
                st = dsr.dsr_serve_poll(rt.ctx, tk)
                if st != dsr.DSR_PENDING:
                    done[tk] = st
                    left.discard(tk)
    finally:
        dsr.dsr_serve_stop(rt.ctx)
    torch.cuda.synchronize()
    return out.cpu().numpy(), status.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE), done


@pytest.mark.parametrize("threads,slab", [(128, 8192), (256, 16384)])
def test_user_hetero_served(user, threads, slab):
    """The user-written hetero program served by the library's request loop
    (dsr_serve_user_start: the server kernel instantiated in the program's
    own library), many requests in flight at once: every output and team
    record equals the oracle's."""
    import paper_1711_10413_gb300 as dsr
    L, rt = user
    work = wl.hetero(n_instances=120, max_teams=24, max_frame=16384, seed=17)
    uw = _as_user(work, L.user_hetero_program())
    rt.configure(16384, 3 * 32768, 4096)
    g, gs, done = _serve_user(L, rt, "user_hetero", uw, threads, slab)
    assert len(done) == len(uw.regions) and all(v == dsr.DSR_OK for v in done.values())
    r, rs = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=3 * 32768)
    assert np.array_equal(g[: r.size], r)
    for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(gs[f], rs[f]), f
    stats = dsr.dsr_serve_stats(rt.ctx)
    assert stats["errors"] == 0


def test_user_serve_refusals(user):
    """Host-side refusals with a user program's server: a built-in program's
    descriptor, and a request indexing past the outputs (nothing runs for
    either); the built-in start refuses a user id."""
    import paper_1711_10413_gb300 as dsr
    L, rt = user
    torch = rt.torch
    work = wl.hetero(n_instances=3, max_teams=4, max_frame=1024, seed=8)
    uw = _as_user(work, L.user_hetero_program())
    rt.configure(16384, 3 * 32768, 4096)
    images, out, status = rt.device_buffers(uw)
    ws = torch.empty(dsr.dsr_serve_workspace_bytes(16), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_serve_start(rt.ctx, uw.regions[0].program, images, out, status, ws,
                            capacity=16)
    assert "dsr_serve_start_user" in str(ei.value)
    L.user_hetero_serve_start.restype = ctypes.c_int32
    L.user_hetero_serve_start.argtypes = [ctypes.c_void_p, ctypes.POINTER(dsr.dsr_serve_cfg),
                                          ctypes.c_void_p, ctypes.c_uint64]
    cfg = dsr.serve_cfg(uw.regions[0].program, images, out, status, 128, 8192, 16)
    _check(L.user_hetero_serve_start(rt.ctx, ctypes.byref(cfg), ws.data_ptr(), ws.numel()), rt)
    try:
        bad = copy.copy(work.regions[0])  # the built-in program's id
        with pytest.raises(dsr.DsrError):
            dsr.dsr_serve_submit(rt.ctx, bad)
        far = copy.copy(uw.regions[0])
        far.out_offset = out.numel() * 4   # past the outputs
        with pytest.raises(dsr.DsrError) as ei:
            dsr.dsr_serve_submit(rt.ctx, far)
        assert "refused" in str(ei.value)
        tk = dsr.dsr_serve_submit(rt.ctx, uw.regions[1])
        assert tk is not None
    finally:
        dsr.dsr_serve_stop(rt.ctx)
    assert dsr.dsr_serve_stats(rt.ctx)["completed"] == 1


def test_user_plain_launch_with_more_teams_than_sms(user):
    """A user program's plain launch of more teams than SMs goes through the
    same balanced-residency padding as the library's (the launch template
    asks for it): the results are the oracle's."""
    import torch
    L, rt = user
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for teams in (2 * sms + 1, 5 * sms):
        work = wl.paper_scalars(9, teams=teams, threads=128, seed=teams)
        uw = _as_user(work, L.user_paper_scalars_program())
        rt.configure(4096, 0, 0)
        g, gs = _plain(L, rt, "user_paper_scalars", uw)
        r, rs = oracle.run_workload(work, slab_bytes=4096)
        assert np.array_equal(g[: r.size], r)
        _same_status(gs, rs)
