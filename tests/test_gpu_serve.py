"""Served form on the GPU: a device-resident request loop with continuous
batching. Every request's result must equal the oracle's (and so its
result alone), whatever else was in flight with it."""
import time

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    dsr.build()
    r = dsr.Runtime(0, slab_bytes=16384, overflow_bytes_per_team=3 * 32768, max_teams=4096)
    yield r
    try:
        r.serve_stop()
    except Exception:
        pass
    r.close()


def _submit_all(dsr, rt, regions, deadline_s=30.0):
    tickets, pending = [], list(regions)
    t0 = time.time()
    while pending:
        assert time.time() - t0 < deadline_s
        tk = dsr.dsr_serve_submit(rt.ctx, pending[0])
        if tk is None:          # admission must wait for completions
            dsr.dsr_serve_poll(rt.ctx, 1 << 62)
            continue
        tickets.append(tk)
        pending.pop(0)
    return tickets


def _wait_all(dsr, rt, tickets, deadline_s=30.0):
    st, left, t0 = {}, set(tickets), time.time()
    while left:
        assert time.time() - t0 < deadline_s, "requests did not complete"
        for tk in list(left):
            s = dsr.dsr_serve_poll(rt.ctx, tk)
            if s != dsr.DSR_PENDING:
                st[tk] = s
                left.discard(tk)
    return st


def test_serve_mix_equals_oracle(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=400, max_teams=24)
    b = rt.serve_start(work, threads=128, slab_bytes=8192, capacity=64)
    try:
        tickets = _submit_all(dsr, rt, work.regions)
        st = _wait_all(dsr, rt, tickets)
    finally:
        rt.serve_stop()
    assert all(v == 0 for v in st.values())
    g = b["out"].cpu().numpy()
    gs = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    r, rs = oracle.run_workload(work, slab_bytes=8192, overflow_bytes=3 * 32768)
    assert np.array_equal(g, r)
    for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(gs[f], rs[f]), f
    stats = dsr.dsr_serve_stats(rt.ctx)
    assert stats["submitted"] == stats["completed"] == 400 and stats["errors"] == 0


def test_serve_result_alone_equals_in_the_mix(rt):
    """Every request in flight at once, then a sample of the same requests
    served one at a time (each submitted only after the previous one has
    completed) on fresh buffers: each sampled request's output rows and
    team records are the same in both runs."""
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=200, max_teams=24, seed=9)
    b = rt.serve_start(work, threads=128, slab_bytes=8192, capacity=64)
    try:
        st = _wait_all(dsr, rt, _submit_all(dsr, rt, work.regions))
    finally:
        rt.serve_stop()
    assert all(v == 0 for v in st.values())
    mix_out = b["out"].cpu().numpy()
    mix_st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    sample = sorted(np.random.default_rng(3).choice(200, 12, replace=False).tolist())
    b = rt.serve_start(work, threads=128, slab_bytes=8192, capacity=64)
    try:
        for i in sample:
            st = _wait_all(dsr, rt, _submit_all(dsr, rt, [work.regions[i]]))
            assert list(st.values()) == [0]
    finally:
        rt.serve_stop()
    out = b["out"].cpu().numpy()
    sts = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    for i in sample:
        reg = work.regions[i]
        o0, n = reg.out_offset // 4, reg.teams * reg.team_width
        assert np.array_equal(out[o0:o0 + n], mix_out[o0:o0 + n]), i
        s0 = reg.status_index
        for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
            assert np.array_equal(sts[f][s0:s0 + reg.teams], mix_st[f][s0:s0 + reg.teams]), (i, f)


def test_serve_open_loop_latencies(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=3000, max_teams=64)
    b = rt.serve_start(work, threads=128, slab_bytes=16384, capacity=1024)
    try:
        arr = wl.poisson_arrivals(3000, 100000.0)
        lat, el = dsr.dsr_serve_bench(rt.ctx, b["descs"], arr)
    finally:
        rt.serve_stop()
    assert (lat > 0).all() and el > 0
    r, _ = oracle.run_workload(work, slab_bytes=16384, overflow_bytes=3 * 32768)
    assert np.array_equal(b["out"].cpu().numpy(), r)


def test_serve_small_ring_admission(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=120, max_teams=6)
    b = rt.serve_start(work, threads=128, slab_bytes=4096, capacity=4)
    try:
        budget_hits = 0
        tickets, pending = [], list(work.regions)
        t0 = time.time()
        while pending:
            assert time.time() - t0 < 30
            tk = dsr.dsr_serve_submit(rt.ctx, pending[0])
            if tk is None:
                budget_hits += 1
                dsr.dsr_serve_poll(rt.ctx, 1 << 62)
                continue
            tickets.append(tk)
            pending.pop(0)
        _wait_all(dsr, rt, tickets)
    finally:
        rt.serve_stop()
    assert budget_hits > 0
    r, _ = oracle.run_workload(work, slab_bytes=4096, overflow_bytes=3 * 32768)
    assert np.array_equal(b["out"].cpu().numpy(), r)


def test_serve_idle_exit_and_restart(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=40, max_teams=4)
    b = rt.serve_start(work, threads=128, slab_bytes=16384, capacity=64,
                       idle_timeout_ns=50_000_000)
    try:
        t1 = _submit_all(dsr, rt, work.regions[:20])
        _wait_all(dsr, rt, t1)
        time.sleep(0.5)   # every server CTA leaves after 50 ms without work
        stats = dsr.dsr_serve_stats(rt.ctx)
        assert stats["idle_exits"] > 0, stats
        t2 = _submit_all(dsr, rt, work.regions[20:])
        _wait_all(dsr, rt, t2)
    finally:
        rt.serve_stop()
    r, _ = oracle.run_workload(work, slab_bytes=16384, overflow_bytes=3 * 32768)
    assert np.array_equal(b["out"].cpu().numpy(), r)


def test_serve_nested_program(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.nested(teams=512, threads=256, depth=3)
    b = rt.serve_start(work, threads=256, slab_bytes=4096, capacity=8)
    try:
        st = _wait_all(dsr, rt, _submit_all(dsr, rt, work.regions))
    finally:
        rt.serve_stop()
    assert list(st.values()) == [0]
    r, rs = oracle.run_workload(work, slab_bytes=4096)
    assert np.array_equal(b["out"].cpu().numpy(), r)


def test_serve_rejects_bad_requests_on_the_host(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=10, max_teams=4)
    rt.serve_start(work, threads=128, slab_bytes=4096, capacity=16)
    try:
        bad = dict(work.regions[0].as_dict(), out_offset=1 << 40)
        with pytest.raises(dsr.DsrError) as ei:
            dsr.dsr_serve_submit(rt.ctx, bad)
        assert ei.value.code == dsr.DSR_ERR_INVALID
        other = dict(work.regions[0].as_dict(), program=dsr.DSR_PROG_NESTED)
        with pytest.raises(dsr.DsrError):
            dsr.dsr_serve_submit(rt.ctx, other)
    finally:
        rt.serve_stop()


@pytest.mark.parametrize("threads,slab", [(128, 8192), (256, 16384)])
def test_serve_full_distribution_equals_oracle(rt, threads, slab):
    """The served form on the full heterogeneous distribution (teams
    log-uniform up to 512, threads up to 1024, frames up to 32 KiB, depth 1-3),
    in both server shapes the bench runs: every request's output rows and
    every team's record equal the oracle's, with up to 512 requests in flight
    at once (frames larger than the slab go to each CTA's overflow slab)."""
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=600, seed=44)
    assert max(r.teams for r in work.regions) > 256
    assert max(r.threads for r in work.regions) > 960
    b = rt.serve_start(work, threads=threads, slab_bytes=slab, capacity=512)
    try:
        st = _wait_all(dsr, rt, _submit_all(dsr, rt, work.regions, deadline_s=60.0),
                       deadline_s=60.0)
    finally:
        rt.serve_stop()
    assert all(v == 0 for v in st.values())
    r, rs = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=3 * 32768)
    assert np.array_equal(b["out"].cpu().numpy()[: r.size], r)
    gs = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
        assert np.array_equal(gs[f], rs[f]), f
