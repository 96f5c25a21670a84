"""Batched launch form on the GPU: many heterogeneous region instances in
one persistent kernel, checked against the CPU oracle (bit for bit)."""
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
    r.close()


def _regions_equal(work, sel, g, gs, r, rs):
    """Compare the outputs and statuses of the selected regions."""
    for i in sel:
        reg = work.regions[i]
        o0, n = reg.out_offset // 4, reg.teams * reg.team_width
        assert np.array_equal(g[o0:o0 + n], r[o0:o0 + n]), "instance %d output" % i
        s0 = reg.status_index
        for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
            assert np.array_equal(gs[f][s0:s0 + reg.teams], rs[f][s0:s0 + reg.teams]), (i, f)


def test_batch_small_full_parity(rt):
    work = wl.hetero(n_instances=300, max_teams=40)
    for tuning in [None, dict(threads=128, slab_bytes=4096), dict(threads=1024, slab_bytes=98304)]:
        g, gs = rt.run_batch(work, tuning)
        r, rs = oracle.run_workload(work, slab_bytes=(tuning or {}).get("slab_bytes", 16384),
                                    overflow_bytes=3 * 32768)
        assert np.array_equal(g, r)
        for f in ("status", "depth_final", "hwm_bytes", "chk"):
            assert np.array_equal(gs[f], rs[f]), f
        assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()


def test_batch_10000_instances_sampled(rt):
    """10,000 instances in one persistent launch; the oracle checks a seeded
    sample of instances plus the largest and the widest ones."""
    work = wl.hetero(n_instances=10000)
    b = rt.batch_buffers(work)
    rt.launch_batch(b, dict(threads=256, slab_bytes=32768), use_graph=True)
    rt.torch.cuda.synchronize()
    g, gs = rt.fetch(b, work)
    assert rt.batch_errors(b) == (0, b["total"])
    assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()
    rng = np.random.default_rng(0)
    sel = set(rng.choice(10000, 120, replace=False).tolist())
    sizes = [sum(r.frame_bytes) * r.teams for r in work.regions]
    sel |= set(np.argsort(sizes)[-5:].tolist())
    sel |= set(np.argsort([r.threads for r in work.regions])[-3:].tolist())
    r, rs = oracle.run_workload(work, slab_bytes=32768, overflow_bytes=3 * 32768,
                                regions=sorted(sel))
    _regions_equal(work, sorted(sel), g, gs, r, rs)
    # hwm of every team equals its frames' reserved sizes
    for reg in work.regions:
        need = sum((x + 15) // 16 * 16 for x in reg.frame_bytes)
        assert (gs["hwm_bytes"][reg.status_index: reg.status_index + reg.teams] == need).all()


def test_batch_spills_to_overflow(rt):
    work = wl.hetero(n_instances=200, max_teams=16)
    g, gs = rt.run_batch(work, dict(threads=256, slab_bytes=1024))
    r, rs = oracle.run_workload(work, slab_bytes=1024, overflow_bytes=3 * 32768)
    assert np.array_equal(g, r)
    assert np.array_equal(gs["spill_bytes"], rs["spill_bytes"])
    assert gs["spill_bytes"].max() > 0


def test_batch_graph_replay_and_reuse(rt):
    work = wl.hetero(n_instances=100, max_teams=8)
    b = rt.batch_buffers(work)
    rt.launch_batch(b, None, use_graph=True)
    rt.torch.cuda.synchronize()
    g1 = b["out"].clone()
    b["out"].zero_()
    rt.launch_batch(b, None, use_graph=True)   # replay of the captured graph
    rt.torch.cuda.synchronize()
    assert rt.torch.equal(g1, b["out"])
    r, _ = oracle.run_workload(work, slab_bytes=16384, overflow_bytes=3 * 32768)
    assert np.array_equal(g1.cpu().numpy(), r)


def test_batch_matches_per_region_launches(rt):
    """Each instance's output is the same alone (its own launch) and in the
    batch."""
    work = wl.hetero(n_instances=80, max_teams=12)
    b = rt.batch_buffers(work)
    rt.launch_regions(b)
    rt.torch.cuda.synchronize()
    alone = b["out"].cpu().numpy().copy()
    st_alone = b["status"].cpu().numpy().copy()
    b["out"].zero_()
    b["status"].zero_()
    rt.launch_batch(b, dict(threads=512, slab_bytes=16384))
    rt.torch.cuda.synchronize()
    assert np.array_equal(alone, b["out"].cpu().numpy())
    assert np.array_equal(st_alone, b["status"].cpu().numpy())


def test_batch_rejects_bad_descriptors_on_device(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=50, max_teams=6)
    b = rt.batch_buffers(work)
    descs = b["descs"].copy()
    descs[3]["image_offset"] = 1 << 40          # past the image buffer
    descs[7]["program"] = dsr.DSR_PROG_NESTED   # another program
    descs[9]["frame_bytes"][0] = 6              # not a multiple of 4
    b["descs_dev"].copy_(rt.torch.from_numpy(descs.view(np.uint8)))
    rt.launch_batch(b)
    rt.torch.cuda.synchronize()
    errors, counted = rt.batch_errors(b)
    bad = {3, 7, 9}
    assert errors == sum(work.regions[i].teams for i in bad)
    g, gs = rt.fetch(b, work)
    r, rs = oracle.run_workload(work, slab_bytes=16384, overflow_bytes=3 * 32768)
    for i, reg in enumerate(work.regions):
        rows = gs["status"][reg.status_index: reg.status_index + reg.teams]
        if i in bad:
            assert (rows == dsr.DSR_ERR_INVALID).all()
        else:
            assert (rows == 0).all()
    _regions_equal(work, [i for i in range(50) if i not in bad], g, gs, r, rs)


def test_batch_other_programs(rt):
    """The persistent kernel runs every program: nested and scalars as batches."""
    nested = wl.nested(teams=300, threads=256, depth=3)
    g, gs = rt.run_batch(nested, dict(threads=256, slab_bytes=4096))
    r, rs = oracle.run_workload(nested, slab_bytes=4096)
    assert np.array_equal(g, r) and np.array_equal(gs["chk"], rs["chk"])
    sc = wl.scalars(n_regions=100, teams=3, threads=128)
    g, gs = rt.run_batch(sc, dict(threads=128, slab_bytes=1024))
    r, rs = oracle.run_workload(sc, slab_bytes=1024)
    assert np.array_equal(g, r)


def test_autotune_returns_fitting_shape(rt):
    work = wl.hetero(n_instances=400, max_teams=32)
    b = rt.batch_buffers(work)
    best, ms = rt.autotune(b)
    assert best["threads"] % 32 == 0 and 64 <= best["threads"] <= 1024 and ms > 0
    rt.torch.cuda.synchronize()
    g, gs = rt.fetch(b, work)
    r, rs = oracle.run_workload(work, slab_bytes=best["slab_bytes"], overflow_bytes=3 * 32768)
    assert np.array_equal(g, r)


def test_autotune_cache_hits_for_the_same_class(rt, tmp_path):
    """The second batch of one distribution takes the tuned shape from the
    cache file without tuning, and runs correctly with it."""
    path = str(tmp_path / "tuning.json")
    b1 = rt.batch_buffers(wl.hetero(n_instances=300, max_teams=32, seed=5))
    best, ms, hit = rt.autotune_cached(b1, path)
    assert not hit and ms > 0
    work = wl.hetero(n_instances=300, max_teams=32, seed=6)
    b2 = rt.batch_buffers(work)
    best2, _, hit2 = rt.autotune_cached(b2, path)
    assert hit2 and best2 == best
    rt.launch_batch(b2, best2)
    rt.torch.cuda.synchronize()
    g, gs = rt.fetch(b2, work)
    r, rs = oracle.run_workload(work, slab_bytes=best2["slab_bytes"], overflow_bytes=3 * 32768)
    assert np.array_equal(g, r) and (gs["status"] == 0).all()


def _sweep_batch(sizes, teams, threads=128, seed=7):
    """Several sweep instances in one batch: instance i has `teams` teams of
    one fp32 frame of sizes[i] bytes, its images and outputs packed."""
    regions, chunks = [], []
    img_off = out_off = st = 0
    w = threads - 32
    for i, S in enumerate(sizes):
        imgs = wl.normal_f32(wl.derive(seed, 30, i, S), teams * (S // 4))
        regions.append(wl.Region(wl.PROG_SWEEP, teams, threads, 1, [S], status_index=st,
                                 image_offset=img_off, out_offset=out_off))
        chunks.append(imgs.view(np.uint8))
        img_off += imgs.nbytes
        out_off += 4 * teams * w
        st += teams
    return wl.Workload("sweep_batch", regions, np.concatenate(chunks), out_off, st,
                       out_dtype="float32")


def test_batch_sweep_streams_across_tasks():
    """The sweep program in the persistent kernel: frames of 32 and 96 KiB
    take the streamed fill (chunk mbarriers set up on a CTA's first streamed
    task, their parity carried from task to task), 8 KiB frames the plain
    bulk fill, interleaved in one CTA. Each CTA runs several tasks. Results
    as the fp32 left-to-right sums of the oracle's order, every team OK."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    rt = dsr.Runtime(0, slab_bytes=16384, wait_timeout_ns=50_000_000)
    try:
        work = _sweep_batch([32768, 8192, 98304, 32768, 8192], teams=120)
        g, gs = rt.run_batch(work, dict(threads=128, slab_bytes=98304, ctas_per_sm=1))
        assert (gs["status"] == 0).all() and (gs["depth_final"] == 0).all()
        assert (gs["spill_bytes"] == 0).all()
        r, _ = oracle.run_workload(work)
        for reg in work.regions:
            T, W, L = reg.teams, reg.team_width, reg.frame_bytes[0] // 4
            o0 = reg.out_offset // 4
            got = g[o0:o0 + T * W].reshape(T, W)
            s64, mag, s32 = oracle.sweep_fields(r[3 * o0: 3 * (o0 + T * W)])
            # the oracle's fp32 index-order sum, bit for bit
            assert np.array_equal(got.view(np.uint32), s32.reshape(T, W).view(np.uint32))
            n = np.array([max(0, (L - t + W - 1) // W) for t in range(W)], dtype=np.float64)
            gamma = (n - 1).clip(0) * 2.0 ** -24 / (1 - (n - 1).clip(0) * 2.0 ** -24)
            tol = 1e-6 * np.abs(s64.reshape(T, W)) + gamma[None, :] * mag.reshape(T, W)
            assert (np.abs(got.astype(np.float64) - s64.reshape(T, W)) <= tol).all()
    finally:
        rt.close()


def test_batch_abort_stops_a_running_batch():
    """dsr_batch_abort on a running 10,000-instance batch: its CTAs stop taking
    tasks, fewer tasks are taken than counted, every team that ran has the
    same output row and record as in a full run, the others were not
    touched, and the next launch on the same workspace runs to completion
    (the scan clears the flag)."""
    import time

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    rt = dsr.Runtime(0, slab_bytes=16384, overflow_bytes_per_team=3 * 32768, max_teams=4096)
    try:
        work = wl.hetero(n_instances=10000)
        b = rt.batch_buffers(work)
        tuning = dict(threads=128, slab_bytes=8192, ctas_per_sm=0)
        rt.launch_batch(b, tuning)
        torch.cuda.synchronize()
        full_out = b["out"].cpu().numpy().copy()
        full_st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE).copy()
        assert dsr.dsr_batch_progress(rt.ctx, b["ws"]) == (b["total"], b["total"])
        b["out"].fill_(-7)
        b["status"].fill_(-1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt.launch_batch(b, tuning)
        time.sleep(0.002)   # the batch takes about 5 ms
        dsr.dsr_batch_abort(rt.ctx, b["ws"])
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        taken, counted = dsr.dsr_batch_progress(rt.ctx, b["ws"])
        assert counted == b["total"] and 0 < taken < counted, (taken, counted, elapsed)
        st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
        out = b["out"].cpu().numpy()
        ran = st["status"] != -1
        assert int(ran.sum()) == taken
        for f in ("status", "depth_final", "hwm_bytes", "chk"):
            assert np.array_equal(st[f][ran], full_st[f][ran]), f
        # element mask: team t of an instance owns W' consecutive output words
        mask = np.zeros(out.size, dtype=bool)
        covered = np.zeros(out.size, dtype=bool)
        for r in work.regions:
            W, o0 = r.team_width, r.out_offset // 4
            mask[o0:o0 + r.teams * W] = np.repeat(ran[r.status_index:r.status_index + r.teams], W)
            covered[o0:o0 + r.teams * W] = True
        assert np.array_equal(out[mask], full_out[mask])
        assert (out[covered & ~mask] == -7).all()
        # the next launch runs everything
        rt.launch_batch(b, tuning)
        torch.cuda.synchronize()
        assert dsr.dsr_batch_progress(rt.ctx, b["ws"]) == (b["total"], b["total"])
        again = b["out"].cpu().numpy()
        assert np.array_equal(again[covered], full_out[covered])  # padding between rows aside
    finally:
        rt.close()
