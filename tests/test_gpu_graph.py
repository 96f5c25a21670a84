"""Launch graphs (dsr_graph_capture_regions / dsr_graph_launch): plain
launches captured once and replayed with one host call give, launch for
launch, the results the oracle gives, and the capture refuses what a plain
launch refuses."""
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


def _sets(rt, work, n):
    torch = rt.torch
    images, out, status = rt.device_buffers(work)
    return [(images, out, status)] + [
        (images.clone(), torch.empty_like(out), torch.zeros_like(status)) for _ in range(n - 1)]


@pytest.mark.parametrize("which", ["nested", "hetero", "sweep"])
def test_graph_replays_equal_the_oracle(rt, which):
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    if which == "nested":
        work, slab = wl.nested(teams=300, threads=256, depth=3, elems_per_team=512), 3264
    elif which == "hetero":
        work, slab = wl.hetero(n_instances=12, max_teams=40, max_frame=16384, seed=31), 8192
    else:
        work, slab = wl.sweep(8192, teams=200), 8192
    rt.configure(slab, 3 * 32768, 4096)
    sets = _sets(rt, work, 3)
    # every region of the workload on every set, in turn: launch i runs
    # region i mod R on set (i // R) mod 3
    regions, bufs = [], []
    for s in range(3):
        for r in work.regions:
            regions.append(r)
            bufs.append(sets[s])
    g = dsr.dsr_graph_capture_regions(rt.ctx, regions, bufs)
    try:
        for _ in range(2):
            for _, o, st in sets:   # outputs the replay must write again (padding
                o.zero_()            # between instances stays zero, as in the oracle)
                st.zero_()
            dsr.dsr_graph_launch(rt.ctx, g)
            torch.cuda.synchronize()
            r, rs = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=3 * 32768)
            for _, o, st in sets:
                go = o.cpu().numpy()
                gs = st.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
                if work.out_dtype == "float32":
                    s32 = oracle.sweep_fields(r)[2]   # the oracle's fp32 sums, bit for bit
                    assert np.array_equal(go[: s32.size].view(np.uint32), s32.view(np.uint32))
                else:
                    assert np.array_equal(go[: r.size], r)
                for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
                    assert np.array_equal(gs[f], rs[f]), f
    finally:
        dsr.dsr_graph_destroy(g)


def test_graph_capture_refuses_and_replays_check_the_stack(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.nested(teams=16, threads=256, depth=3, elems_per_team=256)
    rt.configure(3264, 0, 0)
    images, out, status = rt.device_buffers(work)
    region = work.regions[0]
    # the third launch's outputs are too small: nothing is captured
    short = out[:16]
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_graph_capture_regions(rt.ctx, [region] * 3,
                                      [(images, out, status)] * 2 + [(images, short, status)])
    assert "launch 2" in str(ei.value)
    g = dsr.dsr_graph_capture_regions(rt.ctx, [region] * 2, [(images, out, status)] * 2)
    try:
        dsr.dsr_graph_launch(rt.ctx, g)
        rt.torch.cuda.synchronize()
        r, _ = oracle.run_workload(work, slab_bytes=3264)
        assert np.array_equal(out.cpu().numpy()[: r.size], r)
        rt.configure(3264, 0, 0)      # a new stack configuration
        with pytest.raises(dsr.DsrError) as ei:
            dsr.dsr_graph_launch(rt.ctx, g)
        assert "stack configuration" in str(ei.value)
        other = dsr.Runtime(0, slab_bytes=3264)
        try:
            with pytest.raises(dsr.DsrError):
                dsr.dsr_graph_launch(other.ctx, g)
        finally:
            other.close()
    finally:
        dsr.dsr_graph_destroy(g)


def test_graph_headline_full_size_on_rotating_sets(rt):
    """The headline at full size (1024 teams x 256 threads, depth 3, 4096
    elements per team) in the configuration bench.py times: a launch graph
    of launches over rotating buffer sets, back to back, at most
    ceil(1024 / SMs) teams per SM. Every set's output and team records equal
    the oracle's."""
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    work = wl.nested(teams=1024, threads=256, depth=3, elems_per_team=4096)
    rt.configure(3264, 0, 0)
    sets = _sets(rt, work, 4)
    order = [i % 4 for i in range(10)]
    g = dsr.dsr_graph_capture_regions(rt.ctx, work.regions * len(order), [sets[i] for i in order])
    try:
        dsr.dsr_graph_launch(rt.ctx, g)
        dsr.dsr_graph_launch(rt.ctx, g)
        torch.cuda.synchronize()
    finally:
        dsr.dsr_graph_destroy(g)
    occ = rt.occupancy(work.regions[0])
    assert occ["ctas_per_sm"] == -(-1024 // occ["sm_count"])
    r, rs = oracle.run_workload(work, slab_bytes=3264)
    for _, o, st in sets:
        assert np.array_equal(o.cpu().numpy(), r)
        gs = st.cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
        for f in ("status", "depth_final", "hwm_bytes", "spill_bytes", "chk"):
            assert np.array_equal(gs[f], rs[f]), f
