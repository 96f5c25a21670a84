"""The batched launch that allocates nothing.

Some callers cannot allocate device memory: a code path where cudaMalloc
and cudaFree are off limits because they can synchronise the whole device,
or a plug-in whose host application owns every device byte through its own
allocator. For them the library runs a batch with its workspace in a fixed
device array it carries itself. This file checks, through the C ABI, that
such a run gives exactly what the ordinary batched launch (with a
caller-allocated workspace) gives, on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next result),
and that a batch too large for the array is refused before anything runs.
It is collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

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


def _static(rt, b, tuning, total=None):
    import paper_1711_10413_gb300 as dsr
    dsr.dsr_launch_batch_static(rt.ctx, b["descs_dev"], len(b["descs"]), b["program"],
                                b["total"] if total is None else total, b["images"], b["out"],
                                b["status"], tuning)


@pytest.mark.parametrize("threads,slab", [(128, 8192), (256, 16384), (1024, 4096)])
def test_static_batch_matches_allocated_batch(rt, threads, slab):
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    work = wl.hetero(n_instances=2000)
    b = rt.batch_buffers(work)
    assert dsr.dsr_batch_workspace_bytes(len(b["descs"]), b["total"]) <= \
        dsr.dsr_batch_static_capacity()
    tuning = dict(threads=threads, slab_bytes=slab)
    rt.launch_batch(b, tuning)
    torch.cuda.synchronize()
    ref_out, ref_status = b["out"].clone(), b["status"].clone()
    assert rt.batch_errors(b)[0] == 0
    for _ in range(2):
        b["out"].zero_()
        b["status"].zero_()
        torch.cuda.synchronize()
        _static(rt, b, tuning)
        torch.cuda.synchronize()
        assert torch.equal(b["out"], ref_out)          # integer outputs: bit for bit
        assert torch.equal(b["status"], ref_status)
        assert dsr.dsr_batch_static_errors(rt.ctx) == (0, b["total"])
    st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    assert (st["status"] == 0).all() and (st["depth_final"] == 0).all()


def test_static_batch_accumulating_program(rt):
    """The paper's scalars program adds into its output (a += sum c_i): run
    twice in a row on the same output, each static call must add exactly
    once, as the allocated-workspace launch and the oracle do; leftover
    workspace state from the first call would show as a wrong count."""
    import oracle
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    work = wl.paper_scalars(7, teams=40, threads=128)
    b = rt.batch_buffers(work)
    tuning = dict(threads=128, slab_bytes=4096)
    r, _ = oracle.run_workload(work)
    a0 = b["out"].clone()
    for k in (1, 2):
        _static(rt, b, tuning)
        torch.cuda.synchronize()
        # after k runs every slot holds a0 + k * 28
        expect = (a0.cpu().numpy().astype(np.int64) + k * 28 + 2 ** 31) % 2 ** 32 - 2 ** 31
        assert np.array_equal(b["out"].cpu().numpy().astype(np.int64), expect)
        if k == 1:
            assert np.array_equal(b["out"].cpu().numpy()[: r.size], r)
    b2 = rt.batch_buffers(work)
    rt.launch_batch(b2, tuning)
    rt.launch_batch(b2, tuning)
    torch.cuda.synchronize()
    assert torch.equal(b["out"], b2["out"])


def test_static_batch_reports_undercounted_teams(rt):
    """total_teams below the instances' team sum: the teams with no task slot
    do not run, report INVALID in their statuses, and are counted in the
    errors dsr_batch_static_errors reads back."""
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    work = wl.hetero(n_instances=50, max_teams=16, max_frame=2048, seed=4)
    b = rt.batch_buffers(work)
    short = 7
    b["status"].fill_(-1)
    torch.cuda.synchronize()
    _static(rt, b, dict(threads=128, slab_bytes=8192), total=b["total"] - short)
    torch.cuda.synchronize()
    errors, counted = dsr.dsr_batch_static_errors(rt.ctx)
    assert counted == b["total"] and errors == short
    st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    assert (st["status"] == 1).sum() == short
    assert (st["status"] == 0).sum() == b["total"] - short
    assert not (st["status"] == -1).any()   # every team's status was written


def test_static_batch_refuses_another_current_device(rt):
    """A ctx used while another device is current is refused before anything
    runs (its pool and workspace address belong to its own device)."""
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    work = wl.hetero(n_instances=5, max_teams=4)
    b = rt.batch_buffers(work)
    with torch.cuda.device(1):
        with pytest.raises(dsr.DsrError) as ei:
            _static(rt, b, dict(threads=128, slab_bytes=8192))
    assert ei.value.code == dsr.DSR_ERR_INVALID and "current device" in str(ei.value)


def test_static_batch_refuses_oversized_batch(rt):
    import paper_1711_10413_gb300 as dsr
    work = wl.hetero(n_instances=20, max_teams=4)
    b = rt.batch_buffers(work)
    too_many = dsr.dsr_batch_static_capacity() // 8 + 1
    with pytest.raises(dsr.DsrError) as ei:
        dsr.dsr_launch_batch_static(rt.ctx, b["descs_dev"], len(b["descs"]), b["program"],
                                    too_many, b["images"], b["out"], b["status"])
    assert ei.value.code == dsr.DSR_ERR_BUDGET
    assert "static workspace" in str(ei.value)
    assert not np.any(b["out"].cpu().numpy())
