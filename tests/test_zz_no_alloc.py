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


def test_static_batch_matches_allocated_batch(rt):
    import paper_1711_10413_gb300 as dsr
    torch = rt.torch
    work = wl.hetero(n_instances=2000)
    b = rt.batch_buffers(work)
    assert dsr.dsr_batch_workspace_bytes(len(b["descs"]), b["total"]) <= \
        dsr.dsr_batch_static_capacity()
    tuning = dict(threads=128, slab_bytes=8192)
    rt.launch_batch(b, tuning)
    torch.cuda.synchronize()
    ref_out, ref_status = b["out"].clone(), b["status"].clone()
    assert rt.batch_errors(b)[0] == 0
    for _ in range(2):
        b["out"].zero_()
        b["status"].zero_()
        torch.cuda.synchronize()
        dsr.dsr_launch_batch_static(rt.ctx, b["descs_dev"], len(b["descs"]), b["program"],
                                    b["total"], b["images"], b["out"], b["status"], tuning)
        torch.cuda.synchronize()
        assert torch.equal(b["out"], ref_out)          # integer outputs: bit for bit
        assert torch.equal(b["status"], ref_status)
    st = b["status"].cpu().numpy().view(dsr.TEAM_STATUS_DTYPE)
    assert (st["status"] == 0).all() and (st["depth_final"] == 0).all()


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
