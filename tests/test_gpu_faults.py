"""Failure handling on the GPU without faulting it: a device wait that
nothing completes gives up after its limit and reports DSR_ERR_TIMEOUT, and
the context stays usable afterwards."""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def test_wait_that_nothing_completes_times_out():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    rt = dsr.Runtime(0, slab_bytes=3264)
    try:
        res = torch.zeros(2, dtype=torch.int64, device="cuda")
        for limit in (200_000, 5_000_000):  # 0.2 ms and 5 ms of %globaltimer
            res.zero_()
            dsr.dsr_check_bounded_wait(rt.ctx, limit, res)
            torch.cuda.synchronize()
            status, elapsed = (int(x) for x in res.cpu())
            assert status == dsr.DSR_ERR_TIMEOUT
            # it gave up after the limit, and not long after
            assert limit <= elapsed < limit + 100_000_000, (limit, elapsed)
        # the context is still usable: a region runs and matches the oracle
        work = wl.nested(teams=8, threads=256, depth=3)
        rt.configure(3264, 0, 0)
        g, gs = rt.run_workload(work)
        r, rs = oracle.run_workload(work, slab_bytes=3264)
        assert np.array_equal(g, r) and (gs["status"] == 0).all()
        with pytest.raises(dsr.DsrError) as ei:
            dsr.dsr_check_bounded_wait(rt.ctx, 11_000_000_000, res)
        assert ei.value.code == dsr.DSR_ERR_INVALID
    finally:
        rt.close()


def test_stack_misuse_reports_lifo_and_overflow():
    """The device's push and pop misused on purpose (a 96-byte slab, a
    64-byte overflow slab): a pop of a frame that is not the top, a push that
    fits neither slab, a pop with the wrong size and a full frame table each
    give their status and change nothing else. The placements, the LIFO and
    OVERFLOW outcomes and the peaks agree with the oracle's stack."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1711_10413_gb300 as dsr
    rt = dsr.Runtime(0, slab_bytes=3264)
    try:
        res = torch.full((25,), -1, dtype=torch.int64, device="cuda")
        scratch = torch.zeros(64, dtype=torch.uint8, device="cuda")
        dsr.dsr_check_stack(rt.ctx, res, scratch)
        torch.cuda.synchronize()
        r = res.cpu().numpy().tolist()
    finally:
        rt.close()
    OK, OVF, LIFO = dsr.DSR_OK, dsr.DSR_ERR_OVERFLOW, dsr.DSR_ERR_LIFO
    assert r == [1, 1, 1, 96, 64,           # pushes of 48, 40 (slab) and 64 (overflow)
                 LIFO, 3, 96, 64,           # pop of the second frame: refused
                 OK, OK, OK, 0, 0, 0,       # the pops in order empty the stack
                 LIFO, 160, 64,             # first error kept; peaks
                 OVF, 1, 3,                 # a fourth push fits neither slab
                 LIFO,                      # the top frame popped with a wrong size
                 8, OVF, 8]                 # the frame table holds 8 frames
    # the same script on the oracle's stack
    s = oracle.Stack(96, 64)
    (a, sa), (b, sb), (c, sc) = s.push(48), s.push(40), s.push(64)
    assert (sa, sb, sc) == (True, True, False)
    st = s.state()
    assert (st["slab_used"], st["overflow_used"]) == (r[3], r[4])
    assert s.pop(b) == r[5] and s.state()["depth"] == r[6]
    assert [s.pop(i) for i in (c, b, a)] == r[9:12]
    st = s.state()
    assert (st["depth"], st["slab_used"], st["overflow_used"], st["hwm"], st["spill_hwm"]) == \
        (r[12], r[13], r[14], r[16], r[17])
    s2 = oracle.Stack(96, 64)
    for n in (48, 48, 64):
        assert s2.push(n)[0] >= 0
    assert s2.push(16)[0] == -1 and s2.state()["status"] == r[18]
