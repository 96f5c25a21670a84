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
