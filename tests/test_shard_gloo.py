"""The multi-GPU path's host logic on the CPU: two gloo ranks split a set of
heterogeneous region instances by instance, each runs its share, and rank
0 gathers the per-instance results, which must equal one run of the whole
set. Each rank runs its share through the CPU oracle here (no GPU in this
test); what is under test is the split, the gather and the cross-rank
reductions that bench.py uses under torchrun."""
import os
import socket

import numpy as np
import pytest

import workloads as wl
from paper_1711_10413_gb300 import shard

N_INST, MAX_TEAMS, MAX_FRAME = 24, 6, 1024
SLAB, OVF = 2048, 4096


def _instance_results(work, out, status, ids):
    """Per-instance (output words, team statuses) keyed by global index."""
    res = {}
    for r, gi in zip(work.regions, ids):
        n = r.teams * r.team_width
        o = out[r.out_offset // 4: r.out_offset // 4 + n].copy()
        s = status[r.status_index: r.status_index + r.teams].copy()
        res[int(gi)] = np.concatenate([o.view(np.uint8), s.view(np.uint8)])
    return res


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        teams = wl.hetero_shapes(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME)[0]
        a, b = shard.balanced_ranges(teams, world)[rank]
        ids = np.arange(a, b)
        work = wl.hetero(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME, instances=ids)
        out, status = oracle.run_workload(work, SLAB, OVF)
        merged = shard.gather_to_rank0(_instance_results(work, out, status, ids), dist)
        slowest = shard.max_over_ranks(1.5 + rank, dist)
        units = shard.sum_over_ranks(float(len(ids)), dist)
        dist.barrier()
        if rank == 0:
            full = wl.hetero(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME)
            fo, fs = oracle.run_workload(full, SLAB, OVF)
            want = _instance_results(full, fo, fs, np.arange(N_INST))
            ok = (sorted(merged) == list(range(N_INST))
                  and all(np.array_equal(merged[i], want[i]) for i in range(N_INST))
                  and slowest == 0.5 + world and units == N_INST)
            with open(result_path, "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_split_gather_equals_whole(tmp_path):
    import torch.multiprocessing as mp
    path = str(tmp_path / "result.txt")
    mp.spawn(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True)
    assert open(path).read() == "ok"


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_balanced_ranges_partition(world):
    teams = wl.hetero_shapes(500)[0]
    rs = shard.balanced_ranges(teams, world)
    assert len(rs) == world and rs[0][0] == 0 and rs[-1][1] == 500
    for (a, b), (c, d) in zip(rs, rs[1:]):
        assert b == c and a <= b
    loads = [int(teams[a:b].sum()) for a, b in rs]
    assert max(loads) - min(loads) <= 2 * int(teams.max())


def test_balanced_ranges_edge_cases():
    assert shard.balanced_ranges([], 3) == [(0, 0)] * 3
    assert shard.balanced_ranges([0, 0, 0, 0], 2) == [(0, 2), (2, 4)]
    # one instance goes to the rank its weight's midpoint falls in
    assert shard.balanced_ranges([5], 3) == [(0, 0), (0, 1), (1, 1)]
    with pytest.raises(ValueError):
        shard.balanced_ranges([1, 2], 0)
    assert shard.max_over_ranks(3.0) == 3.0 and shard.sum_over_ranks(2.0) == 2.0


def _serve_rank_main(rank, world, port, result_path):
    """Each rank serves the requests routed to it (through the oracle here);
    rank 0 gathers every request's result, which must equal one run of all
    the requests."""
    import torch.distributed as dist

    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        teams = wl.hetero_shapes(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME)[0]
        routed = shard.route_requests(teams, world)
        ids = np.nonzero(routed == rank)[0]
        work = wl.hetero(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME, instances=ids)
        out, status = oracle.run_workload(work, SLAB, OVF)
        merged = shard.gather_to_rank0(_instance_results(work, out, status, ids), dist)
        if rank == 0:
            full = wl.hetero(N_INST, max_teams=MAX_TEAMS, max_frame=MAX_FRAME)
            fo, fs = oracle.run_workload(full, SLAB, OVF)
            want = _instance_results(full, fo, fs, np.arange(N_INST))
            ok = (sorted(merged) == list(range(N_INST))
                  and all(np.array_equal(merged[i], want[i]) for i in range(N_INST)))
            with open(result_path, "w") as f:
                f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_two_rank_routed_requests_equal_whole(tmp_path):
    import torch.multiprocessing as mp
    path = str(tmp_path / "served.txt")
    mp.spawn(_serve_rank_main, args=(2, _free_port(), path), nprocs=2, join=True)
    assert open(path).read() == "ok"


@pytest.mark.parametrize("world", [1, 2, 4])
def test_route_requests_balances_load(world):
    teams = wl.hetero_shapes(1000)[0]
    rank = shard.route_requests(teams, world)
    assert rank.min() >= 0 and rank.max() < world and len(rank) == 1000
    loads = [int(teams[rank == r].sum()) for r in range(world)]
    # greedy least-loaded: no rank ends more than one request above another
    assert max(loads) - min(loads) <= int(teams.max())
    assert (shard.route_requests(teams, world) == rank).all()  # the same on every rank
