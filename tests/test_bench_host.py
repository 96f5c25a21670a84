"""Host-side logic of bench.py that runs without a GPU: the oracle timing
behind `cpu_baseline` (and the reference arm) on one and several threads."""
import numpy as np

import bench
import oracle
import workloads as wl


def test_threaded_oracle_timing_covers_disjoint_team_slices(monkeypatch):
    """Each thread runs only its own contiguous slice of teams, the slices
    cover every team, and the teams counted are the teams run."""
    work = wl.nested(teams=40, threads=256, depth=3)
    calls = []
    real = oracle.run_region

    def spy(region, images, out, status, slab, ovf, b, e):
        calls.append((b, e))
        return real(region, images, out, status, slab, ovf, b, e)

    monkeypatch.setattr(oracle, "run_region", spy)
    line = bench.time_oracle(work, 3264, 0, budget_s=0.3, threads=3)
    assert line["cores"] == 3 and line["kind"] == "oracle" and line["value"] > 0
    slices = [(0, 13), (13, 26), (26, 40)]
    covered = np.zeros(40, dtype=bool)
    for b, e in calls:
        assert b < e and any(lo <= b and e <= hi for lo, hi in slices), (b, e)
        covered[b:e] = True
    assert covered.all()
    teams = sum(e - b for b, e in calls)
    assert "%d teams" % teams in line["sample"]


def test_cpu_baseline_reports_both_thread_counts(monkeypatch):
    work = wl.nested(teams=16, threads=256, depth=3)
    monkeypatch.setattr(bench, "host_cores", lambda: 2)
    line = bench.cpu_baseline(work, 3264, 0, budget_s=0.4)
    assert line["cores"] == 2 and line["single_thread"]["value"] > 0
    assert line["cpu"] == bench.cpu_model() and line["cpu"]


def test_more_threads_than_teams_is_capped():
    work = wl.nested(teams=2, threads=256, depth=3)
    line = bench.time_oracle(work, 3264, 0, budget_s=0.1, threads=8)
    assert line["cores"] == 2


def test_bench_rank_shares_partition_the_work():
    """bench.py's per-rank shares under torchrun: the batched form's instance
    ranges and the served form's routed requests each cover the work once."""
    for world in (1, 2, 4):
        parts = [bench.batch_share(1000, r, world) for r in range(world)]
        allb = np.concatenate(parts)
        assert np.array_equal(allb, np.arange(1000))
        teams = np.tile(wl.hetero_shapes(300)[0], 3)
        reqs = [bench.served_share(teams, r, world) for r in range(world)]
        alls = np.sort(np.concatenate(reqs))
        assert np.array_equal(alls, np.arange(len(teams)))
        loads = [int(teams[q].sum()) for q in reqs]
        assert max(loads) - min(loads) <= int(teams.max())


def _pool_rank_main(rank, world, port, path):
    import os

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        teams = np.tile(wl.hetero_shapes(200)[0], 2)
        mine = bench.served_share(teams, rank, world)
        pooled = bench._pool_latencies(mine.astype(np.int64), dist)
        if rank == 0:
            ok = np.array_equal(np.sort(pooled), np.arange(len(teams)))
            with open(path, "w") as f:
                f.write("ok" if ok else "mismatch")
        else:
            assert pooled is None
    finally:
        dist.destroy_process_group()


def test_served_latencies_pool_on_rank0_over_two_gloo_ranks(tmp_path):
    """Each rank's request latencies reach rank 0, where the job's
    percentiles are taken (two gloo ranks on the CPU)."""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    path = str(tmp_path / "pool.txt")
    mp.spawn(_pool_rank_main, args=(2, port, path), nprocs=2, join=True)
    assert open(path).read() == "ok"


def test_reference_arm_config_is_the_gpu_arms():
    """Both arms print the same config dict for the same workload."""
    work, slab, ovf, algo_bytes, cfg = bench.make_workload("nested")
    a = bench.bench_config(cfg, work, 1)
    assert a["l2"].startswith("inputs larger than L2: 15 rotating sets")
    assert set(a) >= {"workload", "parallelism", "l2"}
