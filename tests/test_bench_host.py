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
