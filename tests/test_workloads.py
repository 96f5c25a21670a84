"""The seeded workload generator: determinism and the stated distributions."""
import numpy as np

import workloads as wl


def test_splitmix64_reference_outputs():
    # SplitMix64 from state 0: the first outputs as published with the
    # generator (Steele, Lea, Flood 2014; the reference C implementation)
    out = wl.splitmix64_outputs(0, 2)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_deterministic():
    a = wl.nested(teams=4, threads=256, depth=3)
    b = wl.nested(teams=4, threads=256, depth=3)
    assert np.array_equal(a.images, b.images)
    c = wl.nested(teams=4, threads=256, depth=3, seed=5)
    assert not np.array_equal(a.images, c.images)


def test_scalars_range():
    w = wl.scalars(n_regions=1000)
    v = w.images.view(np.uint32)
    assert v.max() < (1 << 20) and v.size == 4000
    assert abs(v.mean() / (1 << 19) - 1) < 0.02


def test_sweep_normal():
    w = wl.sweep(196608, teams=8)
    x = w.images.view(np.float32).astype(np.float64)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01


def test_hetero_distribution():
    teams, threads, depth, fb, salt = wl.hetero_shapes(10000)
    assert teams.min() >= 1 and teams.max() <= 512
    assert 70 < teams.mean() < 95          # log-uniform on [1, 512]: ~82
    assert set(np.unique(threads)) == set(range(32, 1025, 32))
    assert set(np.unique(depth)) == {1, 2, 3}
    assert fb.min() >= 16 and fb.max() <= 32768 and (fb % 4 == 0).all()
    assert 3800 < fb.mean() < 4800         # log-uniform on [16, 32768]: ~4.3 KB


def test_hetero_layout():
    w = wl.hetero(n_instances=50, max_teams=8)
    img_end = 0
    for r in w.regions:
        assert r.image_offset % 16 == 0 and r.out_offset % 16 == 0
        img_end = r.image_offset + sum((b + 15) // 16 * 16 for b in r.frame_bytes)
    assert img_end == w.images.size
    assert w.n_status == sum(r.teams for r in w.regions)
    sub = wl.hetero(n_instances=50, max_teams=8, instances=[3, 7])
    assert [r.teams for r in sub.regions] == [w.regions[3].teams, w.regions[7].teams]


def test_poisson_rate():
    t = wl.poisson_arrivals(100000, 200000.0)
    rate = 100000 / (t[-1] * 1e-9)
    assert abs(rate / 200000.0 - 1) < 0.02
