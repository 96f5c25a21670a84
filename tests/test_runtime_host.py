"""Host logic of the Python runtime wrapper that needs no GPU: the
autotuner cache (keyed by device and batch shape class)."""
import json

import paper_1711_10413_gb300 as dsr
import workloads as wl
from paper_1711_10413_gb300.runtime import Runtime, batch_class


def _batch(**kw):
    return dict(descs=dsr.pack_descs(wl.hetero(**kw).regions))


def test_batch_class_groups_one_distribution():
    same = {batch_class(_batch(n_instances=1000, seed=s)["descs"]) for s in range(1, 6)}
    assert len(same) == 1
    other = [batch_class(_batch(n_instances=1000, max_teams=8, seed=1)["descs"]),
             batch_class(_batch(n_instances=8000, seed=1)["descs"]),
             batch_class(dsr.pack_descs(wl.nested(teams=300).regions))]
    assert len(set(other) | same) == 4


def test_autotune_cache_round_trip(tmp_path):
    rt = object.__new__(Runtime)  # no context: the tuner is replaced below
    calls = []

    def tuner(b, stream=None):
        calls.append(len(b["descs"]))
        return dict(threads=96, slab_bytes=8192, ctas_per_sm=0), 1.5

    rt.autotune = tuner
    path = str(tmp_path / "tuning.json")
    t, ms, hit = rt.autotune_cached(_batch(n_instances=500, seed=1), path, device_key="gpu-a")
    assert not hit and len(calls) == 1 and ms == 1.5
    # another batch of the same distribution on the same device: from the file
    t2, ms2, hit2 = rt.autotune_cached(_batch(n_instances=500, seed=2), path, device_key="gpu-a")
    assert hit2 and t2 == t and ms2 == 1.5 and len(calls) == 1
    # another device, and another shape class: the tuner runs
    assert not rt.autotune_cached(_batch(n_instances=500, seed=1), path, device_key="gpu-b")[2]
    assert not rt.autotune_cached(_batch(n_instances=500, max_teams=8), path,
                                  device_key="gpu-a")[2]
    assert len(calls) == 3 and len(json.load(open(path))) == 3
    # an unreadable file counts as empty and is written again
    open(path, "w").write("{not json")
    assert not rt.autotune_cached(_batch(n_instances=500, seed=1), path, device_key="gpu-a")[2]
    assert len(json.load(open(path))) == 1
