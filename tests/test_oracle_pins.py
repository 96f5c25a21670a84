"""Pins of the CPU oracle against facts fixed outside the oracle itself.

* mix32 against MurmurHash3_x86_32's published test vectors and SMHasher's
  verification value (tests/golden/murmur3_x86_32.txt).
* The paper's two evaluation programs (Sec. 6.1) against their closed forms.
* The scalars body against hand-evaluated values (tests/golden).
* The FP32 sweep against exactly rounded sums, closed-form counts, and
  hand-derived worked examples of its fp32 index-order sum.
* The nested / hetero programs against invariants that any correct
  implementation satisfies (stack depth back to 0, high-water marks, the
  structure that mix32 being a bijection exposes, placement independence).
* The worker-level program against its structure (s2 XORs every output,
  the key follows the worker number across warps, a shared base image) and
  its per-warp stack accounting.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl

M32 = 0xFFFFFFFF


# ---------------------------------------------------------------------------
# mix32 = MurmurHash3 fmix32
# ---------------------------------------------------------------------------
def _rotl(x, r):
    return ((x << r) | (x >> (32 - r))) & M32


def _murmur3_x86_32(data: bytes, seed: int) -> int:
    """MurmurHash3_x86_32 body mixing, finalised with the oracle's mix32."""
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed & M32
    nblocks = len(data) // 4
    for i in range(nblocks):
        k = int.from_bytes(data[4 * i: 4 * i + 4], "little")
        k = (_rotl((k * c1) & M32, 15) * c2) & M32
        h = (_rotl(h ^ k, 13) * 5 + 0xE6546B64) & M32
    tail = data[4 * nblocks:]
    k = 0
    if len(tail) >= 3:
        k ^= tail[2] << 16
    if len(tail) >= 2:
        k ^= tail[1] << 8
    if len(tail) >= 1:
        k ^= tail[0]
        k = (_rotl((k * c1) & M32, 15) * c2) & M32
        h ^= k
    return oracle.mix32(h ^ len(data))


def _golden_lines(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line.split()


def test_mix32_published_vectors(golden_dir):
    n = 0
    for parts in _golden_lines(golden_dir, "murmur3_x86_32.txt"):
        if parts[0] == "verification":
            key = bytearray(256)
            hashes = bytearray()
            for i in range(256):
                key[i] = i
                hashes += _murmur3_x86_32(bytes(key[:i]), 256 - i).to_bytes(4, "little")
            assert _murmur3_x86_32(bytes(hashes), 0) == int(parts[1], 16)
        else:
            data = b"" if parts[0] == "-" else bytes.fromhex(parts[0])
            assert _murmur3_x86_32(data, int(parts[1], 16)) == int(parts[2], 16), parts
        n += 1
    assert n == 8


def _inv_mix32(h):
    """Inverse of fmix32, derived from its definition (xor-shifts and odd
    multipliers are invertible modulo 2^32)."""
    h ^= h >> 16
    h = (h * pow(0xC2B2AE35, -1, 1 << 32)) & M32
    h ^= (h >> 13) ^ (h >> 26)
    h = (h * pow(0x85EBCA6B, -1, 1 << 32)) & M32
    h ^= h >> 16
    return h


def test_mix32_is_a_bijection():
    rng = np.random.default_rng(5)
    for x in [0, 1, 2, M32, 0x80000000] + [int(v) for v in rng.integers(0, 1 << 32, 200)]:
        assert _inv_mix32(oracle.mix32(x)) == x


# ---------------------------------------------------------------------------
# The paper's programs (Sec. 6.1): closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_vars", [1, 2, 7, 8, 16, 20, 21, 64])
@pytest.mark.parametrize("threads", [32, 128, 256])
def test_paper_scalars_closed_form(n_vars, threads):
    w = wl.paper_scalars(n_vars=n_vars, teams=3, threads=threads)
    out, st = oracle.run_workload(w)
    expect = (w.out_init.astype(np.int64) + n_vars * (n_vars + 1) // 2) & M32
    assert np.array_equal(out.view(np.uint32).astype(np.int64), expect)
    assert (st["status"] == 0).all() and (st["depth_final"] == 0).all()
    fb = w.regions[0].frame_bytes[0]
    assert (st["hwm_bytes"] == (fb + 15) // 16 * 16).all()


@pytest.mark.parametrize("n_arrays", [1, 2, 3, 4])
def test_paper_arrays_closed_form(n_arrays):
    w = wl.paper_arrays(n_arrays=n_arrays, teams=5, threads=128)
    out, st = oracle.run_workload(w)
    expect = (w.out_init.astype(np.int64) + 10 * n_arrays) & M32
    assert np.array_equal(out.view(np.uint32).astype(np.int64), expect)
    # an int[96] array is 384 bytes, the "array data shared" column of
    # Tables 5 and 6
    assert w.regions[0].frame_bytes[0] == 384 * n_arrays
    assert (st["hwm_bytes"] == 384 * n_arrays).all()


# ---------------------------------------------------------------------------
# Scalars body: hand-evaluated values
# ---------------------------------------------------------------------------
def test_scalars_worked_values(golden_dir):
    rows = [list(map(int, p)) for p in _golden_lines(golden_dir, "scalars_worked.txt")]
    frames = sorted({tuple(r[:4]) for r in rows})
    images = np.array(frames, dtype=np.uint32).reshape(-1)
    region = wl.Region(wl.PROG_SCALARS, 1, 128, 1, [16], param=len(frames))
    work = wl.Workload("t", [region], images.view(np.uint8), 4 * 96 * len(frames), 1)
    out, st = oracle.run_workload(work)
    out = out.view(np.uint32).reshape(len(frames), 96)
    for s0, s1, s2, s3, tid, expect in rows:
        assert out[frames.index((s0, s1, s2, s3)), tid] == expect, (s0, s1, s2, s3, tid)
    assert st["status"][0] == 0 and st["depth_final"][0] == 0 and st["hwm_bytes"][0] == 16


def test_scalars_regions_are_sequential_and_independent():
    """Region r reads only image r: changing one frame changes one row."""
    w = wl.scalars(n_regions=50)
    out1, _ = oracle.run_workload(w)
    imgs = w.images.view(np.uint32).copy()
    imgs[4 * 17 + 1] ^= 0x5A5A
    w2 = wl.Workload("t", w.regions, imgs.view(np.uint8), w.out_bytes, w.n_status)
    out2, _ = oracle.run_workload(w2)
    diff = (out1 != out2).reshape(50, 96).any(axis=1)
    assert diff.tolist() == [r == 17 for r in range(50)]


# ---------------------------------------------------------------------------
# FP32 sweep: exact sums and closed-form counts
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("frame_bytes", [64, 1024, 8192, 4 * 1000])
def test_sweep_all_ones_counts(frame_bytes):
    teams, threads = 3, 128
    L = frame_bytes // 4
    images = np.ones(teams * L, dtype=np.float32)
    region = wl.Region(wl.PROG_SWEEP, teams, threads, 1, [frame_bytes])
    work = wl.Workload("t", [region], images.view(np.uint8), 4 * teams * 96, teams,
                       out_dtype="float32")
    out, st = oracle.run_workload(work)
    s64, _, s32 = oracle.sweep_fields(out)
    sums, sums32 = s64.reshape(teams, 96), s32.reshape(teams, 96)
    for tid in range(96):
        # elements tid, tid + 96, ... below L
        count = 0 if tid >= L else (L - tid + 95) // 96
        assert (sums[:, tid] == count).all()
        assert (sums32[:, tid] == np.float32(count)).all()
    assert (st["hwm_bytes"] == (frame_bytes + 15) // 16 * 16).all()


def _gamma(n):
    """gamma_n = n u / (1 - n u), u = 2^-24: the a-priori bound of recursive
    fp32 summation of n + 1 terms is gamma_n times the sum of magnitudes."""
    return n * U32 / (1 - n * U32)


U32 = 2.0 ** -24


@pytest.mark.parametrize("frame_bytes", [64, 1024, 32768])
def test_sweep_matches_exact_sum(frame_bytes):
    w = wl.sweep(frame_bytes, teams=4)
    out, _ = oracle.run_workload(w)
    s64, m64, s32 = oracle.sweep_fields(out)
    sums, mags, sums32 = s64.reshape(4, 96), m64.reshape(4, 96), s32.reshape(4, 96)
    x = w.images.view(np.float32).reshape(4, frame_bytes // 4).astype(np.float64)
    for t in range(4):
        for tid in range(96):
            part = x[t, tid::96].tolist()
            exact = math.fsum(part)
            mag = math.fsum(abs(v) for v in part)
            bound = len(part) * 2.0 ** -53 * mag
            assert abs(sums[t, tid] - exact) <= bound
            assert abs(mags[t, tid] - mag) <= bound
            # the fp32 sum within the recursive-summation bound of the exact sum
            assert abs(float(sums32[t, tid]) - exact) <= _gamma(max(len(part) - 1, 0)) * mag


def _one_worker_sweep(values):
    """One team of 64 threads (32 workers) whose worker 0 sums `values`
    (elements 0, 32, 64, ...); the other slots hold zeros."""
    L = 32 * len(values)
    x = np.zeros(L, dtype=np.float32)
    x[0::32] = np.asarray(values, dtype=np.float32)
    region = wl.Region(wl.PROG_SWEEP, 1, 64, 1, [4 * L])
    work = wl.Workload("t", [region], x.view(np.uint8), 4 * 32, 1, out_dtype="float32")
    out, _ = oracle.run_workload(work)
    s64, _, s32 = oracle.sweep_fields(out)
    return float(s64[0]), s32[0]


def test_sweep_fp32_order_and_rounding_worked_example():
    """Worked example with hand-derived results. 1 + 2^-24 is a tie between 1
    and 1 + 2^-23 and rounds to even (1), so in index order each small term
    vanishes: [1, 2^-24, 2^-24, 2^-24] sums to exactly 1 in fp32. Taken the
    other way round the small terms first add to 3 * 2^-24 exactly, and
    1 + 3 * 2^-24 (1.5 ulp above 1) rounds to even, 1 + 2^-22. The fp64 sum
    is exact, 1 + 3 * 2^-24. A sum in another order, in a wider type, or
    with a fused step gives one of the other values."""
    e = 2.0 ** -24
    s64, s32 = _one_worker_sweep([1.0, e, e, e])
    assert s32 == np.float32(1.0)
    assert s64 == 1.0 + 3 * e
    s64, s32 = _one_worker_sweep([e, e, e, 1.0])
    assert s32 == np.float32(1.0 + 2.0 ** -22)
    assert s64 == 1.0 + 3 * e


def test_sweep_fp32_cancellation_worked_example():
    """Catastrophic cancellation by hand: in fp32, 2^24 + 1 rounds to 2^24
    (a tie, to even), so [2^24, 1, -2^24] sums to 0 while the exact (fp64)
    sum is 1; [2^24, -2^24, 1] sums to 1 in both."""
    s64, s32 = _one_worker_sweep([2.0 ** 24, 1.0, -(2.0 ** 24)])
    assert s32 == np.float32(0.0) and s64 == 1.0
    s64, s32 = _one_worker_sweep([2.0 ** 24, -(2.0 ** 24), 1.0])
    assert s32 == np.float32(1.0) and s64 == 1.0


def test_sweep_fp32_equals_numpy_left_to_right():
    """The oracle's fp32 sums against numpy's fp32 running sum in index order
    (np.add.accumulate over rows of W elements), an implementation of its
    own, on a ragged frame (L not a multiple of the width)."""
    w = wl.sweep(4 * 1001, teams=3, threads=160)
    out, _ = oracle.run_workload(w)
    _, _, s32 = oracle.sweep_fields(out)
    W, L = 128, 1001
    x = w.images.view(np.float32).reshape(3, L)
    rows = (L + W - 1) // W
    xp = np.zeros((3, rows * W), dtype=np.float32)
    xp[:, :L] = x
    seq = np.add.accumulate(xp.reshape(3, rows, W), axis=1, dtype=np.float32)[:, -1, :]
    assert np.array_equal(s32.reshape(3, W), seq)


# ---------------------------------------------------------------------------
# Nested program: invariants
# ---------------------------------------------------------------------------
def test_nested_invariants():
    w = wl.nested(teams=6, threads=256, depth=3, elems_per_team=4096)
    out, st = oracle.run_workload(w)
    assert (st["status"] == 0).all()
    assert (st["depth_final"] == 0).all()
    assert (st["hwm_bytes"] == 3 * 1088).all()
    assert (st["spill_bytes"] == 0).all()
    u = out.view(np.uint32).reshape(6, 4096)
    # mix32 is a bijection: inverting it exposes e ^ acc, and acc depends on
    # j only through j mod 256 (the array index; j mod 16 follows from it)
    for t in range(6):
        e = t * 4096 + np.arange(4096, dtype=np.uint64)
        acc = np.array([_inv_mix32(int(v)) for v in u[t]], dtype=np.uint64) ^ e
        acc = acc.reshape(16, 256)
        assert (acc == acc[0]).all()
        assert len(set(acc[0].tolist())) > 200  # not degenerate
    # different teams see different frames (per-team keys)
    assert not np.array_equal(u[0], u[1])


def test_nested_depth_one_and_four():
    for depth in (1, 2, 4):
        w = wl.nested(teams=2, threads=128, depth=depth, elems_per_team=512)
        out, st = oracle.run_workload(w)
        assert (st["depth_final"] == 0).all()
        assert (st["hwm_bytes"] == depth * 1088).all()


def test_nested_overflow_equivalence():
    """Frame placement (slab or overflow) never changes results (Sec. 5.2:
    the global list is a correctness safety net)."""
    w = wl.nested(teams=4, threads=256, depth=3, elems_per_team=4096)
    ref, st_ref = oracle.run_workload(w)
    for slab, ovf, spill in [(0, 1 << 20, 3264), (1088, 1 << 20, 2176),
                             (2176, 1 << 20, 1088), (3264, 0, 0)]:
        out, st = oracle.run_workload(w, slab_bytes=slab, overflow_bytes=ovf)
        assert np.array_equal(out, ref)
        assert np.array_equal(st["chk"], st_ref["chk"])
        assert (st["spill_bytes"] == spill).all()
        assert (st["hwm_bytes"] == 3264).all()


def test_nested_push_failure_unwinds():
    w = wl.nested(teams=2, threads=256, depth=3, elems_per_team=4096)
    out, st = oracle.run_workload(w, slab_bytes=1088, overflow_bytes=1088)
    assert (st["status"] == oracle.ERR_OVERFLOW).all()
    assert (st["depth_final"] == 0).all()
    assert (out == 0).all()  # only the innermost level writes the output


# ---------------------------------------------------------------------------
# Hetero program: invariants
# ---------------------------------------------------------------------------
def test_hetero_invariants_and_placement():
    w = wl.hetero(n_instances=40, max_teams=6)
    ref, st_ref = oracle.run_workload(w)
    assert (st_ref["status"] == 0).all() and (st_ref["depth_final"] == 0).all()
    for r in w.regions:
        need = sum((b + 15) // 16 * 16 for b in r.frame_bytes)
        rows = st_ref[r.status_index: r.status_index + r.teams]
        assert (rows["hwm_bytes"] == need).all()
    out0, st0 = oracle.run_workload(w, slab_bytes=0, overflow_bytes=1 << 20)
    assert np.array_equal(out0, ref) and np.array_equal(st0["chk"], st_ref["chk"])
    assert (st0["spill_bytes"] == st0["hwm_bytes"]).all()


def test_hetero_team_of_one():
    """threads == 32: no workers; the master runs every region as a team of
    one, so the single output per team sums every frame word."""
    shapes = wl.hetero_shapes(400)
    idx = [i for i in range(400) if shapes[1][i] == 32][:5]
    assert idx
    w = wl.hetero(n_instances=400, instances=idx)
    out, st = oracle.run_workload(w)
    assert (st["status"] == 0).all()
    for r in w.regions:
        assert r.team_width == 1
        rows = st[r.status_index: r.status_index + r.teams]
        assert (rows["depth_final"] == 0).all()


def test_hetero_visibility_chain():
    """Level k+1's first word carries c_k, the sum the master read after the
    join of level k: flipping image word 0 of level 1 changes chk[0] of every
    team and, since word 0 of both frames is summed by worker 0 alone, exactly
    the outputs of worker 0."""
    shapes = wl.hetero_shapes(300)
    i = next(i for i in range(300) if shapes[2][i] == 2 and shapes[0][i] >= 2)
    w = wl.hetero(n_instances=300, instances=[i])
    out1, st1 = oracle.run_workload(w)
    imgs = w.images.copy()
    imgs[0] ^= 1
    w2 = wl.Workload("t", w.regions, imgs, w.out_bytes, w.n_status)
    out2, st2 = oracle.run_workload(w2)
    assert (st1["chk"][:, 0] != st2["chk"][:, 0]).all()
    r = w.regions[0]
    n = r.teams * r.team_width
    changed = (out1[:n] != out2[:n]).reshape(r.teams, r.team_width)
    assert changed[:, 0].all() and not changed[:, 1:].any()


# ---------------------------------------------------------------------------
# Worker-level sharing (the paper's future work, Sec. 7): structure and
# stack accounting
# ---------------------------------------------------------------------------
def _workers_run(work, slab=1 << 20, ovf=0):
    out, st = oracle.run_workload(work, slab_bytes=slab, overflow_bytes=ovf)
    r = work.regions[0]
    return out.view(np.uint32).reshape(r.teams, r.team_width), st


def _workers_with_image(work, img_u32):
    return wl.Workload("t", work.regions, img_u32.view(np.uint8), work.out_bytes, work.n_status)


def test_workers_s2_xors_every_output():
    """out[t] = (sum of worker t's frame) ^ s2: flipping bits of s2 flips
    the same bits of every output of that team, and nothing else."""
    w = wl.workers(teams=3, threads=96, frame_bytes=100)
    ref, _ = _workers_run(w)
    img = w.images.view(np.uint32).copy()
    stride = (16 + 112) // 4
    img[stride * 1 + 2] ^= 0x00F0F001  # team 1's s2
    got, _ = _workers_run(_workers_with_image(w, img))
    assert (got[1] ^ ref[1] == 0x00F0F001).all()
    assert np.array_equal(got[[0, 2]], ref[[0, 2]])


def test_workers_key_follows_the_worker_number():
    """Worker t's frame is keyed by mix32(s0 + t): raising s0 by k gives
    worker t the frame worker t + k had, so the outputs shift by k, across
    warp boundaries too."""
    w = wl.workers(teams=2, threads=128, frame_bytes=136)  # W' = 96: three warps
    ref, _ = _workers_run(w)
    img = w.images.view(np.uint32).copy()
    k = 37
    stride = (16 + 144) // 4
    img[0] = (int(img[0]) + k) & M32  # team 0's s0
    got, _ = _workers_run(_workers_with_image(w, img))
    assert np.array_equal(got[0][: 96 - k], ref[0][k:])
    assert np.array_equal(got[1], ref[1])
    assert not np.array_equal(got[0], ref[0])


def test_workers_every_worker_shares_the_base_image():
    """Every worker's frame starts from the same base words: changing one
    base word changes every output of that team (a bijective hash of the
    word is part of every sum), and two teams with the same image agree."""
    w = wl.workers(teams=2, threads=64, frame_bytes=64)
    img = w.images.view(np.uint32).copy()
    stride = (16 + 64) // 4
    img[stride: 2 * stride] = img[:stride]
    same, _ = _workers_run(_workers_with_image(w, img))
    assert np.array_equal(same[0], same[1])
    assert len(set(same[0].tolist())) == same.shape[1]  # distinct keys per worker
    img[4 + 9] ^= 1
    diff, _ = _workers_run(_workers_with_image(w, img))
    assert (diff[0] != same[0]).all() and np.array_equal(diff[1], same[1])


def test_workers_width_keeps_worker_numbers():
    """A narrower region runs workers 0 .. width-1 with the same frames."""
    full, _ = _workers_run(wl.workers(teams=2, threads=128, frame_bytes=40))
    part, _ = _workers_run(wl.workers(teams=2, threads=128, frame_bytes=40, width=45))
    assert np.array_equal(part, full[:, :45])


def test_workers_stack_accounting_and_placement():
    """hwm = the master's 16-byte frame + every warp's live worker frames;
    what the slab shares cannot hold goes to the overflow shares; results
    do not depend on placement."""
    S, fp = 200, 208
    w = wl.workers(teams=2, threads=96, frame_bytes=S, width=40)  # warps of 32 and 8 workers
    ref, st = _workers_run(w, slab=1 << 20)
    assert (st["status"] == 0).all() and (st["depth_final"] == 0).all()
    assert (st["hwm_bytes"] == 16 + 40 * fp).all() and (st["spill_bytes"] == 0).all()
    assert (st["chk"][:, 0] == ref.sum(axis=1, dtype=np.uint32)).all()
    # slab shares of 10 frames per warp, overflow shares of 22
    got, st2 = _workers_run(w, slab=16 + 2 * 10 * fp, ovf=2 * 22 * fp)
    assert np.array_equal(got, ref) and (st2["status"] == 0).all()
    assert (st2["spill_bytes"] == 22 * fp).all() and (st2["hwm_bytes"] == 16 + 40 * fp).all()
    # everything in the overflow slab (the master's frame too)
    got, st3 = _workers_run(w, slab=0, ovf=16 + 2 * 32 * fp)
    assert np.array_equal(got, ref) and (st3["spill_bytes"] == 16 + 40 * fp).all()


def test_workers_overflow_stops_at_the_first_frame_that_fits_nowhere():
    S, fp = 200, 208
    w = wl.workers(teams=1, threads=96, frame_bytes=S, width=40)
    ref, _ = _workers_run(w)
    got, st = _workers_run(w, slab=16 + 2 * 10 * fp, ovf=2 * 10 * fp)
    assert st["status"][0] == oracle.ERR_OVERFLOW and st["depth_final"][0] == 0
    # warp 0 places 20 of its 32 frames; warp 1 all 8 of its frames
    assert np.array_equal(got[0, :20], ref[0, :20]) and (got[0, 20:32] == 0).all()
    assert np.array_equal(got[0, 32:], ref[0, 32:])
    assert st["hwm_bytes"][0] == 16 + 28 * fp and st["spill_bytes"][0] == 10 * fp
    assert (st["chk"][0] == 0).all()


# ---------------------------------------------------------------------------
# Stack allocator (Sec. 5.3 shared stack + Sec. 5.2 fallback)
# ---------------------------------------------------------------------------
def test_stack_lifo_and_placement():
    s = oracle.Stack(slab_bytes=100, overflow_bytes=1000)
    a = s.push(40)     # 48 in slab
    b = s.push(60)     # 64 > 52 left -> overflow
    c = s.push(30)     # 32 fits in slab
    assert (a[1], b[1], c[1]) == (True, False, True)
    st = s.state()
    assert st["slab_used"] == 80 and st["overflow_used"] == 64 and st["hwm"] == 144
    assert s.pop(b[0]) == oracle.ERR_LIFO    # not the top frame
    s2 = oracle.Stack(100, 1000)
    i0, _ = s2.push(16)
    i1, _ = s2.push(16)
    assert s2.pop(i1) == 0 and s2.pop(i0) == 0
    assert s2.state()["depth"] == 0 and s2.state()["hwm"] == 32


def test_stack_capacity_failure():
    s = oracle.Stack(slab_bytes=32, overflow_bytes=32)
    assert s.push(32) == (0, True)
    assert s.push(17) == (1, False)   # rounds to 32: fits the overflow slab exactly
    assert s.push(1)[0] == -1
    s3 = oracle.Stack(slab_bytes=32, overflow_bytes=32)
    assert s3.push(32)[0] == 0 and s3.push(32)[0] == 1 and s3.push(1)[0] == -1
    assert s3.state()["status"] == oracle.ERR_OVERFLOW


def test_invalid_descriptors_rejected():
    bad = [
        wl.Region(wl.PROG_NESTED, 1, 256, 3, [1088, 1088, 1000], param=16),
        wl.Region(wl.PROG_SCALARS, 1, 100, 1, [16]),
        wl.Region(wl.PROG_SCALARS, 1, 128, 1, [16], param=0),
        wl.Region(wl.PROG_SCALARS, 1, 128, 1, [16], width=97, param=1),
        wl.Region(99, 1, 128, 1, [16]),
        wl.Region(wl.PROG_HETERO, 1, 128, 5, [16] * 4),
        wl.Region(wl.PROG_WORKERS, 1, 32, 2, [16, 64]),   # no worker warp
        wl.Region(wl.PROG_WORKERS, 1, 128, 2, [32, 64]),  # master frame is s[4]
        wl.Region(wl.PROG_WORKERS, 1, 128, 1, [16]),
    ]
    for r in bad:
        st = np.zeros(1, dtype=oracle.STATUS_DTYPE)
        assert oracle.run_region(r, np.zeros(64, np.uint8), np.zeros(64, np.int32), st) \
            == oracle.ERR_INVALID
