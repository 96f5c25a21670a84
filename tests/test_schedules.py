"""Schedule enumeration: the oracle's sequential worker order against every
interleaving of the workers.

The oracle runs each parallel region's workers one after another. OpenMP
gives no such order: workers run concurrently between the fork and the join
(Sec. 4, Fig. "codegen-worker"), and master/worker accesses never race
because of the fork/join barriers (Sec. 5.1). For a race-free program every
schedule must give the same result, and the oracle's result must be it.

This file models the runtime independently of the oracle: a word-addressed
memory, frames placed in it by a bump allocator, the master's code run
atomically between joins and forks, and each worker a generator of single
memory operations (read or write of one word). A stateless model checker
replays the program once per schedule and enumerates every interleaving of
worker steps (exhaustively on tiny instances, by random sampling on the
larger nested frames). A racy negative control shows the checker does see
different schedules.
"""
import random

import numpy as np

import oracle
import workloads as wl

M32 = 0xFFFFFFFF


def mix32(x):
    # pinned against published vectors in test_oracle_pins
    return oracle.mix32(x)


class Scheduler:
    """Replays a prefix of choices, then takes choice 0, recording branching."""

    def __init__(self, prefix=(), rng=None):
        self.prefix = list(prefix)
        self.pos = 0
        self.branching = []
        self.rng = rng

    def choose(self, n):
        if n == 1:
            return 0
        if self.rng is not None:
            c = self.rng.randrange(n)
        elif self.pos < len(self.prefix):
            c = self.prefix[self.pos]
        else:
            c = 0
        self.branching.append(n)
        self.pos += 1
        return c


def enumerate_schedules(run, limit=200000):
    """Run `run(scheduler)` once per interleaving; returns the results."""
    results, todo, n = [], [[]], 0
    while todo:
        prefix = todo.pop()
        s = Scheduler(prefix)
        results.append(run(s))
        n += 1
        assert n <= limit, "schedule space too large for exhaustive enumeration"
        taken = prefix + [0] * (len(s.branching) - len(prefix))
        for i in range(len(prefix), len(s.branching)):
            for alt in range(1, s.branching[i]):
                todo.append(taken[:i] + [alt])
    return results


class Machine:
    """Word-addressed memory with a bump-allocated frame stack."""

    FRAMES = 1 << 20
    OUT = 1 << 24

    def __init__(self):
        self.mem = {}
        self.sp = self.FRAMES
        self.frames = []

    def push(self, words):
        base = self.sp
        self.sp += words
        self.frames.append((base, words))
        return base

    def pop(self, base):
        assert self.frames and self.frames[-1][0] == base, "LIFO"
        self.frames.pop()
        self.sp = base

    def parallel(self, sched, bodies):
        """Fork: run the worker generators interleaved; join when all end."""
        pending = []
        for g in bodies:
            try:
                pending.append([g, next(g)])
            except StopIteration:
                pass
        while pending:
            i = sched.choose(len(pending))
            g, op = pending[i]
            if op[0] == "r":
                val = self.mem.get(op[1], 0)
            else:
                self.mem[op[1]] = op[2] & M32
                val = None
            try:
                pending[i][1] = g.send(val)
            except StopIteration:
                pending.pop(i)


# ---------------------------------------------------------------------------
# The hetero program (heterogeneous instances), modelled
# ---------------------------------------------------------------------------
def hetero_model(region, images_u32, sched):
    m = Machine()
    W = region.team_width
    D = region.depth
    outs, chks = {}, {}
    for team in range(region.teams):
        F = []
        c_prev = 0
        woff = region.image_offset // 4
        for k in range(1, D + 1):
            L = region.frame_bytes[k - 1] // 4
            base = m.push(L)
            F.append((base, L))
            key = mix32((region.salt + team * 8 + k) & M32)
            for i in range(L):
                m.mem[base + i] = int(images_u32[woff + i]) ^ key
            woff += ((region.frame_bytes[k - 1] + 15) // 16) * 4
            if k > 1:
                m.mem[base] ^= c_prev

            def update(tid, base=base, L=L):
                for i in range(tid, L, W):
                    v = yield ("r", base + i)
                    yield ("w", base + i, mix32((v + i) & M32))

            def inner(tid, team=team, Fs=list(F)):
                acc = 0
                for mlev, (b, Lm) in enumerate(Fs, start=1):
                    for i in range(tid, Lm, W):
                        v = yield ("r", b + i)
                        acc = (acc + mix32(v ^ (mlev << 24) ^ i)) & M32
                yield ("w", m.OUT + team * W + tid, acc)

            body = update if k < D else inner
            m.parallel(sched, [body(t) for t in range(W)])
            if k < D:
                c_prev = sum(m.mem[base + i] for i in range(L)) & M32
                chks[(team, k - 1)] = c_prev
        chks[(team, D - 1)] = m.mem[F[-1][0]]
        for base, _ in reversed(F):
            m.pop(base)
        for t in range(W):
            outs[team * W + t] = m.mem.get(m.OUT + team * W + t, 0)
    return tuple(outs[i] for i in sorted(outs)), tuple(chks[k] for k in sorted(chks))


def _tiny_hetero(teams, threads, frame_bytes, salt=12345, seed=7):
    r = wl.Region(wl.PROG_HETERO, teams, threads, len(frame_bytes), list(frame_bytes), salt=salt)
    words = sum((b + 15) // 16 * 4 for b in frame_bytes)
    imgs = wl.uniform_u32(wl.derive(seed, 99, len(frame_bytes)), words)
    return r, imgs


def _oracle_hetero(r, imgs):
    w = r.team_width
    work = wl.Workload("t", [r], imgs.view(np.uint8), 4 * r.teams * w, r.teams)
    out, st = oracle.run_workload(work)
    outs = tuple(int(v) for v in out.view(np.uint32))
    chks = tuple(int(st["chk"][t][k]) for t in range(r.teams) for k in range(r.depth))
    return outs, chks


def test_hetero_every_schedule_matches_oracle():
    # (teams, threads, width, frame bytes per level): 2-3 active workers via
    # the region width (the other workers skip the body), or a team of one
    cases = [
        (1, 64, 2, (16, 8)),
        (2, 64, 3, (12,)),
        (1, 64, 2, (8, 8, 8)),
        (1, 32, 0, (16, 12)),
    ]
    for teams, threads, width, fb in cases:
        r, imgs = _tiny_hetero(teams, threads, fb)
        r.width = width
        ref = _oracle_hetero(r, imgs)
        results = enumerate_schedules(lambda s: hetero_model(r, imgs, s))
        assert len(results) > 1 or r.team_width == 1
        assert set(results) == {ref}, (teams, threads, width, fb)


def test_racy_control_shows_several_outcomes():
    """Two workers increment one shared word without atomics: the checker
    must find both the lost-update and the serial outcome."""
    def run(s):
        m = Machine()
        base = m.push(1)
        m.mem[base] = 0

        def body(tid):
            v = yield ("r", base)
            yield ("w", base, v + 1)
        m.parallel(s, [body(t) for t in range(2)])
        return m.mem[base]
    assert set(enumerate_schedules(run)) == {1, 2}


# ---------------------------------------------------------------------------
# The nested program, modelled; 1088-byte frames are too big for
# exhaustive enumeration, so schedules are sampled at random
# ---------------------------------------------------------------------------
def nested_model(region, images_u32, sched):
    m = Machine()
    W, D, E = region.team_width, region.depth, region.param
    outs, chks = {}, {}
    for team in range(region.teams):
        F = []
        for k in range(1, D + 1):
            base = m.push(272)
            F.append(base)
            key = mix32(team * 8 + k)
            src = (team * D + (k - 1)) * 272
            for i in range(272):
                m.mem[base + i] = int(images_u32[src + i]) ^ key
            if k > 1:
                m.mem[base] ^= m.mem[F[k - 2] + 15]

            def update(tid, base=base):
                for i in range(tid, 256, W):
                    v = yield ("r", base + 16 + i)
                    yield ("w", base + 16 + i, mix32((v + i) & M32))

            def inner(tid, team=team, Fs=list(F)):
                for j in range(tid, E, W):
                    acc = 0
                    for b in Fs:
                        a = yield ("r", b + 16 + (j & 255))
                        s = yield ("r", b + (j & 15))
                        acc = (acc + (a ^ s)) & M32
                    e = team * E + j
                    yield ("w", m.OUT + e, mix32(e ^ acc))

            m.parallel(sched, [(update if k < D else inner)(t) for t in range(W)])
            if k < D:
                m.mem[base + 15] = sum(m.mem[base + 16 + i] for i in range(256)) & M32
        for k in range(D, 0, -1):
            chks[(team, k - 1)] = m.mem[F[k - 1] + 15]
            m.pop(F[k - 1])
        for j in range(E):
            outs[team * E + j] = m.mem.get(m.OUT + team * E + j, 0)
    return tuple(outs[i] for i in sorted(outs)), tuple(chks[k] for k in sorted(chks))


def test_nested_sampled_schedules_match_oracle():
    for teams, depth, width, E in [(2, 2, 3, 12), (1, 3, 2, 8)]:
        work = wl.nested(teams=teams, threads=64, depth=depth, elems_per_team=E, seed=11)
        r = work.regions[0]
        r.width = width
        out, st = oracle.run_workload(work)
        ref = (tuple(int(v) for v in out.view(np.uint32)),
               tuple(int(st["chk"][t][k]) for t in range(teams) for k in range(depth)))
        imgs = work.images.view(np.uint32)
        rng = random.Random(1234)
        seen = set()
        for _ in range(60):
            seen.add(nested_model(r, imgs, Scheduler(rng=rng)))
        assert seen == {ref}


# ---------------------------------------------------------------------------
# The scalars program and the paper's programs: exhaustive on tiny instances
# ---------------------------------------------------------------------------
def scalars_model(region, images_u32, sched):
    m = Machine()
    W = region.team_width
    for team in range(region.teams):
        for r in range(region.param):
            base = m.push(4)
            for i in range(4):
                m.mem[base + i] = int(images_u32[4 * r + i])

            def body(tid, base=base, r=r, team=team):
                s0 = yield ("r", base)
                s1 = yield ("r", base + 1)
                s2 = yield ("r", base + 2)
                s3 = yield ("r", base + 3)
                v = ((s0 * tid + s1) & M32) ^ (((s2 >> (tid & 7)) + s3) & M32)
                yield ("w", m.OUT + (r * region.teams + team) * W + tid, v)
            m.parallel(sched, [body(t) for t in range(W)])
            m.pop(base)
    n = region.param * region.teams * W
    return tuple(m.mem.get(m.OUT + i, 0) for i in range(n))


def test_scalars_every_schedule_matches_oracle():
    work = wl.scalars(n_regions=2, teams=1, threads=64, seed=3)
    r = work.regions[0]
    r.width = 2
    work.out_bytes = 4 * 2 * 2
    out, _ = oracle.run_workload(work)
    ref = tuple(int(v) for v in out.view(np.uint32))
    results = enumerate_schedules(lambda s: scalars_model(r, work.images.view(np.uint32), s))
    assert len(results) == 252 * 252  # C(10,5) interleavings per region
    assert set(results) == {ref}


def paper_scalars_model(region, a_init, sched):
    """Fig. "8 variables": the frame holds c[n] and a reference to a."""
    m = Machine()
    W, n = region.team_width, region.param
    A = m.OUT
    for i, v in enumerate(a_init.view(np.uint32).tolist()):
        m.mem[A + i] = v
    for team in range(region.teams):
        base = m.push(n + 1)
        for i in range(n):
            m.mem[base + i] = 0
        for i in range(n):
            m.mem[base + i] += i + 1
        m.mem[base + n] = A  # the shared reference

        def body(tid, base=base, team=team):
            a = yield ("r", base + n)
            total = 0
            for i in range(n):
                c = yield ("r", base + i)
                total += c
            old = yield ("r", a + team * W + tid)
            yield ("w", a + team * W + tid, old + total)
        m.parallel(sched, [body(t) for t in range(W)])
        m.pop(base)
    return tuple(m.mem[A + i] for i in range(region.teams * W))


def test_paper_scalars_every_schedule_matches_oracle():
    work = wl.paper_scalars(n_vars=3, teams=1, threads=64)
    r = work.regions[0]
    r.width = 2
    a0 = work.out_init[: r.teams * 2].copy()
    work.out_init = a0
    work.out_bytes = 4 * a0.size
    out, _ = oracle.run_workload(work)
    ref = tuple(int(v) for v in out.view(np.uint32))
    results = enumerate_schedules(lambda s: paper_scalars_model(r, a0, s))
    assert len(results) == 924 and set(results) == {ref}  # C(12,6)


# ---------------------------------------------------------------------------
# Worker-level sharing (Sec. 7): every worker is the master of a nested
# region run by 32 inner threads. The model interleaves the workers' steps
# and, inside each worker's nested region, its inner threads' steps (the
# scheduler picks the inner thread too), so schedules mix steps of
# different workers' nested regions; they are sampled at random.
# ---------------------------------------------------------------------------
def workers_model(region, images_u32, sched):
    m = Machine()
    Wp = region.team_width
    S = region.frame_bytes[1]
    L = S // 4
    stride = (16 + (S + 15) // 16 * 16) // 4
    outs, chks = {}, {}
    for team in range(region.teams):
        src = team * stride
        F = m.push(4)
        for i in range(4):
            m.mem[F + i] = int(images_u32[src + i])

        def inner(j, g, s1):
            for w in range(j, L, 32):
                v = yield ("r", g + w)
                yield ("w", g + w, mix32((v + s1 + w) & M32))

        def worker(t, team=team, src=src):
            g = m.FRAMES + 4096 + (team * Wp + t) * L  # this worker's frame
            s0 = yield ("r", F)
            key = mix32((s0 + t) & M32)
            for i in range(L):
                yield ("w", g + i, int(images_u32[src + 4 + i]) ^ key)
            s1 = yield ("r", F + 1)
            pending = []
            for j in range(32):
                it = inner(j, g, s1)
                try:
                    pending.append([it, next(it)])
                except StopIteration:
                    pass
            while pending:
                i = sched.choose(len(pending))
                it, op = pending[i]
                val = yield op
                try:
                    pending[i][1] = it.send(val)
                except StopIteration:
                    pending.pop(i)
            total = 0
            for i in range(L):
                v = yield ("r", g + i)
                total = (total + v) & M32
            s2 = yield ("r", F + 2)
            yield ("w", m.OUT + team * Wp + t, total ^ s2)

        m.parallel(sched, [worker(t) for t in range(Wp)])
        chks[team] = sum(m.mem.get(m.OUT + team * Wp + t, 0) for t in range(Wp)) & M32
        m.pop(F)
        for t in range(Wp):
            outs[team * Wp + t] = m.mem.get(m.OUT + team * Wp + t, 0)
    return tuple(outs[i] for i in sorted(outs)), tuple(chks[t] for t in sorted(chks))


def test_workers_sampled_schedules_match_oracle():
    for teams, threads, width, S in [(2, 64, 3, 140), (1, 96, 34, 12)]:
        work = wl.workers(teams=teams, threads=threads, frame_bytes=S, width=width, seed=5)
        r = work.regions[0]
        out, st = oracle.run_workload(work, slab_bytes=1 << 20)
        ref = (tuple(int(v) for v in out.view(np.uint32)),
               tuple(int(st["chk"][t][0]) for t in range(teams)))
        imgs = work.images.view(np.uint32)
        rng = random.Random(99)
        seen = set()
        for _ in range(25):
            seen.add(workers_model(r, imgs, Scheduler(rng=rng)))
        assert seen == {ref}
