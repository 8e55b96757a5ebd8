"""The fused kernel's scheduling protocol, simulated on the CPU.

Each CTA of ntt_fused_kernel has compute warps (a consumer of a ring of three
tile buffers) and one producer thread (an event loop that claims units from
two queues, at most one ahead of the unit in compute, loads tiles, stores
computed tiles and publishes first-pass tiles on per-limb counters; the
producer whose tile completes a limb appends the limb to the publication
order, and second-pass tickets map to limbs in that order).  Here both sides of every CTA are generators mirroring
that control flow; a random scheduler interleaves them and completes the
asynchronous copies after random delays.  Checked for many seeds and shapes:
  * a second-pass tile is loaded only after every first-pass tile of its limb
    has been stored completely;
  * a buffer is refilled only after the store that last used it has read it;
  * a limb counter is raised only for stores that completed;
  * every unit is computed exactly once, the run finishes (no deadlock), and
    every CTA reaches the finished count;
for B-first ordering (window 0), a small look-ahead window and A-first.
"""
import random

import pytest

import kernel_model as KM

NBUF = 3


class Sim:
    def __init__(self, limbs, UA, UB, rng):
        self.limbs, self.UA, self.UB = limbs, UA, UB
        self.totalA, self.totalB = limbs * UA, limbs * UB
        self.ctl = [0, 0, 0]            # next A ticket, next B ticket, CTAs finished
        self.done = [0] * limbs
        self.order = []                 # published limbs, in publication order
        self.a_stored = [set() for _ in range(limbs)]
        self.computedA = [0] * self.totalA
        self.computedB = [0] * self.totalB
        self.rng = rng
        self.now = 0
        self.events = []

    def later(self, fn, lo=1, hi=40):
        self.events.append((self.now + self.rng.randint(lo, hi), fn))


class Cta:
    def __init__(self, sim, peek=True, window=0):
        self.s = sim
        self.peek = peek
        self.window = window
        self.full = [0] * NBUF          # completed phases per buffer
        self.empty = [0] * NBUF
        self.desc = [None] * NBUF
        self.stores = []                # committed stores in order
        self.bufstore = {}

    # async copies ------------------------------------------------------
    def load(self, kind, limb, tile, t, issued):
        s = self.s
        b = issued % NBUF
        if kind == "B":
            assert len(s.a_stored[limb]) == s.UA, "B tile loaded before its limb's A tiles were stored"
        st = self.bufstore.get(b)
        assert st is None or st["read"], "buffer refilled before its store read it"
        self.desc[b] = (kind, limb, tile, t)

        def fin():
            self.full[b] += 1
        s.later(fin)

    def store(self, b):
        s = self.s
        kind, limb, tile, t = self.desc[b]
        st = {"read": False, "done": False}

        def rd():
            st["read"] = True

        def fin():
            st["done"] = True
            if kind == "A":
                s.a_stored[limb].add(tile)
        s.later(rd, 1, 10)
        s.later(fin, 11, 60)
        self.stores.append(st)
        self.bufstore[b] = st
        return st

    # producer ------------------------------------------------------------
    def producer(self):
        s = self.s
        issued = stored = 0
        fifo = []                       # (store, limb or None)
        a_left = b_left = True
        stopped = False
        held = None

        def publish(limb):
            if limb is not None:
                s.done[limb] += 1
                if s.done[limb] == s.UA:
                    s.order.append(limb)

        def wait_all_but(n):
            while not all(x["done"] for x in (self.stores[:-n] if n else self.stores)):
                yield

        def publish_older():
            nonlocal fifo
            if len(fifo) >= 2:
                yield from wait_all_but(1)
                for st, limb in fifo[:-1]:
                    assert st["done"], "limb counter raised before the store completed"
                    publish(limb)
                fifo = fifo[-1:]

        def publish_all():
            nonlocal fifo
            if fifo:
                yield from wait_all_but(0)
                for st, limb in fifo:
                    assert st["done"]
                    publish(limb)
                fifo = []

        def wait_read_all():
            while not all(x["read"] for x in self.stores):
                yield

        def b_limb(t):
            pos = t // s.UB
            return s.order[pos] if pos < len(s.order) else None

        def do_load(kind, limb, tile, t):
            nonlocal issued
            yield from wait_read_all()
            self.load(kind, limb, tile, t, issued)
            issued += 1

        while True:
            progress = False
            while stored < issued and self.empty[stored % NBUF] > stored // NBUF:
                b = stored % NBUF
                kind, limb, tile, t = self.desc[b]
                st = self.store(b)
                fifo.append((st, limb if kind == "A" else None))
                stored += 1
                yield from publish_older()
                progress = True
            if stopped:
                if stored + 1 == issued:
                    break
            elif issued - stored < 2:
                if held is not None:
                    if b_limb(held) is not None:
                        yield from do_load("B", b_limb(held), held % s.UB, held)
                        held = None
                        progress = True
                else:
                    claimed = False
                    if b_left and a_left and self.peek:
                        pk = s.ctl[1]
                        if pk >= s.totalB:
                            b_left = False
                        elif s.ctl[0] // s.UA >= pk // s.UB + self.window and b_limb(pk) is not None:
                            t = s.ctl[1]
                            s.ctl[1] += 1
                            if t < s.totalB:
                                if b_limb(t) is not None:
                                    yield from do_load("B", b_limb(t), t % s.UB, t)
                                else:
                                    held = t
                                claimed = True
                            else:
                                b_left = False
                    if not claimed and a_left:
                        t = s.ctl[0]
                        s.ctl[0] += 1
                        if t < s.totalA:
                            yield from do_load("A", t // s.UA, t % s.UA, t)
                            claimed = True
                        else:
                            a_left = False
                    if not claimed and b_left:
                        t = s.ctl[1]
                        s.ctl[1] += 1
                        if t < s.totalB:
                            if b_limb(t) is not None:
                                yield from do_load("B", b_limb(t), t % s.UB, t)
                            else:
                                held = t
                            claimed = True
                        else:
                            b_left = False
                    if claimed:
                        progress = True
                    if not a_left and not b_left and held is None:
                        b = issued % NBUF
                        self.desc[b] = ("STOP", 0, 0, 0)
                        self.full[b] += 1
                        issued += 1
                        stopped = True
                        progress = True
            if progress:
                yield
                continue
            yield from publish_all()
            yield
        yield from publish_all()
        s.ctl[2] += 1

    # compute warps ----------------------------------------------------------
    def compute(self):
        s = self.s
        k = 0
        while True:
            b = k % NBUF
            while self.full[b] <= k // NBUF:
                yield
            kind, limb, tile, t = self.desc[b]
            if kind == "STOP":
                return
            for _ in range(s.rng.randint(1, 6)):
                yield
            if kind == "A":
                s.computedA[t] += 1
            else:
                s.computedB[limb * s.UB + tile] += 1     # every (limb, tile), not every ticket
            self.empty[b] += 1
            k += 1


def simulate(limbs, UA, UB, ctas, seed, peek=True, window=0, max_steps=3_000_000):
    rng = random.Random(seed)
    sim = Sim(limbs, UA, UB, rng)
    gens = []
    for _ in range(ctas):
        c = Cta(sim, peek, window)
        gens += [c.producer(), c.compute()]
    alive = list(range(len(gens)))
    steps = 0
    while alive:
        steps += 1
        assert steps < max_steps, "no progress (deadlock)"
        sim.now += 1
        due = [e for e in sim.events if e[0] <= sim.now]
        sim.events = [e for e in sim.events if e[0] > sim.now]
        for _, fn in due:
            fn()
        i = rng.choice(alive)
        try:
            next(gens[i])
        except StopIteration:
            alive.remove(i)
    for _, fn in sorted(sim.events, key=lambda e: e[0]):
        fn()
    assert all(c == 1 for c in sim.computedA) and all(c == 1 for c in sim.computedB)
    assert sim.done == [UA] * limbs
    assert sorted(sim.order) == list(range(limbs))
    assert sim.ctl[2] == ctas


@pytest.mark.parametrize("limbs,UA,UB,ctas", [(6, 8, 2, 60), (3, 16, 16, 96), (45, 16, 16, 40),
                                               (45, 16, 16, 304), (1, 4, 4, 8), (20, 2, 8, 7),
                                               (120, 32, 32, 64)])
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("peek,window", [(True, 0), (False, 0), (True, 2), (True, 1 << 24)])
def test_protocol_random_interleavings(limbs, UA, UB, ctas, seed, peek, window):
    simulate(limbs, UA, UB, ctas, seed, peek, window)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
def test_fused_tile_counts_cover_limb(n):
    UC, UR = KM.fused_geometry(n)
    p1, p2 = KM.split(n)
    assert UC * 16 * (1 << p1) == 1 << n          # column tiles: 16 columns x R1 rows
    assert UR * (1 << KM.logc_rows(p2)) * (1 << p2) == 1 << n
