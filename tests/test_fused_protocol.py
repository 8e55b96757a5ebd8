"""The fused kernel's scheduling protocol, simulated on the CPU.

Each CTA of ntt_fused_kernel has compute warps (a consumer of a ring of tile
buffers) and one producer thread (an event loop that claims units from one
queue per phase, at most one ahead of the unit in compute, loads tiles,
stores computed tiles and publishes the tiles of every phase but the last on
per-limb counters; the producer whose tile completes a limb appends the limb
to that phase's publication order, and the next phase's tickets map to limbs
in that order).  A launch has two phases (one transform: column then row
pass, or row then column) or four (forward then inverse).  Claims: a
published ticket of the latest phase by compare-and-swap, else a phase-0
ticket, else, once every ticket of the phases below p is taken, a phase-p
ticket held until its limb is published.  With staged row twiddles, each
CTA's producer copies a row tile's later-round twiddles into one per-CTA
buffer once the previous row tile has released it, and the compute warps
wait for that copy before reading it.

Here both sides of every CTA are generators mirroring that control flow; a
random scheduler interleaves them and completes the asynchronous copies
after random delays.  Checked for many seeds and shapes:
  * a tile of phase p > 0 is loaded only after every tile of phase p - 1 of
    its limb has been stored completely;
  * a buffer is refilled only after the store that last used it has read it
    (the producer waits with the kernel's slack: all but the newest store
    with three buffers, every store with two);
  * a limb counter is raised only for stores that completed;
  * the staged-twiddle buffer is refilled only after the previous row tile
    released it, and read only after its copy landed, in row-tile order;
  * every tile of every phase is computed exactly once, the run finishes (no
    deadlock), and every CTA reaches the finished count.
"""
import random

import pytest


class Sim:
    def __init__(self, limbs, units, rows, rng):
        self.limbs, self.units, self.rows = limbs, units, rows      # units[p]; rows[p]: row-tile phase
        self.NP = len(units)
        self.tickets = [0] * self.NP
        self.done = [[0] * limbs for _ in range(self.NP)]
        self.order = [[] for _ in range(self.NP)]                  # published limbs per phase
        self.stored = [[set() for _ in range(limbs)] for _ in range(self.NP)]
        self.computed = [[[0] * units[p] for _ in range(limbs)] for p in range(self.NP)]
        self.finished = 0
        self.rng = rng
        self.now = 0
        self.events = []

    def later(self, fn, lo=1, hi=40):
        self.events.append((self.now + self.rng.randint(lo, hi), fn))


def kernel_read_slack(nbuf):
    """Stores the kernel lets still read their buffers when it refills one:
    all but the newest with three buffers, none with two."""
    return 0 if nbuf == 2 else 1


class Cta:
    def __init__(self, sim, nbuf, stage, slack=None):
        self.s = sim
        self.NBUF = nbuf
        self.slack = kernel_read_slack(nbuf) if slack is None else slack
        self.stage = stage
        self.full = [0] * nbuf          # completed phases per buffer
        self.empty = [0] * nbuf
        self.desc = [None] * nbuf
        self.stores = []                # committed stores in order
        self.bufstore = {}
        self.htw_full = 0               # staged-twiddle copies landed
        self.htw_empty = 0              # row tiles that released the buffer
        self.htw_tile = []              # (phase, limb, tile) of each fill, in order

    # async copies ------------------------------------------------------
    def load(self, p, limb, tile, issued):
        s = self.s
        b = issued % self.NBUF
        if p > 0:
            assert len(s.stored[p - 1][limb]) == s.units[p - 1], \
                "tile loaded before every tile of the previous phase of its limb was stored"
        st = self.bufstore.get(b)
        assert st is None or st["read"], "buffer refilled before its store read it"
        self.desc[b] = (p, limb, tile)

        def fin():
            self.full[b] += 1
        s.later(fin)

    def store(self, b):
        s = self.s
        p, limb, tile = self.desc[b]
        st = {"read": False, "done": False}

        def rd():
            st["read"] = True

        def fin():
            st["done"] = True
            s.stored[p][limb].add(tile)
        s.later(rd, 1, 10)
        s.later(fin, 11, 60)
        self.stores.append(st)
        self.bufstore[b] = st
        return st

    # producer ------------------------------------------------------------
    def producer(self):
        s = self.s
        NP, NBUF = s.NP, self.NBUF
        issued = stored = 0
        fifo = []                       # (store, (phase, limb) or None)
        left = (1 << NP) - 1
        stopped = False
        held = None                     # (phase, ticket)
        hq = []                         # row units loaded, staged twiddles not yet copied
        fills = 0

        def publish(e):
            if e is not None:
                p, limb = e
                s.done[p][limb] += 1
                if s.done[p][limb] == s.units[p]:
                    s.order[p].append(limb)

        def wait_all_but(n):
            while not all(x["done"] for x in (self.stores[:-n] if n else self.stores)):
                yield

        def publish_older():
            nonlocal fifo
            if len(fifo) >= 2:
                yield from wait_all_but(1)
                for st, e in fifo[:-1]:
                    assert st["done"], "limb counter raised before the store completed"
                    publish(e)
                fifo = fifo[-1:]

        def publish_all():
            nonlocal fifo
            if fifo:
                yield from wait_all_but(0)
                for st, e in fifo:
                    assert st["done"]
                    publish(e)
                fifo = []

        def wait_read(n):
            # cp.async.bulk.wait_group.read n: all but the n newest stores have read
            while not all(x["read"] for x in (self.stores[:-n] if n else self.stores)):
                yield

        def pub_limb(p, i):
            return s.order[p][i] if i < len(s.order[p]) else None

        def do_load(p, limb, tile):
            nonlocal issued
            yield from wait_read(self.slack)
            self.load(p, limb, tile, issued)
            if self.stage and s.rows[p]:
                hq.append(issued)
            issued += 1

        def fill_htw():
            nonlocal fills
            if not self.stage or not hq:
                return False
            if fills and self.htw_empty < fills:
                return False
            assert self.htw_empty == fills, "staged twiddles copied before the previous row tile released them"
            u = hq.pop(0)
            self.htw_tile.append(self.desc[u % NBUF])

            def fin():
                self.htw_full += 1
            s.later(fin)
            fills += 1
            return True

        def claim():
            nonlocal left, held
            for p in range(NP - 1, 0, -1):
                if not (left >> p) & 1:
                    continue
                tot = s.limbs * s.units[p]
                t = s.tickets[p]
                if t >= tot:
                    left &= ~(1 << p)
                    continue
                limb = pub_limb(p - 1, t // s.units[p])
                if limb is not None and s.tickets[p] == t:       # compare-and-swap
                    s.tickets[p] = t + 1
                    yield from do_load(p, limb, t % s.units[p])
                    return True
            if left & 1:
                t = s.tickets[0]
                s.tickets[0] += 1
                if t < s.limbs * s.units[0]:
                    yield from do_load(0, t // s.units[0], t % s.units[0])
                    return True
                left &= ~1
            for p in range(1, NP):
                if left & ((1 << p) - 1):
                    break
                if not (left >> p) & 1:
                    continue
                t = s.tickets[p]
                s.tickets[p] += 1
                if t >= s.limbs * s.units[p]:
                    left &= ~(1 << p)
                    continue
                limb = pub_limb(p - 1, t // s.units[p])
                if limb is not None:
                    yield from do_load(p, limb, t % s.units[p])
                else:
                    held = (p, t)
                return True
            return False

        while True:
            progress = fill_htw()
            while stored < issued and self.empty[stored % NBUF] > stored // NBUF:
                b = stored % NBUF
                p, limb, tile = self.desc[b]
                st = self.store(b)
                fifo.append((st, (p, limb) if p + 1 < NP else None))
                stored += 1
                yield from publish_older()
                progress = True
            if stopped:
                if stored + 1 == issued:
                    break
            elif issued - stored < 2:
                if held is not None:
                    p, t = held
                    limb = pub_limb(p - 1, t // s.units[p])
                    if limb is not None:
                        yield from do_load(p, limb, t % s.units[p])
                        held = None
                        progress = True
                else:
                    if (yield from claim()):
                        progress = True
                    if left == 0 and held is None:
                        b = issued % NBUF
                        self.desc[b] = ("STOP", 0, 0)
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
        s.finished += 1

    # compute warps ----------------------------------------------------------
    def compute(self):
        s = self.s
        NBUF = self.NBUF
        k = rt = 0
        while True:
            b = k % NBUF
            while self.full[b] <= k // NBUF:
                yield
            p, limb, tile = self.desc[b]
            if p == "STOP":
                return
            if self.stage and s.rows[p]:
                while self.htw_full <= rt:
                    yield
                assert self.htw_tile[rt] == (p, limb, tile), "staged twiddles of another row tile"
            for _ in range(s.rng.randint(1, 6)):
                yield
            if self.stage and s.rows[p]:
                self.htw_empty += 1
                rt += 1
            s.computed[p][limb][tile] += 1
            self.empty[b] += 1
            k += 1


def simulate(limbs, units, rows, ctas, seed, nbuf, stage, max_steps=4_000_000, slack=None):
    rng = random.Random(seed)
    sim = Sim(limbs, units, rows, rng)
    gens = []
    for _ in range(ctas):
        c = Cta(sim, nbuf, stage, slack)
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
    for p in range(sim.NP):
        assert all(c == 1 for row in sim.computed[p] for c in row), f"phase {p}: a tile computed twice or never"
    for p in range(sim.NP - 1):
        assert sim.done[p] == [units[p]] * limbs
        assert sorted(sim.order[p]) == list(range(limbs))
    assert sim.finished == ctas


# (units per phase, row-tile phases): forward (column, row), inverse (row,
# column), forward then inverse (column, row, row, column)
SHAPES = {"fwd": ((16, 16), (False, True)), "inv": ((16, 16), (True, False)),
          "chain": ((16, 16, 16, 16), (False, True, True, False)),
          "fwd_uneven": ((8, 32), (False, True)), "chain_uneven": ((8, 4, 4, 8), (False, True, True, False))}


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("nbuf,stage", [(3, False), (2, True)])
@pytest.mark.parametrize("limbs,ctas", [(1, 1), (1, 7), (3, 2), (6, 9), (12, 24)])
def test_protocol(shape, nbuf, stage, limbs, ctas):
    units, rows = SHAPES[shape]
    for seed in range(3):
        simulate(limbs, units, rows, ctas, seed * 7919 + limbs * 31 + ctas, nbuf, stage)


def test_protocol_many_ctas_few_limbs():
    """More CTAs than tiles of a phase: most producers hold tickets."""
    simulate(2, (4, 4, 4, 4), (False, True, True, False), 40, 5, 2, True)


def test_two_buffers_need_every_store_read():
    """With two buffers the refilled buffer is the newest store's: waiting for
    all but the newest store (the three-buffer rule) lets a load overwrite a
    tile its store has not read yet, which the model catches."""
    caught = 0
    for seed in range(20):
        try:
            simulate(6, (16, 16), (False, True), 4, seed, 2, True, slack=1)
        except AssertionError as e:
            assert "before its store read it" in str(e)
            caught += 1
    assert caught > 0
