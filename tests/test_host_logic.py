"""The library's CUDA-free host logic (csrc/host_logic.h), compiled with g++
and checked on the CPU: the host call's segmentation, the batch submission's
grouping and stream placement, the overlap check, and the serving arena."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2012_01968_gb300", "csrc")
DRIVER = os.path.join(ROOT, "tests", "host_logic_driver.cpp")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("hl") / "host_logic")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-I", CSRC, DRIVER, "-o", exe], check=True)

    def call(text):
        return subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.splitlines()
    return call


# -- segments ---------------------------------------------------------------
CASES = [(b, L, m) for b in (1, 2, 3, 4, 5, 6, 7, 13, 100) for L in (1, 2, 5, 45, 60) for m in (1, 3, 6)]


def test_segments_cover_each_limb_once(run):
    out = run("".join(f"segments {b} {L} {m}\n" for b, L, m in CASES))
    for (b, L, m), line in zip(CASES, out):
        v = [int(x) for x in line.split()]
        segs = [tuple(v[1 + 4 * i: 5 + 4 * i]) for i in range(v[0])]
        assert 1 <= len(segs) <= m
        pos = 0
        for first, count, prime0, lview in segs:
            assert first == pos and count >= 1
            pos += count
            inside = first // L == (first + count - 1) // L and prime0 == first % L and lview == count
            whole = first % L == 0 and count % L == 0 and prime0 == 0 and lview == L
            assert inside or whole, (b, L, m, first, count, prime0, lview)
        assert pos == b * L
        if b < m:
            # a polynomial still gives several pieces when it has the limbs for it
            assert len(segs) >= b * min(L, m // b)


# -- overlap check ------------------------------------------------------------
def test_overlap_matches_brute_force(run):
    rng = np.random.default_rng(1)
    lines, want = [], []
    for _ in range(300):
        n = int(rng.integers(1, 8))
        r = []
        for _ in range(n):
            lo = int(rng.integers(0, 200)) * 16
            r.append((lo, lo + int(rng.integers(1, 40)) * 16))
        lines.append(f"overlap {n} " + " ".join(f"{a} {b}" for a, b in r) + "\n")
        want.append(any(r[i][0] < r[j][1] and r[j][0] < r[i][1] for i in range(n) for j in range(i + 1, n)))
    got = [line.strip() == "1" for line in run("".join(lines))]
    assert got == want


# -- grouping into launches ---------------------------------------------------------
def test_chunks_group_by_key_and_cap_jobs(run):
    rng = np.random.default_rng(2)
    for trial in range(40):
        nj = int(rng.integers(1, 80))
        maxj = int(rng.choice([1, 3, 16]))
        jobs = [(int(rng.integers(13, 18)), int(rng.integers(1, 3)), int(rng.integers(0, 3)),
                 int(rng.integers(1, 120)), 1 << int(rng.integers(13, 18))) for _ in range(nj)]
        text = f"chunks {nj} {maxj} " + " ".join(" ".join(map(str, j)) for j in jobs) + "\n"
        line = run(text)[0]
        parts = line.split(";")
        chunks = []
        for p in parts[1:]:
            v = p.split()
            key = tuple(int(x) for x in v[:3])
            limbs, work, cnt = int(v[3]), float(v[4]), int(v[5])
            idx = [int(x) for x in v[6:6 + cnt]]
            chunks.append((key, limbs, work, idx))
        assert int(parts[0]) == len(chunks)
        seen = sorted(i for c in chunks for i in c[3])
        assert seen == list(range(nj))                          # every job exactly once
        for key, limbs, work, idx in chunks:
            assert 1 <= len(idx) <= maxj
            assert all(jobs[i][:3] == key for i in idx)          # one size, direction, OT setting
            assert idx == sorted(idx)                            # submission order within a launch
            assert limbs == sum(jobs[i][3] for i in idx)
            assert work == pytest.approx(sum(jobs[i][3] * jobs[i][4] for i in idx))
        works = [c[2] for c in chunks]
        assert works == sorted(works, reverse=True)              # longest launches first
        # a key's jobs fill whole chunks of maxj except at most one
        for key in {j[:3] for j in jobs}:
            sizes = [len(c[3]) for c in chunks if c[0] == key]
            assert sum(1 for s in sizes if s < maxj) <= 1


def test_least_loaded_placement(run):
    rng = np.random.default_rng(3)
    for _ in range(50):
        nw, st = int(rng.integers(1, 40)), int(rng.integers(1, 5))
        w = sorted((float(x) for x in rng.integers(1, 1000, nw)), reverse=True)
        at = [int(x) for x in run(f"place {nw} {st} " + " ".join(map(str, w)) + "\n")[0].split()]
        assert len(at) == nw and all(0 <= k < st for k in at)
        load = [0.0] * st
        for x, k in zip(w, at):
            load[k] += x
        # greedy least-loaded: the spread of the loads stays within the largest item
        assert max(load) - min(load) <= max(w) + 1e-9


# -- serving arena ------------------------------------------------------------------
def _round(b):
    return (b + 255) // 256 * 256


def _gaps(used, cap):
    pos, out = 0, []
    for a, b in sorted(used):
        if a > pos:
            out.append((pos, a))
        pos = max(pos, b)
    if pos < cap:
        out.append((pos, cap))
    return out


def _check_alloc(ok, off, nbytes, used, cap):
    """One reply of the arena against the free space of the live set `used`."""
    rb = _round(nbytes)
    fitting = [lo for lo, hi in _gaps(used, cap) if hi - lo >= rb]
    assert bool(ok) == bool(fitting), "allocation failed although a gap fits (or succeeded without one)"
    if ok:
        assert off == min(fitting)                      # first fit: the lowest gap that fits
        used.append((off, off + rb))


def _replies(line, n):
    v = line.split("|")[0].split()
    out, i = [], 0
    while len(out) < n:
        if v[i] == "r":
            i += 1
            continue
        out.append((int(v[i]), int(v[i + 1])))
        i += 2
    return out


def test_arena_first_fit_with_frees(run):
    rng = np.random.default_rng(4)
    for trial in range(30):
        cap = int(rng.integers(4, 64)) * 4096
        first = [int(x) for x in rng.integers(1, 20000, int(rng.integers(1, 30)))]
        # pass 1: where the first allocations land
        reps = _replies(run(f"arena {cap} {len(first)} " + " ".join(f"a {b}" for b in first) + "\n")[0], len(first))
        used = []
        for (ok, off), b in zip(reps, first):
            _check_alloc(ok, off, b, used, cap)
        live = [(off, b) for (ok, off), b in zip(reps, first) if ok]
        # pass 2: the same, then free a random subset, then allocate more
        freed = [live[i] for i in sorted(rng.choice(len(live), size=len(live) // 2, replace=False))] if live else []
        more = [int(x) for x in rng.integers(1, 20000, int(rng.integers(1, 20)))]
        cmd = [f"a {b}" for b in first] + [f"r {o} {b}" for o, b in freed] + [f"a {b}" for b in more]
        reps2 = _replies(run(f"arena {cap} {len(cmd)} " + " ".join(cmd) + "\n")[0], len(first) + len(more))
        assert reps2[:len(first)] == reps
        used = [(o, o + _round(b)) for o, b in live if (o, b) not in freed]
        for (ok, off), b in zip(reps2[len(first):], more):
            _check_alloc(ok, off, b, used, cap)


def test_arena_release_coalesces(run):
    """Blocks freed in a shuffled order merge back into the one initial range."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(1, 5000, 20)]
    cap = 1 << 20
    reps = _replies(run(f"arena {cap} {len(sizes)} " + " ".join(f"a {b}" for b in sizes) + "\n")[0], len(sizes))
    assert all(ok for ok, _ in reps)
    order = rng.permutation(len(sizes))
    cmd = [f"a {b}" for b in sizes] + [f"r {reps[i][1]} {sizes[i]}" for i in order]
    line = run(f"arena {cap} {len(cmd)} " + " ".join(cmd) + "\n")[0]
    assert [int(x) for x in line.split("|")[1].split()] == [1, 0, cap]


# -- autotuner candidates and choice ------------------------------------------------
def test_tune_candidates_cover_the_space(run):
    for n in range(1, 18):
        line = run(f"tune {n} 3 12\n")[0]
        cands = [tuple(int(x) for x in c.split()) for c in line.split(";") if c.strip()]
        assert len(set(cands)) == len(cands)                         # no duplicates
        if n <= 12:
            want = [(0, 1, 0, 0), (3, 1, 0, 0), (4, 1, 0, 0)]             # one-pass kernel, radix-2, high radix
            if n >= 10:
                want.append((5, 1, 0, 0))                               # and the cluster kernel
            assert cands == want
            continue
        want = {(k, t, o, g) for g in range(3) for k in (1, 2) for t, o in ((1, 0), (2, 1), (2, 2))}
        want.add((3, 1, 0, 0))                                       # radix-2: table, default geometry
        want.add((4, 1, 0, 0))                                       # high radix: table, default geometry
        assert set(cands) == want


def test_tune_pick_is_the_argmin(run):
    rng = np.random.default_rng(6)
    for _ in range(200):
        m = int(rng.integers(1, 20))
        f = rng.uniform(1, 100, m).round(3)
        v = rng.uniform(1, 100, m).round(3)
        ok = rng.random(m) < 0.8
        if rng.random() < 0.2:
            f[:] = 5.0
            v[:] = 5.0                                               # all tied: the first timed one
        text = f"pick {m} " + " ".join(f"{a} {b} {int(o)}" for a, b, o in zip(f, v, ok)) + "\n"
        got = int(run(text)[0])
        if not ok.any():
            assert got == -1
            continue
        tot = np.where(ok, f + v, np.inf)
        assert got == int(np.argmin(tot))                            # argmin takes the first of ties
