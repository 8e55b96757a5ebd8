"""The CPU model of the pass kernels (index math, lazy ranges) against the oracle.

Checks on the CPU, before any GPU run, that the kernels' tile geometry,
round schedule, twiddle indexing (table and on-the-fly) and lazy reduction
steps compute the oracle's transform, with every intermediate value inside the
bound the kernel assumes.
"""
import random

import numpy as np
import pytest

import ntt_inputs as I
import kernel_model as KM


def _case(n, seed):
    N = 1 << n
    q = I.prime_chain(2, 2 * N)[seed % 2]
    rng = random.Random(seed)
    a = [rng.randrange(q) for _ in range(N)]
    return N, q, a


@pytest.mark.parametrize("n", list(range(1, 15)))
def test_model_matches_oracle_table(orc, n):
    N, q, a = _case(n, n)
    psi = orc.psi(q, N)
    want = orc.ntt_radix2(a, q)
    got = KM.transform(a, q, psi, n, True)
    assert got == [int(v) for v in want]
    back = KM.transform(got, q, psi, n, False)
    assert back == a
    # inverse on arbitrary (not forward-produced) input, with edge values
    y = list(a)
    y[0], y[-1] = q - 1, 0
    assert KM.transform(y, q, psi, n, False) == [int(v) for v in orc.intt_radix2(y, q)]


@pytest.mark.parametrize("n,ots", [(13, 1), (13, 2), (14, 1), (14, 2)])
def test_model_matches_oracle_ot(orc, n, ots):
    N, q, a = _case(n, 100 + n)
    psi = orc.psi(q, N)
    got = KM.transform(a, q, psi, n, True, ots)
    assert got == [int(v) for v in orc.ntt_radix2(a, q)]
    assert KM.transform(got, q, psi, n, False, ots) == a


@pytest.mark.slow
@pytest.mark.parametrize("n,ots", [(15, 0), (16, 1), (17, 2)])
def test_model_large_geometries(orc, n, ots):
    N, q, a = _case(n, 200 + n)
    psi = orc.psi(q, N)
    got = KM.transform(a, q, psi, n, True, ots)
    assert got == [int(v) for v in orc.ntt_radix2(a, q)]
    assert KM.transform(got, q, psi, n, False, ots) == a


def test_model_extreme_values(orc):
    """All-(q-1) input keeps every lazy value in range (worst case for the bounds)."""
    n = 13
    N = 1 << n
    q = I.prime_chain(1, 2 * N)[0]
    psi = orc.psi(q, N)
    a = [q - 1] * N
    assert KM.transform(a, q, psi, n, True) == [int(v) for v in orc.ntt_radix2(a, q)]
    assert KM.transform(a, q, psi, n, False) == [int(v) for v in orc.intt_radix2(a, q)]


def test_final_reduction_every_bit_length():
    """The final reduction's quotient estimate is floor(x / q) or one less for
    every modulus bit length the 64-bit plans accept (2^32 < q < 2^60) and
    every x < 16q: the ends of each bit length, the multiples of q and their
    neighbours, and random values; canon gives x mod q."""
    rng = random.Random(2012)
    for k in range(33, 61):
        qs = [(1 << (k - 1)) + 1, (1 << k) - 1, rng.randrange(1 << (k - 1), 1 << k) | 1]
        for q in qs:
            rc, rsh = KM.reduction_constants(q)
            xs = [0, 16 * q - 1] + [m * q + d for m in range(1, 16) for d in (-1, 0, 1)]
            xs += [rng.randrange(16 * q) for _ in range(200)]
            for x in xs:
                r = KM.reduce2(x, q, rc, rsh)
                assert r % q == x % q
                for X in (5, 12, 16):
                    if x < X * q:
                        assert KM.canon(x, X, q, rc, rsh) == x % q


def test_sign_tested_subtraction_edges():
    """The sign-bit conditional subtraction at its limits: c = 8q for the
    largest q the plans accept (8q just below 2^63), x at 0, c - 1, c and
    2c - 1."""
    for q in ((1 << 60) - 1, (1 << 59) + 1, (1 << 32) + 15):
        for c in (q, 2 * q, 8 * q):
            for x in (0, 1, c - 1, c, c + 1, 2 * c - 1):
                assert KM.csub(x, c) == (x - c if x >= c else x)
    c = 1 << 63
    for x in (0, c - 1, c, 2 * c - 1):
        assert KM.csub(x, c) == (x - c if x >= c else x)


def test_final_reduction_worst_truncation():
    """x just below a multiple of q with every low bit below the shift set:
    the estimate's two truncations at their largest."""
    for k in (33, 40, 59, 60):
        q = (1 << k) - 1
        rc, rsh = KM.reduction_constants(q)
        for m in range(1, 16):
            x = m * q - 1
            x |= (1 << rsh) - 1
            if x < 16 * q:
                assert KM.reduce2(x, q, rc, rsh) % q == x % q


def test_swizzle_is_a_bijection_keeping_pairs():
    for tile in (2, 64, 4096, 8192):
        img = [KM.swz(w) for w in range(tile)]
        assert sorted(img) == list(range(tile))
        assert all(KM.swz(w) + 1 == KM.swz(w + 1) for w in range(0, tile, 2))


@pytest.mark.parametrize("P,LOGC,rows", [(8, 4, True), (8, 4, False), (9, 3, True), (7, 5, True),
                                          (7, 4, False), (6, 4, False), (12, 0, True)])
def test_round_accesses_bank_conflicts(P, LOGC, rows):
    """Shared-memory accesses of each round: at most 2-way bank conflicts.

    For 8-byte accesses a half-warp (16 lanes) is served per 128-byte
    wavefront: conflict-free iff the 16 word addresses are distinct mod 16.
    Rounds whose items are contiguous (rows, last round) use 16-byte accesses:
    a quarter-warp per wavefront, distinct 16-byte chunks mod 8.
    """
    sizes, starts = KM.rounds(P, 4)
    R, C = 1 << P, 1 << LOGC
    worst = 1
    for KR, K0 in zip(sizes, starts):
        NLO = P - K0 - KR
        E = 1 << KR
        pairs = rows and NLO == 0
        T = C << (P - sizes[0])
        for warp0 in range(0, min(T, 256), 32):
            lanes = range(warp0, min(warp0 + 32, T))
            for i in range(0, E, 2 if pairs else 1):
                addrs = []
                for it in lanes:
                    if rows:
                        lo = it & ((1 << NLO) - 1)
                        hi = (it >> NLO) & ((1 << K0) - 1)
                        cc = it >> (NLO + K0)
                    else:
                        cc = it & (C - 1)
                        lo = (it >> LOGC) & ((1 << NLO) - 1)
                        hi = it >> (LOGC + NLO)
                    v = ((hi << (P - K0)) | lo) | (i << NLO)
                    w = cc * R + v if rows else v * C + cc
                    addrs.append(KM.swz(w))
                group = 8 if pairs else 16
                for g0 in range(0, len(addrs), group):
                    grp = addrs[g0:g0 + group]
                    keys = [(a >> 1) % 8 for a in grp] if pairs else [a % 16 for a in grp]
                    worst = max(worst, max(keys.count(k) for k in set(keys)))
    assert worst <= 2, worst


@pytest.mark.parametrize("n,geometry,ots", [(13, 1, 0), (13, 2, 1), (14, 1, 2), (14, 2, 0), (14, 2, 2)])
def test_model_alternative_geometries(orc, n, geometry, ots):
    """The autotuner's geometries (half the row tile; the other pass split):
    the same transform, with the tables laid out for their split."""
    N, q, a = _case(n, 300 + n + geometry)
    psi = orc.psi(q, N)
    got = KM.transform(a, q, psi, n, True, ots, geometry)
    assert got == [int(v) for v in orc.ntt_radix2(a, q)]
    assert KM.transform(got, q, psi, n, False, ots, geometry) == a


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("geometry", [0, 1, 2])
def test_geometry_limits(n, geometry):
    """Each geometry fits the fused kernel: a column tile is one TMA box of 16
    columns x 2^p1 rows (at most 256), a row tile at most 4096 words in whole
    rows, and both passes tile the limb exactly."""
    p1, lr = KM.GEOMETRIES[n][geometry]
    p2 = n - p1
    assert 1 << p1 <= 256 and (1 << p2) >= 16
    assert (1 << (lr + p2)) <= 4096 and lr <= p1
    UC, UR = (1 << p2) // 16, (1 << p1) >> lr
    assert UC * 16 * (1 << p1) == 1 << n and UR * (1 << lr) * (1 << p2) == 1 << n


@pytest.mark.parametrize("n", [1, 2, 5, 7, 10])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_high_radix_index_maps(orc, n, k):
    """The high-radix organisation's items and twiddle indices give the
    oracle's transform for every radix, including a short last group."""
    N, q, a = _case(n, 400 + n + k)
    psi = orc.psi(q, N)
    got = KM.high_radix_transform(a, q, psi, n, k, True)
    assert got == [int(v) for v in orc.ntt_radix2(a, q)]
    assert KM.high_radix_transform(got, q, psi, n, k, False) == a


def test_shoup_product_range_adversarial():
    """The lazy Shoup product's quotient estimate (three partial products,
    32-bit pieces for the remainder) gives y*w mod q in [0, 4q) for any 64-bit
    y, checked at the extremes of y, w and the prime size."""
    rng = random.Random(7)
    primes = [I.prime_chain(1, 1 << 18)[0], (1 << 32) + 15 * (1 << 20) + 1, 1152921504266321921]
    M64 = (1 << 64) - 1
    for q in primes:
        for w in (0, 1, q - 1, q // 2, rng.randrange(q)):
            wp = (w << 64) // q
            for y in (0, 1, M64, M64 - 1, 16 * q - 1, (1 << 63), (1 << 32) - 1, 1 << 32,
                      rng.randrange(1 << 64)):
                r = KM.shoup_lazy(y, w, wp, q)
                assert 0 <= r < 4 * q and r % q == (y * w) % q
        for _ in range(2000):
            w = rng.randrange(q)
            wp = (w << 64) // q
            y = rng.randrange(1 << 64)
            KM.shoup_lazy(y, w, wp, q)
