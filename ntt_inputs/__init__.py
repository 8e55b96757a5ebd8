"""Seeded synthetic inputs for the negacyclic RNS NTT workloads.

This module is the only code shared by the CPU oracle side (tests, the
oracle timing leg of bench.py) and the CUDA side (tests, bench.py, smoke).
It holds no transform arithmetic: it draws coefficients, finds prime chains
that the workloads name, and describes the five workload shapes.

Generator (counter based, so it vectorises): splitmix64 as published by
Steele, Lea and Flood (OOPSLA 2014, "Fast splittable pseudorandom number
generators"; reference C by S. Vigna).  The i-th output (i = 0, 1, ...) of
the stream with 64-bit state ``key`` is ``mix(key + (i + 1) * GAMMA)``.
A stream key is derived from (seed, poly, limb) by ``mix`` chaining.

Uniform residues in [0, q): take the top ``q.bit_length()`` bits of each draw
and keep those < q, in draw order (exact rejection sampling; acceptance is at
least 1/2, and above 1 - 2^-29 for the 60-bit primes used here).

Coefficients of polynomial ``poly`` at limb ``l`` come from stream
key(seed, poly, l); the draw order within a limb is the coefficient order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


# ----------------------------------------------------------------------------
# splitmix64
# ----------------------------------------------------------------------------
def mix64(z: int) -> int:
    """splitmix64 output function on a Python int (mod 2^64)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * _M1) & MASK64
    z = ((z ^ (z >> 27)) * _M2) & MASK64
    return z ^ (z >> 31)


def mix64_np(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function, vectorised over a uint64 array."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(_M2)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, *ids: int) -> int:
    """64-bit stream state for (seed, id0, id1, ...)."""
    k = mix64(seed + GAMMA)
    for i in ids:
        k = mix64(k ^ mix64((i + 1) * GAMMA))
    return k


def draws(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream with state ``key``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + idx * np.uint64(GAMMA)
    return mix64_np(z)


def uniform_mod(q: int, n: int, key: int) -> np.ndarray:
    """n exactly-uniform residues in [0, q) from the stream ``key`` (rejection)."""
    if q < 2:
        raise ValueError("modulus must be >= 2")
    bits = q.bit_length()
    shift = np.uint64(64 - bits)
    out = np.empty(n, dtype=np.uint64)
    have = 0
    pos = 0
    qq = np.uint64(q)
    while have < n:
        need = n - have
        chunk = need + need // 8 + 64
        cand = draws(key, pos, chunk) >> shift
        pos += chunk
        ok = cand[cand < qq]
        take = min(need, ok.size)
        out[have:have + take] = ok[:take]
        have += take
    return out


def poly_uniform(seed: int, poly: int, primes, N: int) -> np.ndarray:
    """One RNS polynomial, shape [L, N], limb l uniform in [0, primes[l])."""
    L = len(primes)
    out = np.empty((L, N), dtype=np.uint64)
    for l, q in enumerate(primes):
        out[l] = uniform_mod(int(q), N, stream_key(seed, poly, l))
    return out


def batch_uniform(seed: int, batch: int, primes, N: int, first_poly: int = 0) -> np.ndarray:
    """``batch`` polynomials, shape [batch, L, N] (the library's layout)."""
    return np.stack([poly_uniform(seed, first_poly + b, primes, N) for b in range(batch)])


def uniform_floats(key: int, n: int) -> np.ndarray:
    """n doubles uniform in (0, 1) (53-bit), for arrival times and choices."""
    d = draws(key, 0, n) >> np.uint64(11)
    return (d.astype(np.float64) + 0.5) * (1.0 / (1 << 53))


def uniform_ints(key: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive), by exact rejection."""
    span = hi - lo + 1
    return uniform_mod(span, n, key).astype(np.int64) + lo if span > 1 else np.full(n, lo, np.int64)


# ----------------------------------------------------------------------------
# primes (input setup: the workloads name their moduli by this rule)
# ----------------------------------------------------------------------------
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (first twelve prime bases)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def prime_chain(count: int, modulus: int, below: int = 1 << 60) -> list[int]:
    """The ``count`` largest primes q < ``below`` with q = 1 mod ``modulus``, descending."""
    out = []
    q = ((below - 2) // modulus) * modulus + 1
    while len(out) < count:
        if q < 2:
            raise ValueError("not enough primes")
        if is_prime(q):
            out.append(q)
        q -= modulus
    return out


def small_ntt_primes(N: int, count: int, start: int = 2) -> list[int]:
    """The ``count`` smallest primes q >= start with q = 1 mod 2N (ascending)."""
    m = 2 * N
    q = ((max(start, 2) - 1 + m - 1) // m) * m + 1
    out = []
    while len(out) < count:
        if is_prime(q):
            out.append(q)
        q += m
    return out


# ----------------------------------------------------------------------------
# workload shapes
# ----------------------------------------------------------------------------
@dataclass
class Job:
    """One transform job of an uneven batch: a polynomial of L limbs of size N."""
    N: int
    L: int
    dir: int            # +1 forward, -1 inverse
    poly: int           # polynomial index, picks the coefficient stream


@dataclass
class Workload:
    name: str
    seed: int
    N: int = 0
    L: int = 0
    batch: int = 1
    primes: list = field(default_factory=list)
    jobs: list = field(default_factory=list)
    note: str = ""


def chain_for(N: int, count: int) -> list[int]:
    return prime_chain(count, 2 * N)


def workload_c1() -> Workload:
    """Single limb, N = 2^12, largest 60-bit prime = 1 mod 2^13, seed 1."""
    return Workload("c1_n4096_l1", 1, N=1 << 12, L=1, batch=1, primes=chain_for(1 << 12, 1))


def workload_c2() -> Workload:
    """N = 2^16, L = 45 (largest primes < 2^60, = 1 mod 2^17, descending), seed 2."""
    return Workload("c2_n65536_l45", 2, N=1 << 16, L=45, batch=1, primes=chain_for(1 << 16, 45))


def workload_c3() -> Workload:
    """N = 2^17, L = 60 (= 1 mod 2^18), batch 2 (one ciphertext), seed 3."""
    return Workload("c3_n131072_l60_b2", 3, N=1 << 17, L=60, batch=2, primes=chain_for(1 << 17, 60))


def workload_c4(count: int = 96) -> Workload:
    """Uneven batch, seed 4: N in {2^14..2^17}, L in [1, 60], dir in {fwd, inv}.

    All jobs draw their primes from one chain of the 60 largest primes < 2^60
    with q = 1 mod 2^18 (valid for every N <= 2^17); a job at level L uses the
    first L primes.
    """
    key = stream_key(4, 0xC4)
    logn = uniform_ints(stream_key(4, 0xC4, 1), count, 14, 17)
    Ls = uniform_ints(stream_key(4, 0xC4, 2), count, 1, 60)
    dirs = uniform_ints(stream_key(4, 0xC4, 3), count, 0, 1)
    del key
    jobs = [Job(1 << int(logn[i]), int(Ls[i]), 1 if dirs[i] == 0 else -1, i) for i in range(count)]
    return Workload("c4_uneven96", 4, primes=prime_chain(60, 1 << 18), jobs=jobs)


@dataclass
class Request:
    t_arrival: float    # seconds from stream start
    N: int
    L: int
    dir: int
    poly: int


def serving_requests(count: int = 20000, rate_per_s: float = 1000.0, seed: int = 5):
    """Poisson arrivals at ``rate_per_s``; N in {2^15, 2^16, 2^17}; L in [4, 60]."""
    u = uniform_floats(stream_key(seed, 0xC5, 0), count)
    gaps = -np.log(u) / rate_per_s
    t = np.cumsum(gaps)
    logn = uniform_ints(stream_key(seed, 0xC5, 1), count, 15, 17)
    Ls = uniform_ints(stream_key(seed, 0xC5, 2), count, 4, 60)
    dirs = uniform_ints(stream_key(seed, 0xC5, 3), count, 0, 1)
    return [Request(float(t[i]), 1 << int(logn[i]), int(Ls[i]), 1 if dirs[i] == 0 else -1, i)
            for i in range(count)]


def workload_c5() -> Workload:
    return Workload("c5_serving20000", 5, primes=prime_chain(60, 1 << 18))


def chain_2_18_60() -> list[int]:
    return prime_chain(60, 1 << 18)


def log2_exact(n: int) -> int:
    k = int(math.log2(n))
    if (1 << k) != n:
        raise ValueError("not a power of two")
    return k
