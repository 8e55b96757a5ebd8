"""Pins for the CPU oracle: checks against facts the oracle does not produce.

Each ``pin_*`` takes a loaded oracle (``oracle.Oracle``) and raises
AssertionError on a mismatch.  They are run on the real oracle by
``test_oracle_pins.py`` and on deliberately broken copies of it by
``test_oracle_mutants.py`` (each planted mistake must trip at least one pin).

What pins what (paper: Kim, Jung, Park, Ahn; sections as printed):
* hand-worked fixtures in tests/golden (Sec. III-A definition, Algorithm 1 order);
* primality, factorisation and the smallest generator against sympy;
* psi^N = -1 and psi^2N = 1 (Sec. III-A: psi is a primitive 2N-th root);
* closed forms of the transform (delta, constants, the all-ones vector);
* every output is the input polynomial evaluated at a root of X^N + 1
  (Sec. III-A: A_k = a(psi^{2k+1})), checked with Python integers;
* the negacyclic product against a full product folded by X^N = -1;
* the convolution theorem of Sec. III-A (NTT, pointwise product, iNTT);
* Algorithm 1 against the O(N^2) definition, the round trip, linearity.
"""
from __future__ import annotations

import os
import random

import numpy as np

import ntt_inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden(name):
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                nums = [int(x) for x in v.split()]
                vals[k.strip()] = nums[0] if len(nums) == 1 else nums
    return vals


def _brv(i, n):
    return int(format(i, f"0{n}b")[::-1], 2) if n else 0


def _rand_vec(rng, N, q):
    return np.array([rng.randrange(q) for _ in range(N)], dtype=np.uint64)


# Primes used across pins: small ones (all classes of N <= 64) and 60-bit
# chain primes of the workloads.
SMALL = {N: I.small_ntt_primes(N, 2) for N in (2, 4, 8, 16, 32, 64)}
BIG_C1 = I.prime_chain(1, 1 << 13)[0]
BIG_C2 = I.prime_chain(2, 1 << 17)
BIG_218 = I.prime_chain(2, 1 << 18)


def pin_golden_q17_n4(o):
    g = _golden("ntt_q17_n4.txt")
    q, N = g["q"], g["N"]
    assert o.smallest_generator(q) == g["generator"]
    assert o.psi(q, N) == g["psi"]
    assert list(o.ntt_schoolbook(g["a"], q)) == g["ntt"]
    assert list(o.ntt_radix2(g["a"], q)) == g["ntt"]
    assert list(o.intt_radix2(g["ntt"], q)) == g["a"]
    assert list(o.intt_schoolbook(g["ntt"], q)) == g["a"]
    assert list(o.negacyclic_schoolbook(g["a"], g["b"], q)) == g["product"]


def pin_golden_q5_n2(o):
    g = _golden("ntt_q5_n2.txt")
    q, N = g["q"], g["N"]
    assert o.smallest_generator(q) == g["generator"]
    assert o.psi(q, N) == g["psi"]
    assert list(o.ntt_radix2(g["a"], q)) == g["ntt"]
    assert list(o.ntt_schoolbook(g["a"], q)) == g["ntt"]
    assert list(o.intt_radix2(g["ntt"], q)) == g["a"]
    assert list(o.intt_schoolbook(g["ntt"], q)) == g["a"]


def pin_primality_vs_sympy(o):
    import sympy
    rng = random.Random(11)
    cases = [0, 1, 2, 3, 4, 561, 1105, 1729, 2047, 3215031751, 2152302898747,
             3474749660383, 341550071728321, 3825123056546413051, (1 << 61) - 1,
             (1 << 64) - 59, (1 << 64) - 1]
    cases += BIG_C2 + BIG_218 + [BIG_C1]
    cases += [rng.getrandbits(64) | 1 for _ in range(300)]
    cases += [rng.getrandbits(rng.randrange(2, 40)) for _ in range(300)]
    for n in cases:
        assert o.is_prime(n) == sympy.isprime(n), n


def pin_factors_vs_sympy(o):
    import sympy
    rng = random.Random(12)
    ms = [q - 1 for q in BIG_C2 + BIG_218 + [BIG_C1]]
    ms += [rng.getrandbits(40) + 2 for _ in range(40)] + [2, 3, 4, 12, 97 * 89 * 89]
    for m in ms:
        assert o.prime_factors(m) == sorted(sympy.factorint(m)), m


def pin_generator_vs_sympy(o):
    import sympy
    qs = [5, 7, 17, 97, 193, 257, 7681, 12289, BIG_C1] + BIG_C2 + BIG_218
    for N, ps in SMALL.items():
        qs += ps
    for q in qs:
        assert o.smallest_generator(q) == sympy.primitive_root(q), q


def pin_psi_is_primitive_2n_root(o):
    cases = [(BIG_C1, 1 << 12)] + [(q, 1 << 16) for q in BIG_C2] + \
            [(q, 1 << k) for q in BIG_218 for k in (14, 15, 16, 17)] + \
            [(q, N) for N, ps in SMALL.items() for q in ps]
    for q, N in cases:
        p = o.psi(q, N)
        assert pow(p, N, q) == q - 1, (q, N)
        assert pow(p, 2 * N, q) == 1
        g = o.smallest_generator(q)
        assert p == pow(g, (q - 1) // (2 * N), q)
    assert o.psi(17, 16) == 0          # 2N = 32 does not divide 16
    assert o.psi(15, 1) == 0           # not prime


def pin_closed_forms(o):
    for N, ps in SMALL.items():
        for q in ps + [BIG_C2[0]]:
            n = N.bit_length() - 1
            p = pow(o.psi(q, N), 1, q)
            delta = np.zeros(N, np.uint64)
            delta[0] = 1
            assert (o.ntt_schoolbook(delta, q) == 1).all()
            assert (o.ntt_radix2(delta, q) == 1).all()
            c = (q - 1) // 3 + 1
            assert (o.ntt_radix2(delta * np.uint64(c), q) == c).all()
            ones = np.ones(N, np.uint64)
            want = [2 * pow((1 - pow(p, 2 * _brv(i, n) + 1, q)) % q, q - 2, q) % q
                    for i in range(N)]
            assert list(o.ntt_schoolbook(ones, q)) == want
            assert list(o.ntt_radix2(ones, q)) == want
            # X^j maps to psi^{j(2 brv(i) + 1)}
            j = N // 2 + 1 if N > 2 else 1
            mono = np.zeros(N, np.uint64)
            mono[j] = 1
            want = [pow(p, j * (2 * _brv(i, n) + 1), q) for i in range(N)]
            assert list(o.ntt_radix2(mono, q)) == want


def pin_outputs_are_root_evaluations(o):
    rng = random.Random(13)
    for N, ps in SMALL.items():
        for q in ps + [BIG_C1]:
            n = N.bit_length() - 1
            p = o.psi(q, N)
            xs = [pow(p, 2 * _brv(i, n) + 1, q) for i in range(N)]
            assert len(set(xs)) == N                       # N distinct points
            assert all(pow(x, N, q) == q - 1 for x in xs)   # roots of X^N + 1
            a = [rng.randrange(q) for _ in range(N)]
            want = [sum(a[j] * pow(x, j, q) for j in range(N)) % q for x in xs]
            assert list(o.ntt_radix2(a, q)) == want
            assert list(o.ntt_schoolbook(a, q)) == want
            assert [o.eval(a, x, q) for x in xs[:4]] == want[:4]


def pin_large_n_spot_evaluations(o):
    rng = random.Random(14)
    for q, N in ((BIG_C2[0], 1 << 16), (BIG_218[1], 1 << 17)):
        n = N.bit_length() - 1
        p = o.psi(q, N)
        a = _rand_vec(rng, N, q)
        out = o.ntt_radix2(a, q)
        al = [int(v) for v in a]
        for i in rng.sample(range(N), 6) + [0, N - 1]:
            x = pow(p, 2 * _brv(i, n) + 1, q)
            acc = 0
            for c in reversed(al):
                acc = (acc * x + c) % q
            assert int(out[i]) == acc, (q, N, i)


def _fold_product(a, b, q):
    """Full product of the polynomials, then X^N = -1 (independent of c_k)."""
    N = len(a)
    full = [0] * (2 * N - 1)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            full[i + j] += int(ai) * int(bj)
    return [(full[k] - (full[k + N] if k + N < 2 * N - 1 else 0)) % q for k in range(N)]


def pin_negacyclic_product(o):
    rng = random.Random(15)
    for N, ps in SMALL.items():
        for q in ps + [BIG_C2[1]]:
            a = [rng.randrange(q) for _ in range(N)]
            b = [rng.randrange(q) for _ in range(N)]
            assert list(o.negacyclic_schoolbook(a, b, q)) == _fold_product(a, b, q)
    # monomial: X^j * a is the signed cyclic shift
    q, N = BIG_C1, 32
    a = [rng.randrange(q) for _ in range(N)]
    for j in (1, 5, 31):
        xj = [0] * N
        xj[j] = 1
        want = [(-a[k - j + N]) % q if k < j else a[k - j] for k in range(N)]
        assert list(o.negacyclic_schoolbook(a, xj, q)) == want


def pin_convolution_theorem(o):
    rng = random.Random(16)
    cases = [(q, N) for N, ps in SMALL.items() for q in ps]
    cases += [(BIG_C1, 256), (BIG_C2[0], 1024), (BIG_218[0], 512)]
    for q, N in cases:
        a = _rand_vec(rng, N, q)
        b = _rand_vec(rng, N, q)
        A, B = o.ntt_radix2(a, q), o.ntt_radix2(b, q)
        C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], np.uint64)
        assert list(o.pointwise(A, B, q)) == list(C)
        c = o.intt_radix2(C, q)
        assert list(c) == list(o.negacyclic_schoolbook(a, b, q)), (q, N)


def pin_radix2_matches_definition(o):
    rng = random.Random(17)
    cases = [(q, N) for N, ps in SMALL.items() for q in ps]
    cases += [(BIG_C1, 64), (BIG_C2[1], 32), (BIG_218[1], 128)]
    for q, N in cases:
        a = _rand_vec(rng, N, q)
        A = o.ntt_schoolbook(a, q)
        assert list(o.ntt_radix2(a, q)) == list(A), (q, N)
        assert list(o.intt_schoolbook(A, q)) == list(a)
        assert list(o.intt_radix2(A, q)) == list(a)
        Y = _rand_vec(rng, N, q)
        assert list(o.intt_radix2(Y, q)) == list(o.intt_schoolbook(Y, q))


def pin_round_trip_and_linearity(o):
    rng = random.Random(18)
    for q, N in ((BIG_C1, 1 << 12), (BIG_C2[0], 1 << 14), (BIG_218[0], 1 << 17)):
        a = _rand_vec(rng, N, q)
        b = _rand_vec(rng, N, q)
        A, B = o.ntt_radix2(a, q), o.ntt_radix2(b, q)
        assert (o.intt_radix2(A, q) == a).all()
        assert (o.ntt_radix2(o.intt_radix2(a, q), q) == a).all()
        s = np.array([(int(x) + int(y)) % q for x, y in zip(a, b)], np.uint64)
        S = np.array([(int(x) + int(y)) % q for x, y in zip(A, B)], np.uint64)
        assert (o.ntt_radix2(s, q) == S).all()
        # edge values: all q-1, zeros
        top = np.full(N, q - 1, np.uint64)
        T = o.ntt_radix2(top, q)
        assert (o.intt_radix2(T, q) == top).all()
        assert (o.ntt_radix2(np.zeros(N, np.uint64), q) == 0).all()


def pin_schoolbook_n4096(o):
    rng = random.Random(19)
    q, N = BIG_C1, 1 << 12
    a = _rand_vec(rng, N, q)
    assert (o.ntt_schoolbook(a, q) == o.ntt_radix2(a, q)).all()


def pin_batch_driver(o):
    rng = random.Random(20)
    primes = BIG_218[:2] + [I.prime_chain(3, 1 << 18)[2]]
    N = 1 << 10
    data = np.stack([np.stack([_rand_vec(rng, N, q) for q in primes]) for _ in range(2)])
    for threads in (1, 3):
        fwd = o.ntt_batch(data, primes, +1, threads)
        for b in range(2):
            for l, q in enumerate(primes):
                assert (fwd[b, l] == o.ntt_radix2(data[b, l], q)).all()
        inv = o.ntt_batch(fwd, primes, -1, threads)
        assert (inv == data).all()
    prod = o.pointwise_batch(data, data[::-1].copy(), primes)
    for l, q in enumerate(primes):
        want = [(int(x) * int(y)) % q for x, y in zip(data[0, l], data[1, l])]
        assert list(prod[0, l]) == want


def pin_word32_primes(o):
    """The oracle on the 28-bit primes the 32-bit word path uses (below 2^28,
    q = 1 mod 2N): radix-2 equals the definition at small N, psi is a
    primitive 2N-th root, and the batch driver round-trips at N = 2^12."""
    rng = random.Random(21)
    for N in (8, 64):
        for q in I.prime_chain(2, 2 * N, below=1 << 28):
            a = _rand_vec(rng, N, q)
            A = o.ntt_schoolbook(a, q)
            assert list(o.ntt_radix2(a, q)) == list(A), (q, N)
            assert list(o.intt_radix2(A, q)) == list(a)
            psi = o.psi(q, N)
            assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
    N = 1 << 12
    primes = I.prime_chain(3, 2 * N, below=1 << 28)
    data = np.stack([_rand_vec(rng, N, q) for q in primes])[None]
    fwd = o.ntt_batch(data, primes, +1, 2)
    assert (o.ntt_batch(fwd, primes, -1, 2) == data).all()
    assert (fwd[0, 1] == o.ntt_radix2(data[0, 1], primes[1])).all()


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
