"""CPU oracle for the negacyclic RNS NTT -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python binding
never import it, and it imports nothing from them.

Thin ctypes binding over ``ntt_oracle.c`` (plain C, unsigned __int128
products).  Functions, with the paper passage each follows (Kim, Jung, Park,
Ahn, "Accelerating Number Theoretic Transformations for Bootstrappable
Homomorphic Encryption on GPUs"):

* ``ntt_schoolbook`` / ``intt_schoolbook`` -- the definition of Sec. III-A
  (A_k = sum_n a_n psi^{n(2k+1)}), outputs listed in bit-reversed order as
  Algorithm 1 produces them.
* ``ntt_radix2`` / ``intt_radix2`` -- Algorithm 1 (Cooley-Tukey with the
  Psi[i] = psi^{brv(i)} table of Sec. III-C) and its Gentleman-Sande inverse
  with the Psi^{-1} twist merged in (Sec. III-A).
* ``negacyclic_schoolbook`` -- the c_k formula of Sec. III-A.
* ``psi`` -- g^{(q-1)/2N} with g the smallest generator of Z_q^*.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntt_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

u64 = ctypes.c_uint64
u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def _bind(L):
    L.orc_powmod.restype = u64
    L.orc_powmod.argtypes = [u64, u64, u64]
    L.orc_invmod.restype = u64
    L.orc_invmod.argtypes = [u64, u64]
    L.orc_is_prime.restype = ctypes.c_int
    L.orc_is_prime.argtypes = [u64]
    L.orc_prime_factors.restype = ctypes.c_int
    L.orc_prime_factors.argtypes = [u64, u64p, ctypes.c_int]
    L.orc_smallest_generator.restype = u64
    L.orc_smallest_generator.argtypes = [u64]
    L.orc_psi.restype = u64
    L.orc_psi.argtypes = [u64, u64]
    L.orc_bitrev.restype = u64
    L.orc_bitrev.argtypes = [u64, ctypes.c_int]
    for f in ("orc_ntt_schoolbook", "orc_intt_schoolbook"):
        getattr(L, f).restype = None
        getattr(L, f).argtypes = [u64p, u64p, u64, u64, u64]
    L.orc_negacyclic_schoolbook.restype = None
    L.orc_negacyclic_schoolbook.argtypes = [u64p, u64p, u64p, u64, u64]
    L.orc_eval.restype = u64
    L.orc_eval.argtypes = [u64p, u64, u64, u64]
    for f in ("orc_ntt_radix2", "orc_intt_radix2"):
        getattr(L, f).restype = ctypes.c_int
        getattr(L, f).argtypes = [u64p, u64, u64, u64]
    L.orc_pointwise.restype = None
    L.orc_pointwise.argtypes = [u64p, u64p, u64p, u64, u64]
    L.orc_ntt_batch.restype = ctypes.c_int
    L.orc_ntt_batch.argtypes = [u64p, u64, u64p, u64, u64, ctypes.c_int, ctypes.c_int]
    L.orc_pointwise_batch.restype = None
    L.orc_pointwise_batch.argtypes = [u64p, u64p, u64p, u64, u64p, u64, u64]
    return Oracle(L)


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(u64p)


def _arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint64))


class Oracle:
    """Python view of one loaded oracle library (see the module docstring)."""

    def __init__(self, L):
        self.L = L

    # number theory ---------------------------------------------------
    def powmod(self, b, e, q):
        return int(self.L.orc_powmod(b, e, q))

    def invmod(self, a, q):
        return int(self.L.orc_invmod(a, q))

    def is_prime(self, n):
        return bool(self.L.orc_is_prime(n))

    def prime_factors(self, m):
        buf = np.zeros(64, dtype=np.uint64)
        k = self.L.orc_prime_factors(m, _ptr(buf), 64)
        return sorted(int(x) for x in buf[:min(k, 64)])

    def smallest_generator(self, q):
        return int(self.L.orc_smallest_generator(q))

    def psi(self, q, N):
        return int(self.L.orc_psi(q, N))

    def bitrev(self, i, nbits):
        return int(self.L.orc_bitrev(i, nbits))

    # single-limb transforms -----------------------------------------
    def ntt_schoolbook(self, a, q, psi=None):
        a = _arr(a)
        N = a.size
        out = np.zeros(N, dtype=np.uint64)
        self.L.orc_ntt_schoolbook(_ptr(a), _ptr(out), N, q, psi or self.psi(q, N))
        return out

    def intt_schoolbook(self, A, q, psi=None):
        A = _arr(A)
        N = A.size
        out = np.zeros(N, dtype=np.uint64)
        self.L.orc_intt_schoolbook(_ptr(A), _ptr(out), N, q, psi or self.psi(q, N))
        return out

    def ntt_radix2(self, a, q, psi=None):
        a = _arr(a).copy()
        if self.L.orc_ntt_radix2(_ptr(a), a.size, q, psi or self.psi(q, a.size)):
            raise MemoryError
        return a

    def intt_radix2(self, A, q, psi=None):
        A = _arr(A).copy()
        if self.L.orc_intt_radix2(_ptr(A), A.size, q, psi or self.psi(q, A.size)):
            raise MemoryError
        return A

    def negacyclic_schoolbook(self, a, b, q):
        a, b = _arr(a), _arr(b)
        c = np.zeros(a.size, dtype=np.uint64)
        self.L.orc_negacyclic_schoolbook(_ptr(a), _ptr(b), _ptr(c), a.size, q)
        return c

    def eval(self, a, x, q):
        a = _arr(a)
        return int(self.L.orc_eval(_ptr(a), a.size, x, q))

    def pointwise(self, a, b, q):
        a, b = _arr(a), _arr(b)
        c = np.zeros(a.size, dtype=np.uint64)
        self.L.orc_pointwise(_ptr(a), _ptr(b), _ptr(c), a.size, q)
        return c

    # batched ([batch][L][N]) -------------------------------------------
    def ntt_batch(self, data, primes, dir: int, threads: int = 1):
        """Transform a copy of data[batch][L][N] (dir +1 forward, -1 inverse)."""
        d = np.array(data, dtype=np.uint64, order="C", copy=True)
        if d.ndim == 2:
            d = d[None]
        B, L, N = d.shape
        pr = _arr(primes)
        assert pr.size == L
        rc = self.L.orc_ntt_batch(_ptr(d), N, _ptr(pr), L, B, int(dir), int(threads))
        if rc == -1:
            raise ValueError("bad prime for this N")
        if rc:
            raise MemoryError
        return d.reshape(np.shape(data))

    def pointwise_batch(self, a, b, primes):
        a, b = _arr(a), _arr(b)
        shp = a.shape
        a3 = a.reshape(-1, len(primes), shp[-1])
        b3 = b.reshape(a3.shape)
        c = np.zeros_like(a3)
        pr = _arr(primes)
        self.L.orc_pointwise_batch(_ptr(a3), _ptr(b3), _ptr(c), a3.shape[2], _ptr(pr),
                                   a3.shape[1], a3.shape[0])
        return c.reshape(shp)


def get() -> Oracle:
    return lib()
