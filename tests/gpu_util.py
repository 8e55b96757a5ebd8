"""Helpers for the GPU tests: device buffers via torch, oracle calls."""
import os

import numpy as np

THREADS = max(1, min(32, os.cpu_count() or 1))


def dev(arr):
    import torch
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint64)


def oracle_fwd(orc, data, primes):
    return orc.ntt_batch(data, primes, +1, THREADS)


def oracle_inv(orc, data, primes):
    return orc.ntt_batch(data, primes, -1, THREADS)
