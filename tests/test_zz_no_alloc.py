"""ntt_transform_noalloc (fixed device work area, no allocation) against the
plan's own entry points, bit for bit.

Kept in a file of its own, collected last, so that it runs both alone and
after every other GPU test has used the library on the same device.
"""
import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import dev, host

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu

FWD, INV = G.NTT_OP_FORWARD, G.NTT_OP_INVERSE


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def _two_calls_in_a_row(p, data, batch, levels):
    """Forward then inverse through the no-allocation call, each compared with
    ntt_forward_levels / ntt_inverse_levels on the same input."""
    want = dev(data)
    got = dev(data)
    G.ntt_forward_levels(p.handle, want, batch, levels)
    G.ntt_transform_noalloc(p.handle, got, batch, levels, FWD)
    torch.cuda.synchronize()
    assert torch.equal(got, want), "first call (forward) differs"
    G.ntt_inverse_levels(p.handle, want, batch, levels)
    G.ntt_transform_noalloc(p.handle, got, batch, levels, INV)
    torch.cuda.synchronize()
    assert torch.equal(got, want), "second call (inverse) differs"
    assert np.array_equal(host(got), data)
    assert p.device_status() == 0


@pytest.mark.parametrize("mode,ots", [(G.NTT_TWIDDLE_TABLE, 0), (G.NTT_TWIDDLE_OT, 1)])
def test_n65536_45_primes(mode, ots):
    w = I.workload_c2()
    data = I.batch_uniform(w.seed, 1, w.primes, w.N)
    with G.Plan(w.N, w.primes, mode, ots) as p:
        _two_calls_in_a_row(p, data, 1, len(w.primes))


@pytest.mark.parametrize("n,L,batch,levels,kernel", [
    (12, 3, 3, 3, G.NTT_KERNEL_AUTO),          # one pass: no scratch used
    (14, 4, 5, 4, G.NTT_KERNEL_PER_PASS),      # launch per pass: no scratch used
    (13, 2, 7, 2, G.NTT_KERNEL_FUSED),
    (17, 8, 2, 5, G.NTT_KERNEL_FUSED),         # a level below the plan's L
])
def test_sizes_and_kernels(n, L, batch, levels, kernel):
    N = 1 << n
    primes = I.prime_chain(L, 2 * N)
    data = I.batch_uniform(60 + n, batch, primes[:levels], N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_AUTO, 0, kernel) as p:
        _two_calls_in_a_row(p, data, batch, levels)


def test_back_to_back_without_sync():
    """Calls queued back to back on one stream: each launch must leave the
    shared work area at zero for the next, whatever its limb count."""
    N = 1 << 15
    primes = I.prime_chain(6, 2 * N)
    xs = [I.batch_uniform(80 + i, b, primes, N) for i, b in enumerate((3, 1, 2))]
    with G.Plan(N, primes) as p:
        want = [dev(x) for x in xs]
        got = [dev(x) for x in xs]
        for x, d in zip(xs, want):
            G.ntt_forward(p.handle, d, x.shape[0])
        for x, d in zip(xs, got):
            G.ntt_transform_noalloc(p.handle, d, x.shape[0], len(primes), FWD)
        torch.cuda.synchronize()
        for a, b in zip(got, want):
            assert torch.equal(a, b)
        assert p.device_status() == 0


def test_maximum_and_over_limit():
    """Exactly NTT_NOALLOC_MAX_LIMBS limbs run; one more is refused with
    NTT_ERR_LIMIT before anything is enqueued (the buffer is large enough
    either way)."""
    N = 1 << 13
    primes = I.prime_chain(1, 2 * N)
    M = G.NTT_NOALLOC_MAX_LIMBS
    gen = torch.Generator(device="cuda").manual_seed(5)
    q = int(primes[0])
    base = torch.randint(0, q, (M + 1, 1, N), dtype=torch.int64, device="cuda", generator=gen)
    with G.Plan(N, primes) as p:
        got = base.clone()
        with pytest.raises(G.NttError) as ei:
            G.ntt_transform_noalloc(p.handle, got, M + 1, 1, FWD)
        assert ei.value.status == G.NTT_ERR_LIMIT
        torch.cuda.synchronize()
        assert torch.equal(got, base)
        want = base.clone()
        G.ntt_forward(p.handle, want, M)
        G.ntt_transform_noalloc(p.handle, got, M, 1, FWD)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert p.device_status() == 0


def test_argument_errors():
    N = 1 << 13
    primes = I.prime_chain(2, 2 * N)
    buf = torch.zeros(2 * N + 2, dtype=torch.int64, device="cuda")
    lib = G.lib()
    with G.Plan(N, primes) as p:
        h = p.handle
        assert lib.ntt_transform_noalloc(h, buf.data_ptr(), 1, 2, FWD | INV, None) == G.NTT_ERR_INVALID_ARG
        assert lib.ntt_transform_noalloc(h, buf.data_ptr(), 1, 3, FWD, None) == G.NTT_ERR_INVALID_ARG
        assert lib.ntt_transform_noalloc(h, buf.data_ptr(), 0, 2, FWD, None) == G.NTT_ERR_INVALID_ARG
        assert lib.ntt_transform_noalloc(h, buf.data_ptr() + 8, 1, 2, FWD, None) == G.NTT_ERR_MISALIGNED
        assert lib.ntt_transform_noalloc(None, buf.data_ptr(), 1, 2, FWD, None) == G.NTT_ERR_INVALID_ARG
