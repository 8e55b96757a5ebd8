"""32-bit word transforms (primes q < 2^28) against the CPU oracle, bit-exact.

The oracle is word-size agnostic (it reduces with exact 128-bit products), so
the same functions that pin the 64-bit path give the expected values here.
"""
import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import oracle_fwd, oracle_inv

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def primes28(N, count):
    """The `count` largest primes below 2^28 with q = 1 mod 2N."""
    return I.prime_chain(count, 2 * N, below=1 << 28)


def dev32(arr):
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    assert int(a.max(initial=0)) < (1 << 32)
    return torch.from_numpy(a.astype(np.uint32).view(np.int32).copy()).cuda()


def host32(t):
    return t.cpu().numpy().view(np.uint32).astype(np.uint64)


def _roundtrip(orc, N, primes, batch, seed, kernel=G.NTT_KERNEL_AUTO, mode=G.NTT_TWIDDLE_AUTO):
    data = I.batch_uniform(seed, batch, primes, N)
    with G.Plan32(N, primes, kernel, mode) as p:
        d = dev32(data)
        p.forward(d, batch)
        torch.cuda.synchronize()
        assert np.array_equal(host32(d), oracle_fwd(orc, data, primes)), f"forward mismatch N={N}"
        p.inverse(d, batch)
        assert np.array_equal(host32(d), data), "inverse(forward(x)) != x"
        y = I.batch_uniform(seed + 1000, batch, primes, N)
        dy = dev32(y)
        p.inverse(dy, batch)
        assert np.array_equal(host32(dy), oracle_inv(orc, y, primes)), "inverse mismatch"
        assert p.device_status() == 0


@pytest.mark.parametrize("n", list(range(1, 18)))
def test_every_size(orc, n):
    N = 1 << n
    _roundtrip(orc, N, primes28(N, 3), 2, 300 + n)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
def test_fused_table_twiddles(orc, n):
    """The fused kernel with the full table instead of OT (the AUTO choice)."""
    N = 1 << n
    _roundtrip(orc, N, primes28(N, 3), 2, 370 + n, G.NTT_KERNEL_FUSED, G.NTT_TWIDDLE_TABLE)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
def test_per_pass_organisation(orc, n):
    """The two-pass sizes also with one launch per pass."""
    N = 1 << n
    _roundtrip(orc, N, primes28(N, 3), 2, 360 + n, G.NTT_KERNEL_PER_PASS)


@pytest.mark.parametrize("n", [12, 13, 14, 15, 16, 17])
def test_several_polynomials_and_limbs(orc, n):
    """Many limbs: tiles of several polynomials and primes in one launch
    (the fused kernel's queues, publication order and work area)."""
    N = 1 << n
    _roundtrip(orc, N, primes28(N, 5), 3, 320 + n)


def test_fused_many_limbs_full_size(orc):
    """The bench's 32-bit workload shape: N = 2^16 with 98 primes (the C2
    modulus size) through the fused kernel."""
    N = 1 << 16
    primes = primes28(N, 98)
    data = I.batch_uniform(350, 1, primes, N)
    with G.Plan32(N, primes) as p:
        d = dev32(data)
        p.forward(d, 1)
        assert np.array_equal(host32(d), oracle_fwd(orc, data, primes))
        p.inverse(d, 1)
        assert np.array_equal(host32(d), data)
        assert p.device_status() == 0


def test_psi_matches_oracle(orc):
    N = 1 << 14
    primes = primes28(N, 4)
    with G.Plan32(N, primes) as p:
        for l, q in enumerate(primes):
            assert G.ntt_plan32_psi(p.handle, l) == orc.psi(q, N)


@pytest.mark.parametrize("n", [4, 12, 13, 17])
def test_extreme_values(orc, n):
    """All residues q - 1 (the largest lazy sums) and all zeros."""
    N = 1 << n
    primes = primes28(N, 2)
    for fill in ("max", "zero"):
        data = np.stack([np.full(N, (q - 1) if fill == "max" else 0, dtype=np.uint64) for q in primes])[None]
        with G.Plan32(N, primes) as p:
            d = dev32(data)
            p.forward(d, 1)
            assert np.array_equal(host32(d), oracle_fwd(orc, data, primes))
            p.inverse(d, 1)
            assert np.array_equal(host32(d), data)


def test_smallest_primes(orc):
    """Primes just above 2N (small q: the lazy bounds are relative to q)."""
    N = 1 << 10
    primes = I.small_ntt_primes(N, 3)
    _roundtrip(orc, N, primes, 2, 340)


def test_more_limbs_than_one_grid(orc):
    """batch * L above the 65535 grid rows of one launch (chunked launches)."""
    N, batch = 4, 70000
    primes = primes28(N, 1)
    data = I.batch_uniform(341, batch, primes, N)
    with G.Plan32(N, primes) as p:
        d = dev32(data)
        p.forward(d, batch)
        assert np.array_equal(host32(d), oracle_fwd(orc, data, primes))


def test_matches_64bit_path_on_common_primes(orc):
    """A prime below 2^28 runs in neither 64-bit plan (q > 2^32 there), so the
    two paths are compared through the negacyclic product they compute: both
    give the schoolbook product mod their own primes."""
    N = 1 << 13
    q = primes28(N, 1)[0]
    a = I.batch_uniform(342, 1, [q], N)[0, 0]
    b = I.batch_uniform(343, 1, [q], N)[0, 0]
    with G.Plan32(N, [q]) as p:
        da, db = dev32(a[None, None]), dev32(b[None, None])
        p.forward(da, 1)
        p.forward(db, 1)
        prod = (host32(da).astype(object) * host32(db).astype(object)) % q
        dc = dev32(np.array(prod, dtype=np.uint64).reshape(1, 1, N))
        p.inverse(dc, 1)
        assert np.array_equal(host32(dc)[0, 0], orc.negacyclic_schoolbook(a, b, q))


def test_rejects_misaligned_and_empty():
    N = 1 << 8
    primes = primes28(N, 1)
    with G.Plan32(N, primes) as p:
        buf = torch.zeros(N + 4, dtype=torch.int32, device="cuda")
        st = G.lib().ntt_forward32(p.handle, buf.data_ptr() + 4, 1, None)
        assert st == G.NTT_ERR_MISALIGNED
        assert G.lib().ntt_forward32(p.handle, buf.data_ptr(), 0, None) == G.NTT_ERR_INVALID_ARG
