"""Pass geometries (radix split, row tile) and the autotuner, on the GPU.

Every compiled geometry of every two-pass size, in both kernel organisations
and every twiddle supply, against the oracle bit for bit; uneven batches whose
jobs mix geometries; the product with a non-default geometry; and the
autotuner's report and choice.
"""
import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import dev, host, oracle_fwd, oracle_inv

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu

# (p1, log2 rows per row tile) of geometries 0, 1, 2 for n = 13 .. 17
GEOMETRY = {13: [(6, 5), (6, 4), (7, 6)], 14: [(7, 5), (7, 4), (6, 4)], 15: [(7, 4), (7, 3), (8, 5)],
            16: [(8, 4), (8, 3), (7, 3)], 17: [(8, 3), (8, 2), (7, 2)]}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("geometry", [1, 2])
@pytest.mark.parametrize("kernel", [G.NTT_KERNEL_FUSED, G.NTT_KERNEL_PER_PASS])
def test_geometry_matches_oracle(orc, n, geometry, kernel):
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    data = I.batch_uniform(400 + n, 2, primes, N)
    y = I.batch_uniform(450 + n, 2, primes, N)
    want_f = oracle_fwd(orc, data, primes)
    want_i = oracle_inv(orc, y, primes)
    for mode, ots in ((G.NTT_TWIDDLE_TABLE, 0), (G.NTT_TWIDDLE_OT, 1), (G.NTT_TWIDDLE_OT, 2)):
        with G.Plan(N, primes, mode, ots, kernel, geometry) as p:
            info = p.info()
            assert (info.pass1_log2, info.row_tile_log2, info.geometry) == (*GEOMETRY[n][geometry], geometry)
            d = dev(data)
            p.forward(d, 2)
            assert np.array_equal(host(d), want_f), f"forward n={n} g={geometry} k={kernel} ots={ots}"
            p.inverse(d, 2)
            assert np.array_equal(host(d), data), "inverse(forward(x)) != x"
            dy = dev(y)
            p.inverse(dy, 2)
            assert np.array_equal(host(dy), want_i), "inverse mismatch"
            assert p.device_status() == 0


def test_default_geometry_reported():
    for n in range(13, 18):
        with G.Plan(1 << n, I.prime_chain(1, 2 << n)) as p:
            info = p.info()
            assert (info.pass1_log2, info.row_tile_log2, info.geometry) == (*GEOMETRY[n][0], 0)


def test_batch_mixes_geometries(orc):
    """Jobs of one size with different geometries go to different launches;
    every result is the oracle's."""
    N = 1 << 15
    primes = I.prime_chain(6, 2 * N)
    plans = [G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED, g) for g in range(3)]
    try:
        jobs, want, bufs = [], [], []
        for j in range(9):
            g, op = j % 3, (G.NTT_OP_FORWARD if j % 2 == 0 else G.NTT_OP_INVERSE)
            levels = 1 + j % 6
            x = I.batch_uniform(470 + j, 1, primes[:levels], N)
            d = dev(x)
            bufs.append(d)
            jobs.append((plans[g].handle, d, 1, levels, op))
            want.append((oracle_fwd if op == G.NTT_OP_FORWARD else oracle_inv)(orc, x, primes[:levels]))
        with G.Batch() as b:
            b.submit(jobs)
            torch.cuda.synchronize()
            assert b.device_status() == 0
        for d, w in zip(bufs, want):
            assert np.array_equal(host(d), w)
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("geometry", [1, 2])
def test_product_with_geometry(orc, geometry):
    N = 1 << 13
    primes = I.prime_chain(2, 2 * N)
    a = I.batch_uniform(480, 1, primes, N)
    b = I.batch_uniform(481, 1, primes, N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED, geometry) as p:
        da, db = dev(a), dev(b)
        dc = torch.empty_like(da)
        G.ntt_mul_negacyclic(p.handle, da, db, dc, 1)
        got = host(dc)
    for l, q in enumerate(primes):
        assert np.array_equal(got[0, l], orc.negacyclic_schoolbook(a[0, l], b[0, l], q))


@pytest.mark.parametrize("n,L,batch", [(10, 2, 3), (14, 4, 2)])
def test_autotune_reports_and_picks_the_fastest(orc, n, L, batch):
    N = 1 << n
    primes = I.prime_chain(L, 2 * N)
    best, entries = G.ntt_autotune(N, primes, batch, reps=3)
    # one-pass sizes: one-pass, radix-2, high radix (and the cluster kernel
    # for 2^10 .. 2^12); two-pass sizes: 3 geometries x 6 + radix-2 + high radix
    assert len(entries) == ((4 if n >= 10 else 3) if n <= 12 else 20)
    assert all(e.status == G.NTT_OK and e.forward_us > 0 and e.inverse_us > 0 for e in entries)
    tot = [e.forward_us + e.inverse_us for e in entries]
    k = int(np.argmin(tot))
    e = entries[k].opts
    assert (best.kernel, best.twiddle_mode, best.ot_stages, best.geometry) == \
        (e.kernel, e.twiddle_mode, e.ot_stages, e.geometry)
    # the cached choice, without timing
    again, none = G.ntt_autotune(N, primes, batch, entries=False)
    assert none == [] and bytes(again) == bytes(best)
    # the chosen configuration is exact
    data = I.batch_uniform(490 + n, batch, primes, N)
    with G.Plan.from_opts(N, primes, best) as p:
        d = dev(data)
        p.forward(d, batch)
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
        p.inverse(d, batch)
        assert np.array_equal(host(d), data)


@pytest.mark.parametrize("n,kernel", [(12, G.NTT_KERNEL_AUTO), (16, G.NTT_KERNEL_FUSED), (16, G.NTT_KERNEL_PER_PASS)])
def test_l2_resident_twiddles_same_results(orc, n, kernel):
    """NTT_PLAN_L2_TWIDDLES changes only the cache policy of the launches."""
    N = 1 << n
    primes = I.prime_chain(4, 2 * N)
    data = I.batch_uniform(495 + n, 2, primes, N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_AUTO, 0, kernel, 0, G.NTT_PLAN_L2_TWIDDLES) as p:
        d = dev(data)
        p.forward(d, 2)
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
        p.inverse(d, 2)
        assert np.array_equal(host(d), data)


def test_config3_full_size_with_tuned_choice(orc):
    """The large ring (N = 2^17, 60 limbs, one ciphertext) with the
    configuration the bench's autotuner picks there (fused, table, half the row
    tile), against the oracle in full."""
    w = I.workload_c3()
    N, primes = w.N, w.primes
    data = I.batch_uniform(w.seed, 2, primes, N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED, G.NTT_GEOMETRY_SMALL_ROW_TILE) as p:
        d = dev(data)
        p.forward(d, 2)
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
        p.inverse(d, 2)
        assert np.array_equal(host(d), data)
        assert p.device_status() == 0


@pytest.mark.parametrize("geometry", [1, 2])
def test_host_call_and_noalloc_with_geometry(orc, geometry):
    """The host-buffer call (segments viewing the tables from a prime offset)
    and the no-allocation call under the alternative geometries."""
    N = 1 << 15
    primes = I.prime_chain(7, 2 * N)
    data = I.batch_uniform(497, 2, primes, N)
    want = oracle_fwd(orc, data, primes)
    with G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED, geometry) as p:
        out = np.empty_like(data)
        G.ntt_execute_host(p.handle, data, out, 2, G.NTT_OP_FORWARD)
        assert np.array_equal(out, want)
        d = dev(data)
        G.ntt_transform_noalloc(p.handle, d, 2, len(primes), G.NTT_OP_FORWARD)
        assert np.array_equal(host(d), want)
        G.ntt_transform_noalloc(p.handle, d, 2, len(primes), G.NTT_OP_INVERSE)
        assert np.array_equal(host(d), data)
