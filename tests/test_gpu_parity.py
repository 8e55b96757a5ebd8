"""CUDA path against the CPU oracle, element by element (bit-exact).

Every call goes through the C ABI (ctypes binding); inputs are the seeded
synthetic workloads of ntt_inputs.  Integer results: the bar is equality.
"""
import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import dev, host, oracle_fwd, oracle_inv

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def _roundtrip_case(orc, N, primes, batch, seed, mode=G.NTT_TWIDDLE_TABLE, ots=0, kernel=G.NTT_KERNEL_AUTO):
    data = I.batch_uniform(seed, batch, primes, N)
    with G.Plan(N, primes, mode, ots, kernel) as p:
        d = dev(data)
        p.forward(d, batch)
        torch.cuda.synchronize()
        got = host(d)
        want = oracle_fwd(orc, data, primes)
        assert np.array_equal(got, want), f"forward mismatch N={N} mode={mode} ots={ots}"
        p.inverse(d, batch)
        assert np.array_equal(host(d), data), "inverse(forward(x)) != x"
        # inverse on input not produced by the forward (arbitrary NTT-domain data)
        y = I.batch_uniform(seed + 1000, batch, primes, N)
        dy = dev(y)
        p.inverse(dy, batch)
        assert np.array_equal(host(dy), oracle_inv(orc, y, primes)), "inverse mismatch"
    return got


def test_config1_n4096_single_limb(orc):
    w = I.workload_c1()
    _roundtrip_case(orc, w.N, w.primes, w.batch, w.seed)


@pytest.mark.parametrize("n", list(range(1, 18)))
def test_every_size_table_mode(orc, n):
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    _roundtrip_case(orc, N, primes, 2, 40 + n)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("ots", [1, 2])
def test_ot_equals_table_and_oracle(orc, n, ots):
    N = 1 << n
    primes = I.prime_chain(2, 2 * N)
    a = _roundtrip_case(orc, N, primes, 1, 70 + n, G.NTT_TWIDDLE_OT, ots)
    b = _roundtrip_case(orc, N, primes, 1, 70 + n, G.NTT_TWIDDLE_TABLE)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,ots", [(G.NTT_TWIDDLE_TABLE, 0), (G.NTT_TWIDDLE_OT, 1), (G.NTT_TWIDDLE_OT, 2)])
def test_config2_full_size(orc, mode, ots):
    w = I.workload_c2()
    _roundtrip_case(orc, w.N, w.primes, w.batch, w.seed, mode, ots)


def test_config3_full_size_and_product(orc):
    w = I.workload_c3()
    N, primes = w.N, w.primes
    data = I.batch_uniform(w.seed, 2, primes, N)              # one ciphertext
    with G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1) as p:
        d = dev(data)
        p.forward(d, 2)
        torch.cuda.synchronize()
        fwd = host(d)
        assert np.array_equal(fwd, oracle_fwd(orc, data, primes))
        p.inverse(d, 2)
        assert np.array_equal(host(d), data)
        # negacyclic product of two more polynomials: NTT, pointwise, iNTT
        a = I.poly_uniform(w.seed, 2, primes, N)[None]
        b = I.poly_uniform(w.seed, 3, primes, N)[None]
        da, db = dev(a), dev(b)
        p.forward(da, 1)
        p.forward(db, 1)
        G.ntt_mul_pointwise(p.handle, da, db, da, 1)
        p.inverse(da, 1)
        torch.cuda.synchronize()
        c = host(da)
        # the same product in one call, in place (fused element-wise step)
        da, db = dev(a), dev(b)
        G.ntt_mul_negacyclic(p.handle, da, db, da, 1)
        torch.cuda.synchronize()
        c_in_place = host(da)
        assert p.device_status() == 0
    A = oracle_fwd(orc, a, primes)
    B = oracle_fwd(orc, b, primes)
    want = oracle_inv(orc, orc.pointwise_batch(A, B, primes), primes)
    assert np.array_equal(c, want)
    assert np.array_equal(c_in_place, want)
    # sampled outputs checked one by one: c(x) = a(x) b(x) at roots of X^N + 1
    rng = np.random.default_rng(3)
    for l in rng.choice(len(primes), 3, replace=False):
        q = primes[l]
        psi = orc.psi(q, N)
        for k in rng.choice(N, 2, replace=False):
            x = pow(psi, 2 * int(k) + 1, q)
            lhs = orc.eval(c[0, l], x, q)
            rhs = orc.eval(a[0, l], x, q) * orc.eval(b[0, l], x, q) % q
            assert lhs == rhs


def test_edge_values(orc):
    N = 1 << 14
    primes = I.prime_chain(3, 2 * N)
    q = np.array(primes, dtype=np.uint64)[:, None]
    cases = [np.zeros((3, N), np.uint64), np.broadcast_to(q - np.uint64(1), (3, N)).copy()]
    one = np.zeros((3, N), np.uint64)
    one[:, 0] = 1
    cases.append(one)
    spike = np.zeros((3, N), np.uint64)
    spike[:, N - 1] = (q[:, 0] - np.uint64(1))
    cases.append(spike)
    with G.Plan(N, primes) as p:
        for data in cases:
            d = dev(data[None])
            p.forward(d, 1)
            torch.cuda.synchronize()
            assert np.array_equal(host(d)[0], oracle_fwd(orc, data[None], primes)[0])
            d2 = dev(data[None])
            p.inverse(d2, 1)
            assert np.array_equal(host(d2)[0], oracle_inv(orc, data[None], primes)[0])


def test_many_limbs_grid_chunking(orc):
    """batch * L above the 65535 grid-y limit is split into several launches."""
    N = 1 << 4
    primes = I.prime_chain(2, 2 * N)
    batch = 33000                                   # 66000 limbs
    data = I.batch_uniform(5, 4, primes, N)
    data = np.tile(data, (batch // 4 + 1, 1, 1))[:batch]
    with G.Plan(N, primes) as p:
        d = dev(data)
        p.forward(d, batch)
        torch.cuda.synchronize()
        got = host(d)
    want = oracle_fwd(orc, data[:4], primes)
    assert np.array_equal(got[-4:], oracle_fwd(orc, data[-4:], primes))
    assert np.array_equal(got[:4], want)


def test_levels_api(orc):
    N = 1 << 15
    primes = I.prime_chain(6, 2 * N)
    data = I.batch_uniform(8, 2, primes[:4], N)
    with G.Plan(N, primes) as p:
        d = dev(data)
        G.ntt_forward_levels(p.handle, d, 2, 4)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes[:4]))
        G.ntt_inverse_levels(p.handle, d, 2, 4)
        assert np.array_equal(host(d), data)
        with pytest.raises(G.NttError):
            G.ntt_forward_levels(p.handle, d, 2, 7)


def test_misaligned_pointer_rejected():
    N = 1 << 12
    primes = I.prime_chain(1, 2 * N)
    buf = torch.zeros(N + 2, dtype=torch.int64, device="cuda")
    with G.Plan(N, primes) as p:
        st = G.lib().ntt_forward(p.handle, buf.data_ptr() + 8, 1, None)
        assert st == G.NTT_ERR_MISALIGNED
        assert G.lib().ntt_forward(p.handle, buf.data_ptr(), 0, None) == G.NTT_ERR_INVALID_ARG


def test_nondefault_stream_and_pointwise(orc):
    N = 1 << 16
    primes = I.prime_chain(4, 2 * N)
    a = I.batch_uniform(9, 1, primes, N)
    b = I.batch_uniform(10, 1, primes, N)
    s = torch.cuda.Stream()
    with G.Plan(N, primes) as p:
        with torch.cuda.stream(s):
            da, db = dev(a), dev(b)
            dc = torch.empty_like(da)
            G.ntt_mul_pointwise(p.handle, da, db, dc, 1, s)
            p.forward(dc, 1, s)
        s.synchronize()
        got = host(dc)
    want = oracle_fwd(orc, orc.pointwise_batch(a, b, primes), primes)
    assert np.array_equal(got, want)


def test_execute_host_roundtrip(orc):
    w = I.workload_c2()
    primes = w.primes[:5]
    data = I.batch_uniform(w.seed, 1, primes, w.N)
    with G.Plan(w.N, primes) as p:
        out = np.empty_like(data)
        G.ntt_execute_host(p.handle, data, out, 1, G.NTT_OP_FORWARD)
        assert np.array_equal(out, oracle_fwd(orc, data, primes))
        back = np.empty_like(data)
        G.ntt_execute_host(p.handle, out, back, 1, G.NTT_OP_INVERSE)
        assert np.array_equal(back, data)
        both = np.empty_like(data)
        G.ntt_execute_host(p.handle, data, both, 1, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE)
        assert np.array_equal(both, data)


def test_execute_host_async_chains(orc):
    """Asynchronous host-buffer calls overlap on one plan: several independent
    calls in flight, then an in-place forward followed by an in-place inverse
    on the same buffer; every result is the oracle's."""
    w = I.workload_c2()
    primes = w.primes[:7]
    datas = [I.batch_uniform(w.seed + k, 2, primes, w.N) for k in range(3)]
    s = torch.cuda.Stream()
    with G.Plan(w.N, primes) as p:
        ins = [torch.from_numpy(d.view(np.int64).copy()).pin_memory() for d in datas]
        outs = [torch.empty_like(x).pin_memory() for x in ins]
        alt = [torch.cuda.Stream(), torch.cuda.Stream()]
        for k, (x, y) in enumerate(zip(ins, outs)):
            G.ntt_execute_host_async(p.handle, x, y, 2, G.NTT_OP_FORWARD, alt[k % 2])    # calls overlap
        torch.cuda.synchronize()
        for d, y in zip(datas, outs):
            assert np.array_equal(y.numpy().view(np.uint64), oracle_fwd(orc, d, primes))
        buf = ins[0]
        G.ntt_execute_host_async(p.handle, buf, buf, 2, G.NTT_OP_FORWARD, s)
        G.ntt_execute_host_async(p.handle, buf, buf, 2, G.NTT_OP_INVERSE, s)
        s.synchronize()
        assert np.array_equal(buf.numpy().view(np.uint64), datas[0])
        # another batch size: other segments, each waiting on the overlapping ones of the previous call
        G.ntt_execute_host_async(p.handle, ins[1][:1], outs[1][:1], 1, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE, s)
        s.synchronize()
        assert np.array_equal(outs[1][:1].numpy().view(np.uint64), datas[1][:1])


def test_plan_query_and_psi(orc):
    w = I.workload_c2()
    with G.Plan(w.N, w.primes[:3], G.NTT_TWIDDLE_OT, 2) as p:
        info = p.info()
        assert (info.N, info.L, info.log2_N, info.passes) == (w.N, 3, 16, 2)
        assert info.twiddle_mode == G.NTT_TWIDDLE_OT and info.ot_stages == 2
        for l in range(3):
            assert G.ntt_plan_psi(p.handle, l) == orc.psi(w.primes[l], w.N)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("mode,ots", [(G.NTT_TWIDDLE_TABLE, 0), (G.NTT_TWIDDLE_OT, 1)])
def test_fused_equals_per_pass(orc, n, mode, ots):
    """The one-launch fused kernel and the launch-per-pass kernels agree, and
    no bounded wait of the fused kernel ran out."""
    N = 1 << n
    primes = I.prime_chain(5, 2 * N)
    data = I.batch_uniform(90 + n, 3, primes, N)               # 15 limbs
    outs = []
    for kernel in (G.NTT_KERNEL_FUSED, G.NTT_KERNEL_PER_PASS):
        with G.Plan(N, primes, mode, ots, kernel) as p:
            d = dev(data)
            p.forward(d, 3)
            torch.cuda.synchronize()
            f = host(d)
            p.inverse(d, 3)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), data)
            assert p.device_status() == 0
            outs.append(f)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], oracle_fwd(orc, data, primes))


def test_fused_many_limbs_and_single_limb(orc):
    """Lag larger than the limb count (1 limb) and many limbs (400): every
    polynomial's forward result against the oracle, then the round trip."""
    N = 1 << 14
    primes = I.prime_chain(4, 2 * N)
    for batch, L in ((1, 1), (100, 4)):
        data = I.batch_uniform(7, batch, primes[:L], N)
        with G.Plan(N, primes[:L]) as p:
            d = dev(data)
            p.forward(d, batch)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), oracle_fwd(orc, data, primes[:L]))
            p.inverse(d, batch)
            torch.cuda.synchronize()
            assert np.array_equal(host(d), data)
            assert p.device_status() == 0


@pytest.mark.parametrize("n", [13, 16, 17])
def test_chained_launches_without_sync(orc, n):
    """Dependent transforms queued back to back on one stream: forward /
    inverse chains on one buffer, alternating between two plans (two work
    areas), with no host synchronisation."""
    N = 1 << n
    primes = I.prime_chain(6, 2 * N)
    data = I.batch_uniform(110 + n, 1, primes, N)
    with G.Plan(N, primes) as p, G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1) as p2:
        d = dev(data)
        for _ in range(10):
            p.forward(d, 1)
            p2.inverse(d, 1)
            p2.forward(d, 1)
            p.inverse(d, 1)
        p.forward(d, 1)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
        assert p.device_status() == 0 and p2.device_status() == 0


@pytest.mark.parametrize("n,want_mode,want_ots", [(12, G.NTT_TWIDDLE_TABLE, 0), (13, G.NTT_TWIDDLE_OT, 1),
                                                  (16, G.NTT_TWIDDLE_OT, 1), (17, G.NTT_TWIDDLE_OT, 1)])
def test_auto_twiddle_mode(n, want_mode, want_ots):
    N = 1 << n
    with G.Plan(N, I.prime_chain(1, 2 * N)) as p:
        info = p.info()
        assert (info.twiddle_mode, info.ot_stages) == (want_mode, want_ots)


@pytest.mark.parametrize("n,L,batch,kernel,mode,ots", [
    (16, 45, 1, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0),         # limb ranges of one polynomial
    (17, 4, 3, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_OT, 2),            # ranges of several polynomials, OT2 views
    (14, 7, 2, G.NTT_KERNEL_PER_PASS, G.NTT_TWIDDLE_TABLE, 0),     # launch-per-pass kernels
    (12, 3, 7, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0),          # groups of whole polynomials, one pass
    (13, 5, 13, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_OT, 1),           # groups, fused
    (13, 6, 4, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0),          # one segment per polynomial
    (15, 2, 5, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0),
])
def test_execute_host_segments(orc, n, L, batch, kernel, mode, ots):
    """The host-buffer call splits the data into segments on several streams;
    every shape of split matches the oracle, in place and out of place."""
    N = 1 << n
    primes = I.prime_chain(L, 2 * N)
    data = I.batch_uniform(130 + n, batch, primes, N)
    with G.Plan(N, primes, mode, ots, kernel) as p:
        out = np.empty_like(data)
        G.ntt_execute_host(p.handle, data, out, batch, G.NTT_OP_FORWARD)
        assert np.array_equal(out, oracle_fwd(orc, data, primes))
        G.ntt_execute_host(p.handle, out, out, batch, G.NTT_OP_INVERSE)     # in place
        assert np.array_equal(out, data)
        both = np.empty_like(data)
        G.ntt_execute_host(p.handle, data, both, batch, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE)
        assert np.array_equal(both, data)
        assert p.device_status() == 0


@pytest.mark.parametrize("n,kernel,mode,ots", [(10, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0),
                                               (14, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_OT, 2),
                                               (16, G.NTT_KERNEL_PER_PASS, G.NTT_TWIDDLE_TABLE, 0),
                                               (17, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_AUTO, 0)])
def test_mul_negacyclic(orc, n, kernel, mode, ots):
    """c = a * b mod (X^N + 1): against the schoolbook product (small N) or the
    oracle's transforms; a and b keep their forward transforms; c may alias a."""
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    a = I.batch_uniform(150 + n, 2, primes, N)
    b = I.batch_uniform(160 + n, 2, primes, N)
    A = oracle_fwd(orc, a, primes)
    B = oracle_fwd(orc, b, primes)
    if n <= 10:
        want = np.stack([np.stack([orc.negacyclic_schoolbook(a[k, l], b[k, l], primes[l]) for l in range(3)])
                         for k in range(2)])
    else:
        want = oracle_inv(orc, orc.pointwise_batch(A, B, primes), primes)
    with G.Plan(N, primes, mode, ots, kernel) as p:
        da, db, dc = dev(a), dev(b), torch.empty(a.shape, dtype=torch.int64, device="cuda")
        G.ntt_mul_negacyclic(p.handle, da, db, dc, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(dc), want)
        assert np.array_equal(host(da), A) and np.array_equal(host(db), B)
        da, db = dev(a), dev(b)
        G.ntt_mul_negacyclic(p.handle, da, db, da, 2)                      # c aliases a
        torch.cuda.synchronize()
        assert np.array_equal(host(da), want)
        assert np.array_equal(host(db), B)
        da, db = dev(a), dev(b)
        G.ntt_mul_negacyclic(p.handle, da, db, db, 2)                      # c aliases b
        torch.cuda.synchronize()
        assert np.array_equal(host(db), want)
        assert np.array_equal(host(da), A)
        assert p.device_status() == 0


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("geometry,ots", [(0, 1), (1, 0), (2, 2)])
def test_fused_product_in_place(orc, n, geometry, ots):
    """The in-place product of fused plans (the inverse's first pass multiplies
    each tile by the other factor) for every geometry, both twiddle supplies and
    both aliasings, against the oracle's transforms; several polynomials so that
    tiles of different limbs and primes meet in one launch."""
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    a = I.batch_uniform(170 + n, 3, primes, N)
    b = I.batch_uniform(180 + n, 3, primes, N)
    A = oracle_fwd(orc, a, primes)
    B = oracle_fwd(orc, b, primes)
    want = oracle_inv(orc, orc.pointwise_batch(A, B, primes), primes)
    mode = G.NTT_TWIDDLE_OT if ots else G.NTT_TWIDDLE_TABLE
    with G.Plan(N, primes, mode, ots, G.NTT_KERNEL_FUSED, geometry) as p:
        for alias_a in (True, False):
            da, db = dev(a), dev(b)
            G.ntt_mul_negacyclic(p.handle, da, db, da if alias_a else db, 3)
            torch.cuda.synchronize()
            assert np.array_equal(host(da if alias_a else db), want), f"n={n} g={geometry} ots={ots} a={alias_a}"
            assert np.array_equal(host(db if alias_a else da), B if alias_a else A)
        # the plan's own inverse is unaffected afterwards
        d = dev(A)
        p.inverse(d, 3)
        assert np.array_equal(host(d), a)
        assert p.device_status() == 0


@pytest.mark.parametrize("n", [1, 2, 7, 12, 13, 16, 17])
def test_radix2_organisation(orc, n):
    """One launch per radix-2 stage (the paper's starting point), natural-order
    table: the same transforms as the oracle."""
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    _roundtrip_case(orc, N, primes, 2, 170 + n, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_RADIX2)
    with G.Plan(N, primes, G.NTT_TWIDDLE_AUTO, 0, G.NTT_KERNEL_RADIX2) as p:
        info = p.info()
        assert (info.kernel, info.twiddle_mode) == (G.NTT_KERNEL_RADIX2, G.NTT_TWIDDLE_TABLE)
    with pytest.raises(G.NttError):
        G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_RADIX2)


@pytest.mark.parametrize("n", list(range(1, 18)))
def test_high_radix_organisation(orc, n):
    """One launch per 2^k-point group of stages in registers (the paper's
    register-based high radix), every radix 2^1 .. 2^5, including the short
    last group when k does not divide log2 N."""
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    data = I.batch_uniform(180 + n, 2, primes, N)
    y = I.batch_uniform(190 + n, 2, primes, N)
    want_f, want_i = oracle_fwd(orc, data, primes), oracle_inv(orc, y, primes)
    for k in (1, 2, 3, 4, 5):
        with G.Plan(N, primes, G.NTT_TWIDDLE_AUTO, 0, G.NTT_KERNEL_HIGH_RADIX, radix_log2=k) as p:
            info = p.info()
            assert (info.kernel, info.radix_log2, info.twiddle_mode) == (G.NTT_KERNEL_HIGH_RADIX, k,
                                                                           G.NTT_TWIDDLE_TABLE)
            d = dev(data)
            p.forward(d, 2)
            assert np.array_equal(host(d), want_f), f"forward n={n} radix 2^{k}"
            p.inverse(d, 2)
            assert np.array_equal(host(d), data), f"roundtrip n={n} radix 2^{k}"
            dy = dev(y)
            p.inverse(dy, 2)
            assert np.array_equal(host(dy), want_i), f"inverse n={n} radix 2^{k}"
    with G.Plan(N, primes, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_HIGH_RADIX) as p:
        assert p.info().radix_log2 == 4                   # the default: radix 16


def test_bench_launch_configuration(orc):
    """The bench's configuration at full size: two plans on two streams with
    independent C2 polynomials in flight together, forward then inverse each;
    every forward output against the oracle."""
    w = I.workload_c2()
    datas = [I.batch_uniform(w.seed + 10 * k, 1, w.primes, w.N) for k in range(4)]
    with G.Plan(w.N, w.primes) as p0, G.Plan(w.N, w.primes) as p1:
        plans = [p0, p1]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        bufs = [dev(d) for d in datas]
        fwd = [torch.empty_like(b) for b in bufs]
        torch.cuda.synchronize()
        for k, b in enumerate(bufs):
            s = streams[k % 2]
            with torch.cuda.stream(s):
                plans[k % 2].forward(b, 1, s)
                fwd[k].copy_(b)
                plans[k % 2].inverse(b, 1, s)
        torch.cuda.synchronize()
        for k, d in enumerate(datas):
            assert np.array_equal(host(fwd[k]), oracle_fwd(orc, d, w.primes))
            assert np.array_equal(host(bufs[k]), d)
        assert p0.device_status() == 0 and p1.device_status() == 0


def test_butterfly_rate_measurement():
    """The roofline helper: a register-only butterfly loop runs at a rate of
    the order of the multiply-pipe bound (152 SMs x 2.07 GHz x 3.56/clock)."""
    r = G.ntt_measure_butterfly_rate()
    derived = 152 * 2.07 * 3.556                   # G butterflies per second
    assert 0.3 * derived < r < 1.5 * derived, r


@pytest.mark.parametrize("shape", ["c2", "c3"])
def test_monomial_product_is_signed_shift_full_size(shape):
    """At full size, a * X^k mod (X^N + 1) is a rotation of a by k with the
    wrapped coefficients negated: a property of the product that needs no
    oracle, checked through the forward, product and inverse kernels."""
    w = I.workload_c2() if shape == "c2" else I.workload_c3()
    N, primes = w.N, w.primes
    L = len(primes)
    a = I.batch_uniform(w.seed + 40, 1, primes, N)
    rng = np.random.default_rng(41)
    q = np.array(primes, dtype=np.uint64)[:, None]
    with G.Plan(N, primes) as p:
        for k in (0, 1, int(rng.integers(2, N - 1)), N - 1):
            x = np.zeros((1, L, N), np.uint64)
            x[:, :, k] = 1
            want = np.roll(a[0], k, axis=1)
            want[:, :k] = np.where(want[:, :k] == 0, 0, q - want[:, :k])     # -a mod q for the wrapped part
            da, dx = dev(a), dev(x)
            dc = torch.empty_like(da)
            G.ntt_mul_negacyclic(p.handle, da, dx, dc, 1)
            torch.cuda.synchronize()
            assert np.array_equal(host(dc)[0], want), f"k={k}"
        assert p.device_status() == 0


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
@pytest.mark.parametrize("mode,ots", [(G.NTT_TWIDDLE_TABLE, 0), (G.NTT_TWIDDLE_OT, 1), (G.NTT_TWIDDLE_OT, 2)])
def test_execute_forward_then_inverse_one_launch(orc, n, mode, ots):
    """ntt_execute with both operations (one chained launch for fused plans):
    the round trip restores the input, and each single operation through the
    same call equals the oracle."""
    N = 1 << n
    L = 3 if n < 17 else 2
    primes = I.prime_chain(L, 2 * N)
    data = I.batch_uniform(40 + n, 2, primes, N)
    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
    with G.Plan(N, primes, mode, ots) as p:
        d = dev(data)
        p.execute(d, both, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)
        p.execute(d, G.NTT_OP_FORWARD, 2)
        torch.cuda.synchronize()
        want = oracle_fwd(orc, data, primes)
        assert np.array_equal(host(d).reshape(data.shape), want)
        # the inverse through the call, on forward output and on arbitrary NTT-domain input
        p.execute(d, G.NTT_OP_INVERSE, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)
        d = dev(data)
        p.execute(d, G.NTT_OP_INVERSE, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), oracle_inv(orc, data, primes))
        assert p.device_status() == 0


@pytest.mark.parametrize("geometry", [G.NTT_GEOMETRY_DEFAULT, G.NTT_GEOMETRY_SMALL_ROW_TILE, G.NTT_GEOMETRY_ALT_SPLIT])
@pytest.mark.parametrize("n", [16, 17])
def test_execute_chain_many_limbs_every_geometry(n, geometry):
    """The chained launch at the C2 / C3 shapes in every geometry, with
    queued calls and no synchronisation between them: equal to separate
    forward and inverse calls on the same data (a forward, then a chained
    call, then an inverse, leaves the forward's result of the input)."""
    N = 1 << n
    L = 45 if n == 16 else 60
    primes = I.prime_chain(L, 2 * N)
    data = I.batch_uniform(70 + n, 2 if n == 17 else 1, primes, N)
    b = data.shape[0]
    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
    with G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED, geometry) as p:
        d = dev(data)
        ref = dev(data)
        for _ in range(3):
            p.execute(d, both, b)
        p.forward(ref, b)
        p.execute(d, G.NTT_OP_FORWARD, b)
        p.execute(d, both, b)
        p.execute(ref, both, b)
        torch.cuda.synchronize()
        assert torch.equal(d, ref)
        p.inverse(d, b)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)
        assert p.device_status() == 0


@pytest.mark.parametrize("kernel", [G.NTT_KERNEL_PER_PASS, G.NTT_KERNEL_RADIX2])
def test_execute_other_organisations(kernel):
    """Plans that do not chain run the two operations as two calls."""
    N = 1 << 14
    primes = I.prime_chain(2, 2 * N)
    data = I.batch_uniform(90, 1, primes, N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_TABLE, 0, kernel) as p:
        d = dev(data)
        p.execute(d, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE, 1)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)
        with pytest.raises(G.NttError):
            p.execute(d, 4, 1)


def test_plan_clone_shares_tables_and_runs_concurrently(orc):
    """A clone gives the same results, on another stream at the same time,
    and outlives the plan it was cloned from."""
    N = 1 << 15
    primes = I.prime_chain(6, 2 * N)
    data = I.batch_uniform(123, 2, primes, N)
    p = G.Plan(N, primes)
    c = p.clone()
    assert c.info().device_bytes == p.info().device_bytes
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a, b = dev(data), dev(data)
    for _ in range(4):
        p.execute(a, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE, 2, s1)
        c.execute(b, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE, 2, s2)
    p.forward(a, 2, s1)
    c.forward(b, 2, s2)
    torch.cuda.synchronize()
    want = oracle_fwd(orc, data, primes)
    assert np.array_equal(host(a).reshape(data.shape), want)
    assert np.array_equal(host(b).reshape(data.shape), want)
    p.close()
    c.inverse(b, 2)
    torch.cuda.synchronize()
    assert np.array_equal(host(b).reshape(data.shape), data)
    assert c.device_status() == 0
    c.close()


@pytest.mark.parametrize("n", [13, 16, 17])
@pytest.mark.parametrize("ctas", [1, 2, 8])
def test_ctas_per_sm_option(orc, n, ctas):
    """Plans with one or two persistent CTAs per SM (8: capped by what fits)
    give the oracle's results, alone and with clones running side by side on
    two streams; the plan reports the option."""
    N = 1 << n
    L = 5
    primes = I.prime_chain(L, 2 * N)
    data = [I.batch_uniform(70 + n + k, 1, primes, N) for k in range(4)]
    want = [oracle_fwd(orc, x, primes) for x in data]
    with G.Plan(N, primes, G.NTT_TWIDDLE_OT, 1, ctas_per_sm=ctas) as p:
        assert p.info().ctas_per_sm == ctas
        q = p.clone()
        try:
            assert q.info().ctas_per_sm == ctas
            ss = [torch.cuda.Stream(), torch.cuda.Stream()]
            ds = [dev(x) for x in data]
            for k, d in enumerate(ds):
                (p if k % 2 == 0 else q).forward(d, 1, ss[k % 2])
            torch.cuda.synchronize()
            for d, w in zip(ds, want):
                assert np.array_equal(host(d).reshape(w.shape), w)
            both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
            for k, d in enumerate(ds):
                (p if k % 2 == 0 else q).execute(d, both, 1, ss[k % 2])
            torch.cuda.synchronize()
            for d, w in zip(ds, want):
                assert np.array_equal(host(d).reshape(w.shape), w)
            # the clone switched back to as many CTAs as fit; the source keeps its own
            q.set_ctas_per_sm(0)
            assert q.info().ctas_per_sm == 0 and p.info().ctas_per_sm == ctas
            for k, d in enumerate(ds):
                (p if k % 2 == 0 else q).execute(d, G.NTT_OP_INVERSE, 1, ss[k % 2])
            torch.cuda.synchronize()
            for d, x in zip(ds, data):
                assert np.array_equal(host(d).reshape(x.shape), x)
            assert p.device_status() == 0 and q.device_status() == 0
        finally:
            q.close()


@pytest.mark.parametrize("n", [10, 11, 12])
def test_cluster_organisation(orc, n):
    """The cluster kernel (one limb per cluster of N / 512 CTAs, the passes'
    exchange through distributed shared memory): forward and inverse equal the
    oracle, forward + inverse in one launch restores the input, on several
    limbs of several primes (prime l % L per limb) and through the levels
    call (tables viewed from prime 0, fewer limbs per polynomial)."""
    N = 1 << n
    primes = I.prime_chain(3, 2 * N)
    got = _roundtrip_case(orc, N, primes, 4, 300 + n, kernel=G.NTT_KERNEL_CLUSTER)
    assert np.array_equal(got, _roundtrip_case(orc, N, primes, 4, 300 + n))   # the one-pass kernel agrees
    data = I.batch_uniform(320 + n, 3, primes, N)
    with G.Plan(N, primes, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_CLUSTER) as p:
        info = p.info()
        assert info.kernel == G.NTT_KERNEL_CLUSTER and info.passes == 2 and info.pass1_log2 == n // 2
        d = dev(data)
        p.execute(d, G.NTT_OP_FORWARD | G.NTT_OP_INVERSE, 3)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)
        p.execute(d, G.NTT_OP_FORWARD, 3)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), oracle_fwd(orc, data, primes))
        lv = I.batch_uniform(340 + n, 5, primes[:2], N)
        dl = dev(lv)
        G.ntt_forward_levels(p.handle, dl, 5, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(dl).reshape(lv.shape), oracle_fwd(orc, lv, primes[:2]))
        G.ntt_inverse_levels(p.handle, dl, 5, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(dl).reshape(lv.shape), lv)
        assert p.device_status() == 0


def test_cluster_many_limbs_and_edges(orc):
    """More clusters than fit on the GPU at once (several waves), and the edge
    values 0, 1 and q - 1 in every position."""
    N = 1 << 12
    primes = I.prime_chain(2, 2 * N)
    data = I.batch_uniform(360, 200, primes, N)
    data[0, 0, :] = 0
    data[0, 1, :] = primes[1] - 1
    data[1, 0, ::2] = 1
    with G.Plan(N, primes, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_CLUSTER) as p:
        d = dev(data)
        p.forward(d, 200)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), oracle_fwd(orc, data, primes))
        p.inverse(d, 200)
        torch.cuda.synchronize()
        assert np.array_equal(host(d).reshape(data.shape), data)


def test_every_c2_candidate_full_size(orc):
    """Every configuration the bench's C2 selection can run, at full C2 size:
    a plan and its clones on the candidate's streams, each step one
    ntt_execute(FORWARD | INVERSE) of its own polynomial, as the timed region
    issues them; the forward of each plan, alone, against the oracle."""
    import bench
    w = I.workload_c2()
    both = G.NTT_OP_FORWARD | G.NTT_OP_INVERSE
    datas = [I.batch_uniform(w.seed + 20 * k, 1, w.primes, w.N) for k in range(3)]
    want = oracle_fwd(orc, datas[0], w.primes)
    kernels = {"fused": G.NTT_KERNEL_FUSED, "per_pass": G.NTT_KERNEL_PER_PASS}
    lib = G.lib()
    for kname, tw, geom, ctas, S in bench.C2_CANDIDATES:
        plans = [G.Plan(w.N, w.primes, *bench.TWIDDLES[tw], kernels[kname], geom, ctas_per_sm=ctas)]
        try:
            plans += [plans[0].clone() for _ in range(S - 1)]
            streams = [torch.cuda.Stream() for _ in range(S)]
            bufs = [dev(d) for d in datas]
            torch.cuda.synchronize()
            for i in range(2 * len(bufs)):
                j = i % S
                st = lib.ntt_execute(plans[j].handle, bufs[i % len(bufs)].data_ptr(), 1, both,
                                     streams[j].cuda_stream)
                assert st == 0, (kname, tw, geom, S)
            torch.cuda.synchronize()
            for b, d in zip(bufs, datas):
                assert np.array_equal(host(b), d), f"round trip {kname} {tw} g{geom} s{S}"
            for p in plans:
                x = dev(datas[0])
                p.forward(x, 1)
                torch.cuda.synchronize()
                assert np.array_equal(host(x), want), f"forward {kname} {tw} g{geom} s{S}"
                assert p.device_status() == 0
        finally:
            for p in reversed(plans):
                p.close()
