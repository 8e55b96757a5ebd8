"""The serving loop: requests of mixed sizes arriving over time, admitted by
device memory and batched continuously; every result must equal the same
request run alone, bit for bit."""
import threading
import time

import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import dev, host, oracle_fwd, oracle_inv

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


@pytest.fixture(scope="module")
def plans():
    chain = I.chain_2_18_60()
    ps = {n: G.Plan(1 << n, chain) for n in (13, 15, 16, 17)}
    yield ps
    for p in ps.values():
        p.close()


def _requests(count, seed, logn=(15, 16, 17), lmax=20):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(logn))
        L = int(rng.integers(4, lmax + 1))
        op = FWD if rng.integers(0, 2) == 0 else INV
        out.append((n, L, op, i))
    return out


def test_mixed_requests_equal_alone(plans):
    """Requests submitted from a thread at random times, under a budget that
    admits only a few at once: each equals the same transform run alone."""
    chain = I.chain_2_18_60()
    reqs = _requests(60, 1)
    datas = [I.batch_uniform(500 + i, 1, chain[:L], 1 << n) for n, L, _, i in reqs]
    mix = [dev(d) for d in datas]
    alone = [dev(d) for d in datas]
    for (n, L, op, _), t in zip(reqs, alone):
        (G.ntt_forward_levels if op == FWD else G.ntt_inverse_levels)(plans[n].handle, t, 1, L)
    torch.cuda.synchronize()
    budget = 48 << 20                                 # a few requests at a time (largest: 20 MB)
    with G.Server(budget, max_batch_jobs=8, slots=3) as srv:
        tickets = [None] * len(reqs)

        def producer():
            rng = np.random.default_rng(2)
            for k, ((n, L, op, _), t) in enumerate(zip(reqs, mix)):
                tickets[k] = srv.submit(plans[n].handle, t, 1, L, op)
                time.sleep(float(rng.exponential(50e-6)))

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        for t in tickets:
            srv.wait(t)
        times = [srv.times(t) for t in tickets]
    for k, (a, b) in enumerate(zip(mix, alone)):
        assert torch.equal(a, b), f"request {k} differs from the same request alone"
    for s, st, d, dev_ns in times:
        assert 0 < s <= st <= d
        assert 0 < dev_ns <= d - st              # the batch's device time fits its wall time


def test_host_requests_through_arena(plans, orc):
    """Host-buffer requests are copied through the device arena; results
    match the oracle, also in place (host_out = data)."""
    chain = I.chain_2_18_60()
    reqs = _requests(12, 3, logn=(13, 15), lmax=6)
    datas = [I.batch_uniform(600 + i, 1, chain[:L], 1 << n) for n, L, _, i in reqs]
    outs = [np.empty_like(d) for d in datas]
    inplace = [d.copy() for d in datas]
    with G.Server(64 << 20, arena_bytes=8 << 20, max_batch_jobs=4, slots=2) as srv:
        tk = []
        for (n, L, op, _), d, o, ip in zip(reqs, datas, outs, inplace):
            tk.append(srv.submit(plans[n].handle, d, 1, L, op, host_out=o))
            tk.append(srv.submit(plans[n].handle, ip, 1, L, op, host_out=ip))
        for t in tk:
            srv.wait(t)
    for (n, L, op, _), d, o, ip in zip(reqs, datas, outs, inplace):
        if op == FWD:
            want = oracle_fwd(orc, d, chain[:L])
        else:
            want = orc.ntt_batch(d, chain[:L], -1, 8)
        assert np.array_equal(o, want)
        assert np.array_equal(ip, want)


def test_served_c5_shapes_against_oracle(plans, orc):
    """Requests of the serving workload's own shapes (its seeded draws of
    N in {2^15, 2^16, 2^17}, L in [4, 60] and the direction, plus one
    N = 2^17, L = 60 request per direction), uniform residues in [0, q),
    served together under a budget that admits several at once: every
    result against the oracle, element by element."""
    chain = I.chain_2_18_60()
    reqs = [(r.N.bit_length() - 1, r.L, FWD if r.dir > 0 else INV) for r in I.serving_requests(14, seed=5)]
    reqs += [(17, 60, FWD), (17, 60, INV)]
    datas = [I.batch_uniform(900 + i, 1, chain[:L], 1 << n) for i, (n, L, _) in enumerate(reqs)]
    bufs = [dev(d) for d in datas]
    with G.Server(256 << 20, max_batch_jobs=6, slots=3) as srv:
        tickets = [srv.submit(plans[n].handle, b, 1, L, op) for (n, L, op), b in zip(reqs, bufs)]
        for t in tickets:
            srv.wait(t)
    assert any(n == 17 and L == 60 for n, L, _ in reqs)
    for k, ((n, L, op), d, b) in enumerate(zip(reqs, datas, bufs)):
        want = oracle_fwd(orc, d, chain[:L]) if op == FWD else oracle_inv(orc, d, chain[:L])
        assert np.array_equal(host(b).reshape(d.shape), want), f"request {k} (N=2^{n}, L={L})"


def test_release_and_stats(plans):
    """A finished request can be released (its ticket is then unknown); an
    unfinished one cannot; the scheduler counters count batches and
    requests."""
    chain = I.chain_2_18_60()
    big = torch.zeros(60 << 17, dtype=torch.int64, device="cuda")
    a = dev(I.batch_uniform(31, 1, chain[:8], 1 << 15))
    with G.Server(1 << 30, max_batch_jobs=4, slots=2) as srv:
        tk = srv.submit(plans[17].handle, big, 1, 60, FWD)
        busy = srv.release_status(tk)         # a 60-limb N = 2^17 batch is still running (almost surely)
        srv.wait(tk)
        assert busy in (G.NTT_ERR_BUSY, G.NTT_OK)
        t2 = srv.submit(plans[15].handle, a, 1, 8, FWD)
        srv.wait(t2)
        srv.times(t2)
        srv.release(t2)
        assert srv.release_status(t2) == G.NTT_ERR_INVALID_ARG
        with pytest.raises(G.NttError):
            srv.times(t2)
        st = srv.stats()
        assert st["batches"] >= 2 and st["requests"] >= 2
        assert 0 < st["max_device_ns"] and 0 < st["max_launch_ns"] and 0 < st["max_loop_gap_ns"]
        if busy == G.NTT_OK:
            return
        srv.release(tk)


def test_admission_refused_when_queue_full(plans):
    """With max_queue requests waiting, a submission is refused (BUSY)."""
    N = 1 << 17
    bufs = [torch.zeros(60 * N, dtype=torch.int64, device="cuda") for _ in range(8)]
    with G.Server(61 * N * 8, max_batch_jobs=1, slots=1, max_queue=2) as srv:
        sts, tickets = [], []
        for b in bufs:
            st, t = srv.submit_status(plans[17].handle, b, 1, 60, FWD)
            sts.append(st)
            if st == G.NTT_OK:
                tickets.append(t)
        assert G.NTT_ERR_BUSY in sts
        for t in tickets:
            srv.wait(t)
    assert len(tickets) >= 3            # one admitted, two waiting


def test_wait_timeout_and_drain(plans):
    """A wait that runs out returns TIMEOUT and the request still completes;
    destroying the server waits for every request."""
    N = 1 << 17
    big = torch.zeros(60 * N, dtype=torch.int64, device="cuda")
    other = torch.zeros(60 * N, dtype=torch.int64, device="cuda")
    srv = G.Server(61 * N * 8, max_batch_jobs=1, slots=1)
    t1 = srv.submit(plans[17].handle, big, 1, 60, FWD)
    t2 = srv.submit(plans[17].handle, other, 1, 60, FWD)       # waits for t1's memory
    assert srv.wait_status(t2, 0.0) == G.NTT_ERR_TIMEOUT
    srv.wait(t1)
    srv.wait(t2)
    t3 = srv.submit(plans[17].handle, big, 1, 60, INV)
    srv.close()                                                   # drains t3
    torch.cuda.synchronize()
    assert int(big.abs().sum()) == 0 and int(other.abs().sum()) == 0   # NTT of zero is zero


def test_request_errors(plans):
    buf = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
    with G.Server(1 << 20) as srv:
        h = plans[13].handle
        assert srv.submit_status(h, buf, 1, 61, FWD)[0] == G.NTT_ERR_INVALID_ARG      # levels > L
        assert srv.submit_status(h, buf, 1, 2, 9)[0] == G.NTT_ERR_INVALID_ARG        # op
        assert srv.submit_status(h, buf.data_ptr() + 8, 1, 2, FWD)[0] == G.NTT_ERR_MISALIGNED
        assert srv.submit_status(h, buf, 1, 60, FWD)[0] == G.NTT_ERR_INVALID_ARG     # above the budget
        assert srv.submit_status(h, np.zeros(4 << 13, np.uint64), 1, 4, FWD,
                                 host_out=np.zeros(4 << 13, np.uint64))[0] == G.NTT_ERR_INVALID_ARG  # no arena
