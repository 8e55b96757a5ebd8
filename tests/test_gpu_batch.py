"""Uneven batches through ntt_batch_submit, against the oracle and against
single calls, bit for bit; graph capture and argument checks."""
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
def chain():
    return I.chain_2_18_60()          # q = 1 mod 2^18: valid for every N <= 2^17


def _job_data(w, job, chain):
    return I.batch_uniform(w.seed, 1, chain[:job.L], job.N, first_poly=job.poly)


# the configurations the autotuner picks for these sizes on GB300 (fused kernel,
# table twiddles; geometry per size), as the bench's tuned C4 / C5 legs use them
TUNED_C4 = {14: (G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED, 1), 15: (G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED, 2),
            16: (G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED, 0), 17: (G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_FUSED, 1)}


@pytest.mark.parametrize("options", ["default", "tuned"])
def test_uneven_batch_c4_against_oracle(orc, chain, options):
    """The 96-job uneven workload (N in 2^14..2^17, L in [1, 60], mixed
    directions) in one submission, every job against the oracle; with the
    default plan options and with the tuned ones."""
    w = I.workload_c4()
    plans = {n: (G.Plan(1 << n, chain, *TUNED_C4[n]) if options == "tuned" else G.Plan(1 << n, chain))
             for n in range(14, 18)}
    try:
        datas = [_job_data(w, j, chain) for j in w.jobs]
        devs = [dev(d) for d in datas]
        with G.Batch() as b:
            b.submit([(plans[I.log2_exact(j.N)].handle, devs[i], 1, j.L, FWD if j.dir > 0 else INV)
                      for i, j in enumerate(w.jobs)])
            torch.cuda.synchronize()
            assert b.device_status() == 0
            if options == "default":
                assert _last_launches(b) == 1          # all 96 jobs, four sizes, both directions
        for i, j in enumerate(w.jobs):
            want = (oracle_fwd if j.dir > 0 else oracle_inv)(orc, datas[i], chain[:j.L])
            assert np.array_equal(host(devs[i]), want), f"job {i}: N={j.N} L={j.L} dir={j.dir}"
    finally:
        for p in plans.values():
            p.close()


def test_batch_equals_single_calls(chain):
    """Mixed sizes (including one-pass sizes and a launch-per-pass plan),
    batches > 1, levels < L: the batch gives what single calls give."""
    rng = np.random.default_rng(7)
    specs = [(12, 3, 2, FWD), (13, 2, 5, INV), (14, 4, 17, FWD), (14, 1, 60, INV), (16, 2, 45, FWD),
             (17, 1, 8, INV), (15, 3, 1, FWD), (16, 1, 3, INV)]
    plans = {n: G.Plan(1 << n, chain) for n in {s[0] for s in specs}}
    pp = G.Plan(1 << 15, chain, G.NTT_TWIDDLE_TABLE, 0, G.NTT_KERNEL_PER_PASS)
    specs_plans = [(plans[n], n, bt, lv, op) for n, bt, lv, op in specs] + [(pp, 15, 2, 6, INV)]
    try:
        datas = [I.batch_uniform(200 + i, bt, chain[:lv], 1 << n) for i, (_, n, bt, lv, _) in enumerate(specs_plans)]
        got = [dev(d) for d in datas]
        want = [dev(d) for d in datas]
        for (p, n, bt, lv, op), t in zip(specs_plans, want):
            (G.ntt_forward_levels if op == FWD else G.ntt_inverse_levels)(p.handle, t, bt, lv)
        with G.Batch() as b:
            jobs = [(p.handle, t, bt, lv, op) for (p, n, bt, lv, op), t in zip(specs_plans, got)]
            rng.shuffle(jobs)
            b.submit(jobs)
            torch.cuda.synchronize()
            assert b.device_status() == 0
        for a, c in zip(got, want):
            assert torch.equal(a, c)
    finally:
        for p in list(plans.values()) + [pp]:
            p.close()


def _last_launches(b):
    import ctypes
    fn = G.lib().ntt_internal_batch_last_launches
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]
    n = ctypes.c_uint32()
    assert fn(b.handle, ctypes.byref(n)) == 0
    return n.value


@pytest.mark.parametrize("geometry", [G.NTT_GEOMETRY_DEFAULT, G.NTT_GEOMETRY_SMALL_ROW_TILE])
def test_many_jobs_one_size(chain, geometry):
    """40 jobs of one size and direction: one mixed launch with the default
    geometry, launches of up to 16 jobs with another."""
    p = G.Plan(1 << 13, chain, G.NTT_TWIDDLE_OT, 1, G.NTT_KERNEL_FUSED, geometry)
    try:
        datas = [I.batch_uniform(300 + i, 1, chain[:1 + i % 5], 1 << 13) for i in range(40)]
        got = [dev(d) for d in datas]
        want = [dev(d) for d in datas]
        for d, t in zip(datas, want):
            G.ntt_forward_levels(p.handle, t, 1, d.shape[1])
        with G.Batch() as b:
            b.submit([(p.handle, t, 1, d.shape[1], FWD) for d, t in zip(datas, got)])
            torch.cuda.synchronize()
            assert b.device_status() == 0
            assert _last_launches(b) == (1 if geometry == G.NTT_GEOMETRY_DEFAULT else 3)
        for a, c in zip(got, want):
            assert torch.equal(a, c)
    finally:
        p.close()


def test_batch_graph_capture_and_replay(orc, chain):
    """A submission captured into a CUDA graph after one eager submission of
    the same shape; replays on new inputs match the oracle."""
    plans = {n: G.Plan(1 << n, chain) for n in (14, 16)}
    shapes = [(14, 7, FWD), (16, 5, INV), (16, 9, FWD), (14, 3, INV)]
    try:
        bufs = [torch.zeros((lv << n,), dtype=torch.int64, device="cuda") for n, lv, _ in shapes]
        jobs = G.make_jobs([(plans[n].handle, t, 1, lv, op) for (n, lv, op), t in zip(shapes, bufs)])
        with G.Batch() as b:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                b.submit(jobs, s)                       # sizes the work area
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                b.submit(jobs, s)
            for rep in range(2):
                datas = [I.batch_uniform(400 + 10 * rep + i, 1, chain[:lv], 1 << n)
                         for i, (n, lv, _) in enumerate(shapes)]
                for t, d in zip(bufs, datas):
                    t.copy_(dev(d).reshape(-1))
                g.replay()
                torch.cuda.synchronize()
                for (n, lv, op), t, d in zip(shapes, bufs, datas):
                    want = (oracle_fwd if op == FWD else oracle_inv)(orc, d, chain[:lv])
                    assert np.array_equal(host(t), want.reshape(-1))
            assert b.device_status() == 0
    finally:
        for p in plans.values():
            p.close()


def _sets_of_jobs(chain, sets, seed):
    """Device arrays with fresh inputs for each set of (n, levels, op) jobs."""
    datas = [[I.batch_uniform(seed + 10 * k + i, 1, chain[:lv], 1 << n) for i, (n, lv, _) in enumerate(js)]
             for k, js in enumerate(sets)]
    return datas, [[dev(d) for d in ds] for ds in datas]


def _check_sets(orc, chain, sets, datas, bufs):
    for js, ds, ts in zip(sets, datas, bufs):
        for (n, lv, op), d, t in zip(js, ds, ts):
            want = (oracle_fwd if op == FWD else oracle_inv)(orc, d, chain[:lv])
            assert np.array_equal(host(t), want), f"n={n} levels={lv} op={op}"


def test_changed_descriptors_do_not_drain_the_stream(orc, chain):
    """Three submissions with different mixed-launch descriptors, queued on a
    stream behind a long kernel, return while that kernel still runs (the
    host does not wait for the stream), and their results match the oracle."""
    plans = {n: G.Plan(1 << n, chain) for n in (14, 15)}
    sets = [[(14, 5, FWD), (15, 3, INV)], [(15, 4, FWD), (14, 2, FWD)], [(14, 6, INV)]]
    try:
        with G.Batch() as b:
            s = torch.cuda.Stream()
            _, bufs = _sets_of_jobs(chain, sets, 700)
            for js, ts in zip(sets, bufs):             # sizes the work area and descriptor arrays
                b.submit([(plans[n].handle, t, 1, lv, op) for (n, lv, op), t in zip(js, ts)], s)
            torch.cuda.synchronize()
            datas, bufs = _sets_of_jobs(chain, sets, 800)
            torch.cuda.synchronize()
            with torch.cuda.stream(s):
                torch.cuda._sleep(1_000_000_000)        # about 0.5 s of device time
            for js, ts in zip(sets, bufs):
                b.submit([(plans[n].handle, t, 1, lv, op) for (n, lv, op), t in zip(js, ts)], s)
            assert not s.query(), "a submission waited for the stream"
            torch.cuda.synchronize()
            assert b.device_status() == 0
        _check_sets(orc, chain, sets, datas, bufs)
    finally:
        for p in plans.values():
            p.close()


def test_many_changed_submissions_in_flight(orc, chain):
    """Seven submissions with different descriptors back to back on one
    stream (more than the four descriptor generations, so the later ones
    reuse generations of earlier ones still queued): all match the oracle."""
    plans = {n: G.Plan(1 << n, chain) for n in (13, 14, 16)}
    sets = [[(13, 2 + k, FWD if k % 2 else INV), (16, 1 + k % 3, FWD), (14, 3, INV if k % 3 else FWD)]
            for k in range(7)]
    try:
        with G.Batch() as b:
            s = torch.cuda.Stream()
            datas, bufs = _sets_of_jobs(chain, sets, 900)
            torch.cuda.synchronize()
            for js, ts in zip(sets, bufs):
                b.submit([(plans[n].handle, t, 1, lv, op) for (n, lv, op), t in zip(js, ts)], s)
            torch.cuda.synchronize()
            assert b.device_status() == 0
        _check_sets(orc, chain, sets, datas, bufs)
    finally:
        for p in plans.values():
            p.close()


def test_batch_argument_errors(chain):
    p = G.Plan(1 << 13, chain[:4])
    buf = torch.zeros(4 << 14, dtype=torch.int64, device="cuda")
    lib = G.lib()
    try:
        with G.Batch() as b:
            def status(jobs):
                arr = G.make_jobs(jobs)
                return lib.ntt_batch_submit(b.handle, arr, len(arr), None)
            h, a = p.handle, buf.data_ptr()
            assert status([(h, a, 1, 5, FWD)]) == G.NTT_ERR_INVALID_ARG            # levels > L
            assert status([(h, a, 1, 2, 3)]) == G.NTT_ERR_INVALID_ARG              # op
            assert status([(h, a, 0, 2, FWD)]) == G.NTT_ERR_INVALID_ARG            # batch 0
            assert status([(h, a + 8, 1, 2, FWD)]) == G.NTT_ERR_MISALIGNED
            assert status([(None, a, 1, 2, FWD)]) == G.NTT_ERR_INVALID_ARG
            # overlapping arrays: the second starts inside the first
            assert status([(h, a, 1, 2, FWD), (h, a + (1 << 13) * 8, 1, 2, INV)]) == G.NTT_ERR_INVALID_ARG
            assert lib.ntt_batch_submit(b.handle, None, 0, None) == G.NTT_ERR_INVALID_ARG
            torch.cuda.synchronize()
            assert int(buf.abs().sum()) == 0                                        # nothing ran
    finally:
        p.close()
