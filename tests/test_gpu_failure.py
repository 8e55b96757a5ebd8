"""Failure detection on the GPU without a fault: a dependency that is never
published makes the fused kernel's bounded waits run out; the kernel reports
it in the plan's status word, touches no data, resets its work area, and the
context stays usable."""
import ctypes

import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import dev, host, oracle_fwd

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu

STATUS_DEP_TIMEOUT = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    lib = G.lib()
    lib.ntt_internal_test_stalled_forward.restype = ctypes.c_int
    lib.ntt_internal_test_stalled_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                                      ctypes.c_uint32]


@pytest.mark.parametrize("n", [13, 16])
def test_unpublished_dependency_times_out_and_recovers(orc, n):
    N = 1 << n
    primes = I.prime_chain(4, 2 * N)
    data = I.batch_uniform(180 + n, 2, primes, N)
    lib = G.lib()
    with G.Plan(N, primes) as p:
        d = dev(data)
        assert lib.ntt_internal_test_stalled_forward(p.handle, d.data_ptr(), 2, 1 << 14) == G.NTT_OK
        st = p.device_status()                   # read and cleared
        assert st & STATUS_DEP_TIMEOUT
        assert np.array_equal(host(d), data)     # no tile was computed or stored
        assert p.device_status() == 0
        # the work area was reset and the context works: a normal transform
        p.forward(d, 2)
        torch.cuda.synchronize()
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
        assert p.device_status() == 0


def test_served_batch_reports_a_stalled_kernel(orc):
    """A served batch whose kernels' bounded waits run out fails its requests
    with NTT_ERR_DEVICE (the status word is read back with the batch, without
    a device synchronisation); the next request on the same server is exact."""
    N = 1 << 14
    primes = I.prime_chain(3, 2 * N)
    data = I.batch_uniform(190, 1, primes, N)
    lib = G.lib()
    lib.ntt_internal_server_test_stall_next.restype = ctypes.c_int
    lib.ntt_internal_server_test_stall_next.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
    with G.Plan(N, primes) as p, G.Server(1 << 30, max_batch_jobs=1, slots=1) as srv:
        d = dev(data)
        assert lib.ntt_internal_server_test_stall_next(srv.handle, 1 << 12) == G.NTT_OK
        t = srv.submit(p.handle, d, 1, len(primes), G.NTT_OP_FORWARD)
        assert srv.wait_status(t) == G.NTT_ERR_DEVICE
        assert np.array_equal(host(d), data)     # no tile was stored
        t = srv.submit(p.handle, d, 1, len(primes), G.NTT_OP_FORWARD)
        assert srv.wait_status(t) == G.NTT_OK
        assert np.array_equal(host(d), oracle_fwd(orc, data, primes))
