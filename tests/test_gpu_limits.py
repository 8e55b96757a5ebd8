"""The API's largest shapes on the GPU: N = 2^17 with L = 4096 primes (one
4 GB polynomial), checked on limbs sampled by the oracle, and a full round
trip."""
import numpy as np
import pytest

import ntt_inputs as I
from gpu_util import host, oracle_fwd

torch = pytest.importorskip("torch")
G = pytest.importorskip("paper_2012_01968_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.build()
    G.lib()


def test_largest_plan_n131072_l4096(orc):
    """The largest plan (N = 2^17, 4096 primes, 4 GiB of data).  A limits
    test: the inputs are uniform in [0, 2^59), below every prime of the chain
    (all primes exceed 2^59) rather than uniform in [0, q); six sampled limbs
    are compared with the oracle and the whole array round-trips."""
    N, L = 1 << 17, 4096
    primes = I.prime_chain(L, 1 << 18)
    assert min(primes) > 1 << 59
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4096)
    data = torch.randint(0, 1 << 59, (L * N,), dtype=torch.int64, device="cuda", generator=gen)   # < every q
    saved = data.clone()
    rng = np.random.default_rng(17)
    sample = sorted({0, L - 1, *(int(x) for x in rng.choice(L, 4, replace=False))})
    inputs = {l: host(data[l * N:(l + 1) * N]) for l in sample}
    with G.Plan(N, primes) as p:
        assert p.info().L == L
        p.forward(data, 1)
        torch.cuda.synchronize()
        for l in sample:
            want = oracle_fwd(orc, inputs[l][None, None, :], [primes[l]])[0, 0]
            assert np.array_equal(host(data[l * N:(l + 1) * N]), want), f"limb {l}"
        p.inverse(data, 1)
        torch.cuda.synchronize()
        assert torch.equal(data, saved)
        assert p.device_status() == 0
