"""The CPU oracle against its pins (values and facts it does not produce itself)."""
import pytest

import os, sys
sys.path.insert(0, os.path.dirname(__file__))
import oracle_pins as P  # noqa: E402

_NEEDS_SYMPY = {"pin_primality_vs_sympy", "pin_factors_vs_sympy", "pin_generator_vs_sympy"}


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(orc, pin):
    if pin.__name__ in _NEEDS_SYMPY:
        pytest.importorskip("sympy")
    pin(orc)


def test_psi_of_first_primes_against_sympy(orc):
    """psi for the first prime of each chain, recomputed live with sympy."""
    sympy = pytest.importorskip("sympy")
    import ntt_inputs as I
    for q, N in ((I.workload_c1().primes[0], 1 << 12),
                 (I.workload_c2().primes[0], 1 << 16),
                 (I.workload_c3().primes[0], 1 << 17)):
        g = sympy.primitive_root(q)
        assert orc.psi(q, N) == pow(g, (q - 1) // (2 * N), q)
