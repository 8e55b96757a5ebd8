"""C ABI: the library loads, exports every declared symbol, and validates
arguments on the host (no GPU needed for any of these)."""
import ctypes
import os
import subprocess

import pytest

import ntt_inputs as I

G = pytest.importorskip("paper_2012_01968_gb300")


@pytest.fixture(scope="module")
def lib():
    G.build()
    return G.lib()


def test_exports_every_declared_symbol(lib):
    names = G.declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    # and nm agrees (dynamic symbol table)
    out = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in names:
        assert n in exported, n


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "ntt_gb300.h"\nint main(void){ntt_plan_info i; (void)i; return NTT_OK;}\n')
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(G.ROOT, "include"),
                           "-c", str(src), "-o", str(tmp_path / "t.o")])


def test_status_strings(lib):
    for s in range(9):
        assert G.ntt_status_string(s).startswith("NTT_")
    assert "unknown" in G.ntt_status_string(99)


BIG = I.prime_chain(3, 1 << 18)


@pytest.mark.parametrize("N,primes,kw,want", [
    (0, BIG[:1], {}, G.NTT_ERR_INVALID_ARG),
    (1, BIG[:1], {}, G.NTT_ERR_INVALID_ARG),
    (3, BIG[:1], {}, G.NTT_ERR_INVALID_ARG),
    (1 << 18, BIG[:1], {}, G.NTT_ERR_INVALID_ARG),
    (1 << 12, [], {}, G.NTT_ERR_INVALID_ARG),
    (1 << 12, [17], {}, G.NTT_ERR_BAD_PRIME),                       # below 2^32
    (1 << 12, [(1 << 61) - 1], {}, G.NTT_ERR_BAD_PRIME),            # above 2^60
    (1 << 12, [(1 << 59) + 1], {}, G.NTT_ERR_BAD_PRIME),            # 1 mod 2N, divisible by 3
    (1 << 17, I.prime_chain(1, 1 << 13), {}, G.NTT_ERR_BAD_PRIME),  # not 1 mod 2^18
    (1 << 12, BIG[:1], {"twiddle_mode": 7}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"twiddle_mode": G.NTT_TWIDDLE_OT, "ot_stages": 3}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"twiddle_mode": G.NTT_TWIDDLE_TABLE, "ot_stages": 1}, G.NTT_ERR_INVALID_ARG),
    (1 << 12, BIG[:1], {"reserved": [1]}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"ctas_per_sm": 9}, G.NTT_ERR_INVALID_ARG),             # more CTAs per SM than any fit
    (1 << 9, BIG[:1], {"kernel": G.NTT_KERNEL_CLUSTER}, G.NTT_ERR_INVALID_ARG),   # below the cluster sizes
    (1 << 13, BIG[:1], {"kernel": G.NTT_KERNEL_CLUSTER}, G.NTT_ERR_INVALID_ARG),  # above them
    (1 << 12, BIG[:1], {"kernel": G.NTT_KERNEL_CLUSTER, "twiddle_mode": G.NTT_TWIDDLE_OT},
     G.NTT_ERR_INVALID_ARG),                                                     # table twiddles only
    (1 << 12, BIG[:1], {"kernel": 6}, G.NTT_ERR_INVALID_ARG),                  # no such organisation
    (1 << 16, BIG[:1], {"geometry": 3}, G.NTT_ERR_INVALID_ARG),                # no such geometry
    (1 << 12, BIG[:1], {"geometry": 1}, G.NTT_ERR_INVALID_ARG),                # one-pass size
    (1 << 16, BIG[:1], {"geometry": 2, "kernel": G.NTT_KERNEL_RADIX2}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"flags": 2}, G.NTT_ERR_INVALID_ARG),                   # unknown flag bit
    (1 << 16, BIG[:1], {"kernel": G.NTT_KERNEL_HIGH_RADIX, "radix_log2": 6}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"radix_log2": 4}, G.NTT_ERR_INVALID_ARG),              # radix only for HIGH_RADIX
    (1 << 16, BIG[:1], {"kernel": G.NTT_KERNEL_HIGH_RADIX, "twiddle_mode": G.NTT_TWIDDLE_OT}, G.NTT_ERR_INVALID_ARG),
    (1 << 16, BIG[:1], {"kernel": G.NTT_KERNEL_HIGH_RADIX, "geometry": 1}, G.NTT_ERR_INVALID_ARG),
])
def test_plan_create_rejects(lib, N, primes, kw, want):
    st, h = G.ntt_plan_create_status(N, primes, **kw)
    assert st == want
    assert h == 0


SMALL = I.small_ntt_primes(1 << 12, 2, start=1 << 27)      # 28-bit primes = 1 mod 2^13


@pytest.mark.parametrize("N,primes,want", [
    (0, SMALL[:1], G.NTT_ERR_INVALID_ARG),
    (3, SMALL[:1], G.NTT_ERR_INVALID_ARG),
    (1 << 18, SMALL[:1], G.NTT_ERR_INVALID_ARG),
    (1 << 12, [], G.NTT_ERR_INVALID_ARG),
    (1 << 12, [1 << 28 | 1], G.NTT_ERR_BAD_PRIME),                       # not below 2^28
    (1 << 12, BIG[:1], G.NTT_ERR_BAD_PRIME),                             # a 60-bit prime
    (1 << 12, [3 * 8192 + 1], G.NTT_ERR_BAD_PRIME),                      # 1 mod 2N, composite (7 * 3511)
    (1 << 13, SMALL[1:2], G.NTT_ERR_BAD_PRIME),                          # 8193 mod 2^14
    (2, [2], G.NTT_ERR_BAD_PRIME),                                       # 2 is not 1 mod 4
])
def test_plan32_create_rejects(lib, N, primes, want):
    st, h = G.ntt_plan32_create_status(N, primes)
    assert st == want
    assert h == 0


@pytest.mark.parametrize("kernel", [G.NTT_KERNEL_RADIX2, G.NTT_KERNEL_HIGH_RADIX, 9])
def test_plan32_rejects_kernel(lib, kernel):
    st, h = G.ntt_plan32_create_status(1 << 13, SMALL[:1], kernel)
    assert st == G.NTT_ERR_INVALID_ARG and h == 0


@pytest.mark.parametrize("N,kernel,mode", [(1 << 12, G.NTT_KERNEL_AUTO, G.NTT_TWIDDLE_OT),       # one pass
                                           (1 << 13, G.NTT_KERNEL_PER_PASS, G.NTT_TWIDDLE_OT),  # per pass: table
                                           (1 << 13, G.NTT_KERNEL_AUTO, 3)])
def test_plan32_rejects_twiddle_mode(lib, N, kernel, mode):
    st, h = G.ntt_plan32_create_status(N, SMALL[:1], kernel, mode)
    assert st == G.NTT_ERR_INVALID_ARG and h == 0


def test_plan32_primes_are_28_bit():
    assert all((1 << 27) <= q < (1 << 28) and q % (1 << 13) == 1 and I.is_prime(q) for q in SMALL)
    assert SMALL[1] % (1 << 14) != 1


def test_null_arguments_rejected(lib):
    assert lib.ntt_forward(None, None, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_inverse(None, None, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_mul_pointwise(None, None, None, None, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_execute_host(None, None, None, 1, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan_query(None, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan_create(None, 16, None, 1, None) == G.NTT_ERR_INVALID_ARG
    lib.ntt_plan_destroy(None)
    assert lib.ntt_forward32(None, None, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_inverse32(None, None, 1, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan32_psi(None, 0, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan32_create(None, 16, None, 1, 0, 0) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_plan32_device_status(None, None) == G.NTT_ERR_INVALID_ARG
    best = G.PlanOpts()
    assert lib.ntt_autotune(16, None, 1, 1, 1, ctypes.byref(best), None, 0, None) == G.NTT_ERR_INVALID_ARG
    arr = (ctypes.c_uint64 * 1)(BIG[0])
    assert lib.ntt_autotune(16, arr, 1, 0, 1, ctypes.byref(best), None, 0, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_autotune(3, arr, 1, 1, 1, ctypes.byref(best), None, 0, None) == G.NTT_ERR_INVALID_ARG
    assert lib.ntt_autotune(16, arr, 1, 1, 1, None, None, 0, None) == G.NTT_ERR_INVALID_ARG
    lib.ntt_plan32_destroy(None)


def test_no_oracle_in_product_path():
    """The CUDA library and its binding never reference the oracle."""
    pkg = os.path.dirname(G.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "oracle" not in txt.lower(), f
    out = subprocess.run(["nm", "-D", G.LIB_PATH], capture_output=True, text=True).stdout
    assert "orc_" not in out
