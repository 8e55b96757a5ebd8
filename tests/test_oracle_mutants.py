"""Planted mistakes in copies of the oracle must each trip at least one pin.

Each mutant is the oracle's C source with one edit (a dropped term, a wrong
sign, index or exponent, a transposed operand), compiled on the CPU into a
temporary directory.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

sys.path.insert(0, os.path.dirname(__file__))
import oracle  # noqa: E402
import oracle_pins as P  # noqa: E402

SRC = os.path.join(os.path.dirname(oracle.__file__), "ntt_oracle.c")

# (name, text to find, replacement, occurrence index to replace)
MUTANTS = [
    ("fwd_twiddle_index", "u64 w = Psi[m + j];", "u64 w = Psi[m + ((j + 1) % m)];", 0),
    ("fwd_butterfly_sign", "a[k + t] = submod(U, V, q);", "a[k + t] = submod(V, U, q);", 0),
    ("fwd_drop_last_stage", "for (u64 m = 1; m < N; m *= 2)", "for (u64 m = 1; m < N / 2; m *= 2)", 0),
    ("psi_nth_not_2nth", "return orc_powmod(g, (q - 1) / (2 * N), q);",
     "return orc_powmod(g, (q - 1) / N, q);", 0),
    ("inv_drop_ninv", "for (u64 k = 0; k < N; ++k) a[k] = mulmod(a[k], n_inv, q);",
     "for (u64 k = 0; k < N; ++k) a[k] = a[k];", 0),
    ("inv_uses_psi", "twiddles_bitrev(Pinv, N, q, orc_invmod(psi, q));",
     "twiddles_bitrev(Pinv, N, q, psi);", 0),
    ("inv_butterfly_operands", "a[k + t] = mulmod(submod(U, V, q), w, q);",
     "a[k + t] = mulmod(submod(V, U, q), w, q);", 0),
    ("product_sign", "acc = submod(acc, mulmod(a[i], b[N + k - i], q), q);",
     "acc = addmod(acc, mulmod(a[i], b[N + k - i], q), q);", 0),
    ("product_index", "mulmod(a[i], b[N + k - i], q)", "mulmod(a[i], b[(N + i - k) % N], q)", 0),
    ("schoolbook_unmerged_root", "u64 root = orc_powmod(psi, 2 * k + 1, q);",
     "u64 root = orc_powmod(psi, 2 * k, q);", 0),
    ("schoolbook_natural_order", "u64 k = orc_bitrev(i, n);\n        u64 root = orc_powmod(psi,",
     "u64 k = i;\n        u64 root = orc_powmod(psi,", 0),
    ("bitrev_wrong_bit", "r = (r << 1) | (i & 1);", "r = (r << 1) | ((i >> 1) & 1);", 0),
    ("generator_skips_factors", "int nf = orc_prime_factors(q - 1, f, 64);",
     "int nf = 1; f[0] = 2;", 0),
    ("mr_short_witness_loop", "for (int r = 1; r < s; ++r) {", "for (int r = 2; r < s; ++r) {", 0),
    ("factor_step", "d += 2) {", "d += 4) {", 0),
    ("pointwise_operand", "c[i] = mulmod(a[i], b[i], q);", "c[i] = mulmod(a[i], a[i], q);", 0),
    ("horner_reversed", "acc = addmod(mulmod(acc, x, q), a[j], q);",
     "acc = addmod(mulmod(acc, x, q), a[N - 1 - j], q);", 0),
    ("intt_schoolbook_drop_scale", "for (u64 j = 0; j < N; ++j) out[j] = mulmod(out[j], n_inv, q);",
     "for (u64 j = 0; j < N; ++j) out[j] = out[j];", 0),
    ("batch_wrong_limb_prime", "u64 l = idx % j->L;", "u64 l = (idx + 1) % j->L;", 0),
]


def _apply(src, find, repl, occ):
    parts = src.split(find)
    assert len(parts) > occ + 1, f"pattern not found: {find!r}"
    return find.join(parts[:occ + 1]) + repl + find.join(parts[occ + 1:])


@pytest.mark.parametrize("name,find,repl,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, find, repl, occ):
    pytest.importorskip("sympy")
    with open(SRC) as f:
        src = f.read()
    mutated = _apply(src, find, repl, occ)
    assert mutated != src
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", str(so), str(c)])
    o = oracle.lib(str(so))
    tripped = []
    for pin in P.ALL_PINS:
        try:
            pin(o)
        except (AssertionError, ValueError, MemoryError, ZeroDivisionError):
            tripped.append(pin.__name__)
    assert tripped, f"mutant {name} passed every pin"
