"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (CPU only; the committed oracle is untouched)."""
import os

import pytest

import oracle
import oracle_pins as P

with open(oracle.SRC) as f:
    SRC = f.read()

MUTANTS = {
    "drop_direct": ("sign * (a * b - exc)", "sign * (-exc)"),
    "exchange_sign": ("sign * (a * b - exc)", "sign * (a * b + exc)"),
    "drop_exchange": ("sign * (a * b - exc)", "sign * (a * b)"),
    "transposed_exchange": ("exc += gat(G[sp], Nw2, N, k2, n2, k1, n1)",
                            "exc += gat(G[sp], Nw2, N, k1, n1, k2, n2)"),
    "b_shift_wrong_side": ("b += spin[sp] * gat(G[sp], Nw2, N, k2, n2, k2q, n2 + m)",
                           "b += spin[sp] * gat(G[sp], Nw2, N, k2q, n2 + m, k2, n2)"),
    "a_spin_unsigned": ("a += spin[sp] *", "a += 1.0 *"),
    "exchange_shift_only_row": ("gat(G[sp], Nw2, N, k1q, n1 + m, k2q, n2 + m)",
                                "gat(G[sp], Nw2, N, k1q, n1 + m, k2, n2 + m)"),
    "build_sign": ("cplx v = -g0[i]", "cplx v = g0[i]"),
    "build_transpose": ("m[(size_t)i * N + j]", "m[(size_t)j * N + i]"),
    "kplus_square_only": ("((ay + by) % d->Ly)", "((ay + by) % d->Lx)"),
    "grid_off_by_one": ("nb < 0 || nb >= Nw2", "nb < 0 || nb > Nw2"),
    "no_normalisation": ("o[i] /= S;", "o[i] /= 1.0;"),
    "frequency_minus": ("gat(G[sp], Nw2, N, k1q, n1 + m, k1, n1)",
                        "gat(G[sp], Nw2, N, k1q, n1 - m, k1, n1)"),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, name
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    oracle.build(str(src), so)
    lib = oracle.load(so)
    bad = P.failing_pins(lib, first_only=True)
    assert bad, "mutant %s passed every pin" % name
