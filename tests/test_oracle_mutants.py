"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (CPU only; the committed oracle is untouched)."""
import os

import pytest

import oracle
import oracle_pins as P

with open(oracle.SRC) as f:
    SRC = f.read()

MUTANTS = {
    # particle-hole magnetic (default channel)
    "drop_direct": ("term = a * b - exc;", "term = -exc;"),
    "exchange_sign": ("term = a * b - exc;", "term = a * b + exc;"),
    "drop_exchange": ("term = a * b - exc;", "term = a * b;"),
    "transposed_exchange": ("exc += gat(G[sp], Nw2, N, k2, n2, k1, n1)",
                            "exc += gat(G[sp], Nw2, N, k1, n1, k2, n2)"),
    "b_shift_wrong_side": ("b += w * gat(G[sp], Nw2, N, k2, n2, k2q, n2 + m)",
                           "b += w * gat(G[sp], Nw2, N, k2q, n2 + m, k2, n2)"),
    "a_spin_unsigned": ("const double w = channel == 0 ? spin[sp] : 1.0;",
                        "const double w = 1.0;"),
    "exchange_shift_only_row": ("gat(G[sp], Nw2, N, k1q, n1 + m, k2q, n2 + m);\n                            }",
                                "gat(G[sp], Nw2, N, k1q, n1 + m, k2, n2 + m);\n                            }"),
    "build_sign": ("cplx v = -g0[i]", "cplx v = g0[i]"),
    "build_transpose": ("m[(size_t)i * N + j]", "m[(size_t)j * N + i]"),
    "kplus_square_only": ("return (ax + bx) % d->Lx + d->Lx * ((ay + by) % d->Ly);",
                          "return (ax + bx) % d->Lx + d->Lx * ((ay + by) % d->Lx);"),
    "grid_off_by_one": ("nb < 0 || nb >= Nw2", "nb < 0 || nb > Nw2"),
    "no_normalisation": ("o[i] /= S;", "o[i] /= 1.0;"),
    "frequency_minus": ("a += w * gat(G[sp], Nw2, N, k1q, n1 + m, k1, n1)",
                        "a += w * gat(G[sp], Nw2, N, k1q, n1 - m, k1, n1)"),
    # other channels
    "density_signed": ("const double w = channel == 0 ? spin[sp] : 1.0;",
                       "const double w = spin[sp];"),
    "pp_same_spin": ("gat(G[1 - sp], Nw2, N, k2, n2, k1, n1);\n                        } else if",
                     "gat(G[sp], Nw2, N, k2, n2, k1, n1);\n                        } else if"),
    "pp_reflection_offset": ("const int f1 = m + Nw2 - 1 - n1, f2 = m + Nw2 - 1 - n2;",
                             "const int f1 = m + Nw2 - n1, f2 = m + Nw2 - n2;"),
    "pp_momentum_order": ("const int qk1 = kminus(d, q, k1), qk2 = kminus(d, q, k2);",
                          "const int qk1 = kminus(d, k1, q), qk2 = kminus(d, k2, q);"),
    "pp_swapped_arguments": ("term += gat(G[sp], Nw2, N, qk2, f2, qk1, f1)",
                             "term += gat(G[sp], Nw2, N, qk1, f1, qk2, f2)"),
    "transverse_same_spin": ("term -= gat(G[1 - sp], Nw2, N, k2, n2, k1, n1)",
                             "term -= gat(G[sp], Nw2, N, k2, n2, k1, n1)"),
    "transverse_sign": ("term -= gat(G[1 - sp]", "term += gat(G[1 - sp]"),
    # the step before: non-uniform Fourier transform of a vertex configuration
    "nfft_time_sign": ("const double ph1 = w1 * tau[i] - (kx1 * xi + ky1 * yi);\n                const cplx e1",
                       "const double ph1 = -w1 * tau[i] - (kx1 * xi + ky1 * yi);\n                const cplx e1"),
    "nfft_momentum_sign": ("const double ph1 = w1 * tau[i] - (kx1 * xi + ky1 * yi);\n                const cplx e1",
                           "const double ph1 = w1 * tau[i] + (kx1 * xi + ky1 * yi);\n                const cplx e1"),
    "nfft_bosonic_grid": ("const double w1 = (2.0 * (n1 - d->Nw) + 1.0) * pi / beta;\n            const double w2 = (2.0 * (n2 - d->Nw) + 1.0) * pi / beta;\n            cplx acc = 0.0;\n            for (int i = 0; i < n; ++i) {\n                const int xi",
                          "const double w1 = (2.0 * (n1 - d->Nw)) * pi / beta;\n            const double w2 = (2.0 * (n2 - d->Nw)) * pi / beta;\n            cplx acc = 0.0;\n            for (int i = 0; i < n; ++i) {\n                const int xi"),
    "nfft_no_conjugate": ("const cplx e2 = cos(ph2) - I * sin(ph2);\n                    acc += e1 * mt[(size_t)i * n + j] * e2;\n                }\n            }\n            out[(size_t)K1",
                          "const cplx e2 = cos(ph2) + I * sin(ph2);\n                    acc += e1 * mt[(size_t)i * n + j] * e2;\n                }\n            }\n            out[(size_t)K1"),
    "nfft_normalisation": ("out[(size_t)K1 * N + K2] = acc / (beta * Nc);", "out[(size_t)K1 * N + K2] = acc / beta;"),
    "nfft_transposed": ("acc += e1 * mt[(size_t)i * n + j] * e2;\n                }\n            }\n            out[(size_t)K1",
                        "acc += e1 * mt[(size_t)j * n + i] * e2;\n                }\n            }\n            out[(size_t)K1"),
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
