"""The CPU oracle against closed forms, brute-force Wick contraction,
symmetries and library special cases (no GPU)."""
import numpy as np
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("name", list(P.PINS))
def test_pin(lib, name):
    fn, tol = P.PINS[name]
    err = fn(lib)
    assert err <= tol, (name, err)


def test_kplus_matches_vector_sum(lib):
    for Lx, Ly in ((1, 1), (2, 2), (4, 2), (6, 6), (3, 5)):
        p = P.problem(Lx, Ly, 1, 1, Lx * Ly)
        d = P.dims_of(p)
        for a in range(p.Nc):
            for b in range(p.Nc):
                assert lib.g4o_kplus(d, a, b) == P.kplus_vec(p, a, b)


def test_zero_sign_sum_returns_unnormalised(lib):
    p = P.problem(2, 2, 2, 2, 4, R=2)
    M, G0, _ = P.draw(p)
    s = np.array([1.0, -1.0])
    d = P.dims_of(p)
    slabs, S = oracle.run(d, M, G0, s, lib=lib)
    assert S == 0.0
    a, _ = oracle.run(d, M[:1], G0, s[:1], lib=lib)
    b, _ = oracle.run(d, M[1:], G0, s[1:], lib=lib)
    np.testing.assert_allclose(slabs, a * 1.0 + b * -1.0, rtol=1e-12, atol=1e-14)


def test_transfer_beyond_grid_is_zero(lib):
    """Nwex > 2Nw: every m >= 2Nw slab vanishes (G is zero off the grid)."""
    p = P.problem(2, 1, 1, 4, 2, R=3)
    M, G0, s = P.draw(p)
    g4, _ = P.full(p, M, G0, s, lib)
    assert np.abs(g4[p.Nw2:]).max() == 0.0
    assert np.abs(g4[:p.Nw2]).max() > 0.0


def test_stream_matches_run(lib):
    p = P.problem(2, 2, 2, 2, 3, R=3)
    M, G0, s = P.draw(p)
    d = P.dims_of(p)
    qs, ms = np.array([0, 2, 1], np.int32), np.array([1, 0, 1], np.int32)
    a, Sa = oracle.run(d, M, G0, s, qs, ms, lib=lib)
    b, Sb = oracle.run_stream(d, zip(M, s), G0, qs, ms, lib=lib)
    assert Sa == Sb
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)


def test_errors_metric_values():
    """Eqs. (2)-(3) on vectors whose norms are known in closed form."""
    ref = np.array([3 + 4j, 0, -5, 12j])
    test = ref + np.array([1, 0, 0, -1j])
    e = oracle.errors(ref, test)
    assert abs(e["L1"] - 2 / 22) < 1e-15
    assert abs(e["L2"] - np.sqrt(2) / np.sqrt(25 + 25 + 144)) < 1e-15
    assert abs(e["L1_re"] - 1 / 8) < 1e-15
    assert abs(e["L1_im"] - 1 / 16) < 1e-15
