"""Deferred staging (options.deferred): the tensor-core operands of a batch are
formed from the staged measurements' M directly when the batch accumulates.
Checked against the CPU oracle element by element (Eq. (3) norm and per-entry
bounds, exact structural zeros) and against the same run staged eagerly,
which forms every G~ with the same FP32 arithmetic and therefore the same
operands."""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import (TOL, check_entries, cuda, draw, ensure_built, exported_to_slabs,
                      oracle_full, run_lib)

pytestmark = pytest.mark.gpu

P = inputs.Problem

SHAPES = [
    (2, 2, 8, 3, 3, 37, 16),     # several batches, ragged tail, Nkex < Nc
    (1, 1, 1, 3, 1, 5, 4),       # Nc = 1, 2Nw = 2, Nwex > 2Nw
    (4, 2, 4, 2, 8, 9, 4),       # non-square cluster
    (3, 3, 6, 5, 9, 20, 7),      # odd cluster, Nwex = 5, 2Nw = 12 (rows per block not a power of two)
    (2, 2, 16, 8, 2, 12, 12),    # 2Nw = 32, Nkex < Nc
    (4, 4, 4, 16, 16, 6, 6),     # Nwex = 16: the widest tensor-core window
    (1, 2, 64, 2, 2, 5, 5),      # 2Nw = 128: one row of M per block
]


def _check(p, channel="ph_magnetic", operands="fp16", batch=None, seed=0, own_g0=False, **kw):
    M, G0, s = draw(p, seed=seed)
    got, S, h = run_lib(p, M, G0, s, "mixed", batch=batch, channel=channel, exchange="tensor_cores",
                        operands=operands, deferred=True, own_g0=own_g0, **kw)
    h.close()
    ref, Sref = oracle_full(p, M, G0, s, channel=channel)
    assert S == Sref
    err = oracle.errors(ref, got)
    assert err["L2"] <= TOL["mixed"], err
    ref_s, msel = exported_to_slabs(p, ref)
    got_s, _ = exported_to_slabs(p, got)
    check_entries(p, ref_s, got_s, msel, TOL["mixed"], channel)
    return got


@pytest.mark.parametrize("operands", ["fp16", "tf32"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
@pytest.mark.parametrize("shape", SHAPES)
def test_deferred_matches_oracle(shape, channel, operands):
    Lx, Ly, Nw, Nwex, Nkex, R, batch = shape
    _check(P(Lx, Ly, Nw, Nwex, Nkex, 8.0, R, batch), channel=channel, operands=operands)


@pytest.mark.parametrize("m_dtype", ["c128", "c64"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
def test_deferred_equals_eager(channel, m_dtype):
    """The same measurements staged both ways.  In one batch both form G~ with
    one FP32 routine and take the operand scale from the batch's own largest
    component, so the results are identical; over several batches the
    deferred handle keeps its scale while it stays within one binade of the
    batch's own (other roundings of the pairs' low parts), and the two agree
    far inside the mixed bound."""
    p = P(2, 2, 8, 4, 4, 10.0, 45, 16, m_dtype=m_dtype)
    M, G0, s = draw(p, seed=3)
    for R in (16, 45):
        eager, S1, h1 = run_lib(p, M[:R], G0, s[:R], "mixed", channel=channel,
                                exchange="tensor_cores")
        h1.close()
        dfr, S2, h2 = run_lib(p, M[:R], G0, s[:R], "mixed", channel=channel,
                              exchange="tensor_cores", deferred=True)
        h2.close()
        assert S1 == S2
        if R == 16:
            assert np.array_equal(dfr, eager)
        else:
            assert oracle.errors(eager, dfr)["L2"] <= 1e-6


def test_deferred_own_G0_per_measurement():
    """Every measurement with its own G0 array (the kernels then read each
    slot's G0): the same result as one shared G0 with the same values."""
    p = P(2, 2, 8, 3, 4, 10.0, 21, 8)
    a = _check(p)
    b = _check(p, own_g0=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown"])
def test_deferred_batch_max(channel):
    """Largest batch (256 slots in the kernels' slot table)."""
    _check(P(2, 2, 2, 2, 4, 5.0, 300, 256), channel=channel)


@pytest.mark.parametrize("M_scale", [1e-4, 1e6])
def test_deferred_operand_range(M_scale):
    p = P(2, 2, 8, 4, 4, 10.0, 21, 8)
    M, G0, s = draw(p)
    M = M * M_scale
    got, S, h = run_lib(p, M, G0, s, "mixed", exchange="tensor_cores", deferred=True)
    h.close()
    ref, _ = oracle_full(p, M, G0, s)
    assert oracle.errors(ref, got)["L2"] <= TOL["mixed"]


@pytest.mark.parametrize("direct_batches", [1, 2])
def test_deferred_direct_window(direct_batches):
    """The direct term's window filled from M over several batches (flushed
    in the run and at g4_finalize)."""
    _check(P(2, 2, 8, 4, 4, 10.0, 53, 8), direct_batches=direct_batches)


def test_deferred_transfer_slab():
    """A slab of the transfer frequencies (one rank's share of G4)."""
    p = P(2, 2, 8, 5, 4, 10.0, 19, 8)
    M, G0, s = draw(p)
    full, _ = oracle_full(p, M, G0, s)
    full = full.reshape(p.Nwex, -1)
    got, S, h = run_lib(p, M, G0, s, "mixed", exchange="tensor_cores", deferred=True,
                        wex_slab=(1, 3))
    h.close()
    ref = full[1:4].reshape(-1)
    assert oracle.errors(ref, got.reshape(-1))["L2"] <= TOL["mixed"]


def test_deferred_refusals():
    """What a deferred handle does not take: the FP64 path, the CUDA-core
    exchange, vertex staging and grouped accumulation."""
    torch = cuda()
    g4 = ensure_built()
    p = P(2, 2, 4, 2, 4, 10.0, 4, 4)
    with pytest.raises(g4.G4Error):
        g4.G4.for_problem(p, precision="fp64", batch=4, deferred=True)
    with pytest.raises(g4.G4Error):
        g4.G4.for_problem(p, precision="mixed", batch=4, deferred=True, exchange="cuda_cores")
    h = g4.G4.for_problem(p, precision="mixed", batch=4, deferred=True)
    dev = torch.device("cuda")
    G0 = torch.from_numpy(inputs.g0(p)).to(dev)
    tau = torch.zeros(2, dtype=torch.float64, device=dev)
    site = torch.zeros(2, dtype=torch.int32, device=dev)
    Mtau = torch.ones(2, dtype=torch.float64, device=dev)
    with pytest.raises(g4.G4Error):
        h.compute_G_vertices(p.beta, 1, 1, tau, site, Mtau, G0, 1.0)
    with pytest.raises(g4.G4Error):
        g4.accumulate_group([h])
    h.close()


@pytest.mark.parametrize("operands", ["fp16", "tf32"])
def test_deferred_scale_changes_between_batches(operands):
    """Batches whose G differ in magnitude by orders (M scaled by 1, 1e4,
    1e-3, 1, ...): the kept FP16 scale must be replaced (the batch's operands
    formed again) whenever the batch's largest component leaves its binade,
    and kept otherwise; every batch stays within the mixed bound."""
    p = P(2, 2, 8, 4, 4, 10.0, 40, 8)
    M, G0, s = draw(p, seed=5)
    factors = [1.0, 1e4, 1e-3, 1.0, 1.0]
    for b, f in enumerate(factors):
        M[b * 8:(b + 1) * 8] *= f
    got, S, h = run_lib(p, M, G0, s, "mixed", exchange="tensor_cores", operands=operands,
                        deferred=True)
    h.close()
    ref, Sref = oracle_full(p, M, G0, s)
    assert S == Sref
    err = oracle.errors(ref, got)
    assert err["L2"] <= TOL["mixed"], err
    ref_s, msel = exported_to_slabs(p, ref)
    got_s, _ = exported_to_slabs(p, got)
    check_entries(p, ref_s, got_s, msel, TOL["mixed"])
