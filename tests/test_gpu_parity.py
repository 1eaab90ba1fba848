"""GPU path against the CPU oracle, element by element (Eq. (3) relative
Frobenius error, with Eq. (2) reported), through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import (TOL, check_entries, cuda, draw, ensure_built, exported_to_slabs,
                      oracle_full, oracle_slabs, run_lib)

pytestmark = pytest.mark.gpu

P = inputs.Problem


def _check(p, precision, batch=None, seed=0, R=None, channel="ph_magnetic", exchange="auto",
           operands="fp16", M_scale=1.0, accum="fp64"):
    M, G0, s = draw(p, seed=seed, R=R)
    M = M * M_scale
    got, S, h = run_lib(p, M, G0, s, precision, batch=batch, channel=channel, exchange=exchange,
                        operands=operands, accum=accum)
    ref, Sref = oracle_full(p, M, G0, s, channel=channel)
    assert S == Sref
    err = oracle.errors(ref, got)
    assert err["L2"] <= TOL[precision], err
    ref_s, msel = exported_to_slabs(p, ref)
    got_s, _ = exported_to_slabs(p, got)
    check_entries(p, ref_s, got_s, msel, TOL[precision], channel)
    h.close()
    return err


def test_build_G_matches_oracle():
    torch = cuda()
    g4 = ensure_built()
    p = P(4, 4, 4, 1, 1, 10.0, 1, 1)
    M, G0, _ = draw(p, R=1)
    Gd = g4.build_G(M[0].cuda(), torch.from_numpy(G0).cuda())
    got = Gd.cpu().numpy()
    for sp in range(2):
        ref = oracle.build_G(M[0, sp].numpy(), G0[sp])
        assert np.abs(got[sp] - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiny_2x2_full(precision):
    _check(inputs.workload("tiny_2x2"), precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [
    (2, 2, 8, 3, 3, 37, 16),     # several batches, ragged tail
    (1, 1, 1, 3, 1, 5, 4),       # Nc = 1, 2Nw = 2, Nwex > 2Nw
    (4, 2, 4, 2, 8, 9, 4),       # non-square cluster
    (3, 3, 6, 5, 9, 20, 7),      # odd cluster, Nwex = 5 (two m chunks)
    (2, 2, 16, 8, 2, 12, 12),    # 2Nw = 32, Nkex < Nc
])
def test_small_shapes(precision, shape):
    Lx, Ly, Nw, Nwex, Nkex, R, batch = shape
    _check(P(Lx, Ly, Nw, Nwex, Nkex, 8.0, R, batch), precision)


SHAPES_X = [
    (2, 2, 8, 3, 3, 37, 16),     # several batches, ragged tail, Nkex < Nc
    (1, 1, 1, 3, 1, 5, 4),       # Nc = 1, 2Nw = 2, Nwex > 2Nw
    (4, 2, 4, 2, 8, 9, 4),       # non-square cluster
    (3, 3, 6, 5, 9, 20, 7),      # odd cluster, Nwex = 5
    (2, 2, 16, 8, 2, 12, 12),    # 2Nw = 32, Nkex < Nc
    (4, 4, 4, 16, 16, 6, 6),     # Nwex = 16: the widest tensor-core window (one row frequency)
]


@pytest.mark.parametrize("exchange", ["cuda_cores", "tensor_cores", "tensor_cores_tf32"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
@pytest.mark.parametrize("shape", SHAPES_X)
def test_exchange_kernels(exchange, channel, shape):
    """Both exchange kernels of the mixed path (tensor cores with FP16 and with
    TF32 operand pairs), every channel."""
    Lx, Ly, Nw, Nwex, Nkex, R, batch = shape
    ops = "tf32" if exchange.endswith("tf32") else "fp16"
    _check(P(Lx, Ly, Nw, Nwex, Nkex, 8.0, R, batch), "mixed", channel=channel,
           exchange=exchange.replace("_tf32", ""), operands=ops)


@pytest.mark.parametrize("operands", ["fp16", "tf32"])
@pytest.mark.parametrize("M_scale", [1e-4, 1e3, 1e6])
def test_operand_range(operands, M_scale):
    """G spanning very different magnitudes (M scaled by 1e-4 .. 1e6: G from
    about G0 up to entries far beyond the FP16 maximum of 65504): the FP16
    pairs' power-of-two scale keeps the mixed path within its bound."""
    _check(P(2, 2, 8, 4, 4, 10.0, 21, 8), "mixed", operands=operands, M_scale=M_scale)


def test_mixed_complex64_input():
    p = P(2, 2, 4, 4, 4, 10.0, 10, 8, m_dtype="c64")
    _check(p, "mixed")


@pytest.mark.parametrize("exchange", ["cuda_cores", "tensor_cores", "tensor_cores_tf32"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
def test_mixed_batch_max(channel, exchange):
    """Largest batch (256): the longest FP32 sums inside one accumulation."""
    ops = "tf32" if exchange.endswith("tf32") else "fp16"
    _check(P(2, 2, 2, 2, 4, 5.0, 300, 256), "mixed", channel=channel,
           exchange=exchange.replace("_tf32", ""), operands=ops)


@pytest.mark.parametrize("operands", ["fp16", "tf32"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "ph_density"])
def test_mixed_zeeman_split(channel, operands):
    """Spin-split G0 (Zeeman field): the direct term's Q = 0 operands then carry
    the coherent G0 part of every measurement."""
    _check(P(4, 4, 8, 4, 16, 20.0, 64, 64, h=0.3), "mixed", channel=channel, operands=operands)


def _sampled(p, precision, R, qsel, msel, batch=None, tol=None, channel="ph_magnetic",
             exchange="auto"):
    M, G0, s = draw(p, R=R)
    got, S, h = run_lib(p, M, G0, s, precision, batch=batch, channel=channel, exchange=exchange)
    h.close()
    ref, Sref = oracle_slabs(p, M, G0, s, qsel, msel, channel=channel)
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    sub = oracle.slabs_from_exported(d, got, qsel, msel)
    err = oracle.errors(ref, sub)
    assert err["L2"] <= (tol or TOL[precision]), err
    check_entries(p, ref, sub, msel, tol or TOL[precision], channel)
    return err


def test_c16_w64_fp64_sampled_slabs():
    """4x4 cluster, 2Nw = 64, Nwex = 8, Nkex = 16 at full size; 8 (q, m) slabs
    checked against the oracle on a 32-measurement prefix."""
    p = inputs.workload("c16_w64")
    _sampled(p, "fp64", 32, [0, 3, 5, 15, 7, 9, 12, 1], [0, 7, 2, 4, 1, 5, 6, 3], batch=32)


@pytest.mark.parametrize("exchange", ["cuda_cores", "tensor_cores"])
def test_c16_w64_mixed_sampled_slabs(exchange):
    p = inputs.workload("c16_w64")
    _sampled(p, "mixed", 96, [0, 3, 5, 15, 7, 9, 12, 1], [0, 7, 2, 4, 1, 5, 6, 3], batch=64,
             exchange=exchange)


@pytest.mark.slow
def test_c36_w64_mixed_sampled_slabs():
    """6x6 cluster, 2Nw = 64, Nwex = 8, Nkex = 36, batches of 64 as the
    benchmark runs them; 6 slabs on a 128-measurement prefix."""
    p = inputs.workload("c36_w64")
    _sampled(p, "mixed", 128, [0, 35, 7, 20, 14, 1], [0, 7, 3, 5, 1, 6], batch=64)


@pytest.mark.slow
@pytest.mark.parametrize("staging", ["deferred", "eager"])
def test_c64_w64_mixed_sampled_slabs(staging):
    """8x8 cluster, 2Nw = 64, Nwex = 4, Nkex = 64, complex64 M, batches of 128
    as the benchmark runs them: the full-size G4 (4.3 G entries, one 69 GB FP64
    accumulator and a 69 GB result), checked on 3 slabs read back one by one.
    136 measurements (a full batch of 128 and a ragged one of 8) with a
    direct-term window of one batch, so that the window is added once in the
    run and once at g4_finalize.  M is generated, uploaded and fed to the
    oracle one measurement at a time (with deferred staging each batch's M
    stay on the device until the batch is accumulated)."""
    torch = cuda()
    g4 = ensure_built()
    p = inputs.workload("c64_w64")
    R, qsel, msel = 136, [0, 63, 27], [0, 3, 2]
    G0 = inputs.g0(p)
    s = inputs.signs(p, seed=0)[:R]
    deferred = staging == "deferred"
    h = g4.G4.for_problem(p, precision="mixed", batch=128, direct_batches=1, deferred=deferred)
    G0d = torch.from_numpy(np.ascontiguousarray(G0)).cuda()
    held = []
    for r in range(R):
        Md = inputs.measurement_M(p, r, seed=0).cuda()
        h.compute_G(Md, G0d, float(s[r]))
        if deferred:
            held.append(Md)
            if len(held) == 128:
                h.accumulate()
                held = []
        del Md
    res, S = h.finalize()
    del held
    h.close()
    v = res.view(p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc)
    sub = np.stack([v[m, :, :, q].cpu().numpy() for q, m in zip(qsel, msel)])
    del res, v
    torch.cuda.empty_cache()
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    meas = ((inputs.measurement_M(p, r, seed=0).numpy().astype(np.complex128), s[r]) for r in range(R))
    ref, Sref = oracle.run_stream(d, meas, G0, np.asarray(qsel, np.int32), np.asarray(msel, np.int32))
    assert S == Sref
    err = oracle.errors(ref, sub)
    assert err["L2"] <= TOL["mixed"], err
    check_entries(p, ref, sub, msel, TOL["mixed"])


@pytest.mark.parametrize("operands", ["fp16", "tf32"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "ph_density"])
@pytest.mark.parametrize("direct_batches", [1, 2, 3])
def test_direct_window_flushes(channel, direct_batches, operands):
    """The direct term held over windows of 1, 2 and 3 batches: flushes in the
    middle of the run (including after a ragged batch) and at g4_finalize all
    match the oracle."""
    p = P(2, 2, 8, 3, 4, 8.0, 37, 4)
    M, G0, s = draw(p, seed=2)
    g4 = ensure_built()
    h = g4.G4.for_problem(p, precision="mixed", channel=channel, direct_batches=direct_batches,
                          operands=operands)
    got, S, h = run_lib(p, M, G0, s, "mixed", handle=h, channel=channel)
    h.close()
    ref, Sref = oracle_full(p, M, G0, s, channel=channel)
    assert S == Sref
    assert oracle.errors(ref, got)["L2"] <= TOL["mixed"]
    ref_s, msel = exported_to_slabs(p, ref)
    got_s, _ = exported_to_slabs(p, got)
    check_entries(p, ref_s, got_s, msel, TOL["mixed"], channel)


CHANNELS = ["pp_updown", "ph_density", "ph_transverse"]


@pytest.mark.parametrize("channel", CHANNELS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [
    (2, 2, 8, 3, 3, 37, 16),     # several batches, ragged tail, Nkex < Nc
    (1, 1, 1, 3, 1, 5, 4),       # Nc = 1, 2Nw = 2, Nwex > 2Nw
    (4, 2, 4, 2, 8, 9, 4),       # non-square cluster
    (3, 3, 6, 5, 9, 20, 7),      # odd cluster, Nwex = 5
])
def test_other_channels_small(channel, precision, shape):
    Lx, Ly, Nw, Nwex, Nkex, R, batch = shape
    _check(P(Lx, Ly, Nw, Nwex, Nkex, 8.0, R, batch), precision, channel=channel)


@pytest.mark.parametrize("channel", CHANNELS)
def test_other_channels_c16_w64_sampled(channel):
    """4x4 cluster, 2Nw = 64, Nwex = 8, Nkex = 16 at full size, mixed path, 6 slabs, 64-measurement prefix."""
    p = inputs.workload("c16_w64")
    _sampled(p, "mixed", 64, [0, 3, 15, 7, 9, 1], [0, 7, 4, 1, 5, 3], batch=64, channel=channel)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
def test_selection_rule_k_diagonal_M(precision, channel):
    """A translation-invariant configuration (M diagonal in momentum) makes G
    momentum-diagonal, so G4 vanishes exactly wherever k1 != k2 and, for the
    direct term, q != 0 (particle-particle: wherever k1 != k2).  The library
    must produce exact zeros there (a wrong momentum shift in any kernel
    would put products of non-zero blocks there) and match the oracle
    elsewhere."""
    p = P(3, 2, 4, 3, 6, 8.0, 11, 4)
    M, G0, s = draw(p, seed=3)
    kk = np.arange(p.N) // p.Nw2
    M = M * torch_mask(kk[:, None] == kk[None, :])
    got, S, h = run_lib(p, M, G0, s, precision, channel=channel)
    h.close()
    ref, Sref = oracle_full(p, M, G0, s, channel=channel)
    assert S == Sref
    assert oracle.errors(ref, got)["L2"] <= TOL[precision]
    e = got.reshape(p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc)
    k1 = np.arange(p.Nc)[None, :]
    k2 = np.arange(p.Nc)[:, None]
    q = np.arange(p.Nkex)[:, None, None]
    if channel in ("ph_magnetic", "ph_density"):
        zero = (k1 != k2) & (q != 0)
    else:
        zero = np.broadcast_to(k1 != k2, (p.Nkex, p.Nc, p.Nc))
    assert np.all(e[:, :, :, zero] == 0)
    assert np.all(ref.reshape(e.shape)[:, :, :, zero] == 0)


def torch_mask(mask):
    import torch
    return torch.from_numpy(mask.astype(np.float64))


@pytest.mark.slow
@pytest.mark.parametrize("operands", ["fp16", "tf32"])
def test_c16_w64_long_direct_window(operands):
    """4x4 cluster, 2Nw = 64, Nwex = 8, Nkex = 16, batches of 64 with a
    direct-term window of 16 batches: the direct GEMM sums 1024 measurements
    in FP32 before its one flush (the longest window the default settings
    make: 8 batches of 128); 6 slabs against the oracle."""
    p = inputs.workload("c16_w64")
    M, G0, s = draw(p, R=1024)
    g4 = ensure_built()
    h = g4.G4.for_problem(p, precision="mixed", batch=64, direct_batches=16, operands=operands)
    got, S, h = run_lib(p, M, G0, s, "mixed", handle=h)
    h.close()
    qsel, msel = [0, 3, 15, 7, 9, 1], [0, 7, 4, 1, 5, 3]
    ref, Sref = oracle_slabs(p, M, G0, s, qsel, msel)
    assert S == Sref
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    sub = oracle.slabs_from_exported(d, got, qsel, msel)
    err = oracle.errors(ref, sub)
    assert err["L2"] <= TOL["mixed"], err
    check_entries(p, ref, sub, msel, TOL["mixed"])


@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
@pytest.mark.parametrize("shape", [
    (2, 2, 8, 3, 3, 37, 16),     # several batches, ragged tail, Nkex < Nc
    (3, 3, 6, 5, 9, 20, 7),      # odd cluster, Nwex = 5
    (4, 4, 4, 16, 16, 6, 6),     # Nwex = 16
])
def test_accumulator_of_fp32_pairs(channel, shape):
    """The mixed path with the running sums in compensated FP32 pairs instead of
    FP64: the same element checks (the exchange epilogue and the direct-term
    merge add into the pairs; the finalize sums them in FP64)."""
    Lx, Ly, Nw, Nwex, Nkex, R, batch = shape
    _check(P(Lx, Ly, Nw, Nwex, Nkex, 8.0, R, batch), "mixed", channel=channel, accum="f32pair")


@pytest.mark.slow
@pytest.mark.parametrize("workload,R,qsel,msel", [
    ("c36_w64", 256, [0, 35, 7, 20], [0, 7, 3, 5]),
    ("c64_w64", 136, [0, 63, 27], [0, 3, 2]),
])
def test_accumulator_choice_measured(workload, R, qsel, msel):
    """FP64 against compensated FP32-pair accumulation on the benchmark's shapes
    (sampled slabs of a several-batch prefix): both within the bound; the
    errors, printed, are what the choice of the accumulator rests on."""
    torch = cuda()
    g4 = ensure_built()
    p = inputs.workload(workload)
    G0 = inputs.g0(p)
    s = inputs.signs(p, seed=0)[:R]
    G0d = torch.from_numpy(np.ascontiguousarray(G0)).cuda()
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    subs = {}
    for accum in ("fp64", "f32pair"):
        h = g4.G4.for_problem(p, precision="mixed", accum=accum, direct_batches=1)
        for r in range(R):
            h.compute_G(inputs.measurement_M(p, r, seed=0).cuda(), G0d, float(s[r]))
        res, S = h.finalize()
        h.close()
        v = res.view(p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc)
        subs[accum] = np.stack([v[m, :, :, q].cpu().numpy() for q, m in zip(qsel, msel)])
        del res, v
        torch.cuda.empty_cache()
    meas = ((inputs.measurement_M(p, r, seed=0).numpy().astype(np.complex128), s[r]) for r in range(R))
    ref, Sref = oracle.run_stream(d, meas, G0, np.asarray(qsel, np.int32), np.asarray(msel, np.int32))
    for accum, sub in subs.items():
        err = oracle.errors(ref, sub)
        print("accumulator %s on %s: L2 %.3e L1 %.3e" % (accum, workload, err["L2"], err["L1"]))
        assert err["L2"] <= TOL["mixed"], (accum, err)
        check_entries(p, ref, sub, msel, TOL["mixed"])
    diff = oracle.errors(subs["fp64"], subs["f32pair"])
    print("FP64 vs FP32 pairs on %s: L2 %.3e" % (workload, diff["L2"]))
