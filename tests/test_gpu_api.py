"""Behaviour of the C ABI on the GPU: state machine, sign-sum edge cases,
host output, checkpoint/restore, grouped accumulation, allocation limits."""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import TOL, check_entries, cuda, draw, ensure_built, oracle_full, run_lib

pytestmark = pytest.mark.gpu

P = inputs.Problem


def _handle(p, precision, **kw):
    """precision "mixed_f32pair": the mixed path with the accumulator of
    compensated FP32 pairs; "mixed_deferred": the mixed path with deferred
    staging (M must stay on the device until its batch is accumulated)."""
    g4 = ensure_built()
    if precision == "mixed_f32pair":
        precision, kw = "mixed", dict(kw, accum="f32pair")
    if precision == "mixed_deferred":
        precision, kw = "mixed", dict(kw, deferred=True)
    return g4, g4.G4.for_problem(p, precision=precision, **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_state_machine_and_reset(precision):
    torch = cuda()
    p = P(2, 2, 2, 2, 4, 5.0, 6, 4)
    M, G0, s = draw(p)
    g4, h = _handle(p, precision)
    G0d = torch.from_numpy(G0).cuda()
    for r in range(p.R):
        h.compute_G(M[r].cuda(), G0d, s[r])
    out1, S1 = h.finalize()
    with pytest.raises(g4.G4Error) as e:
        h.compute_G(M[0].cuda(), G0d, 1.0)
    assert e.value.status == g4.G4_ERR_STATE
    with pytest.raises(g4.G4Error):
        h.accumulate()
    with pytest.raises(g4.G4Error):
        h.finalize()
    h.reset()
    for r in range(p.R):
        h.compute_G(M[r].cuda(), G0d, s[r])
    out2, S2 = h.finalize()
    assert S1 == S2
    assert torch.equal(out1, out2)  # same inputs, same order: bitwise identical
    e_, n_ = h.query()
    assert e_ == p.entries and n_ == p.R
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_sign_sum_writes_unnormalised(precision):
    torch = cuda()
    p = P(2, 2, 2, 2, 4, 5.0, 2, 2)
    M, G0, _ = draw(p)
    s = np.array([1.0, -1.0])
    g4, h = _handle(p, precision)
    G0d = torch.from_numpy(G0).cuda()
    for r in range(2):
        h.compute_G(M[r].cuda(), G0d, s[r])
    out, S = h.finalize(allow_zero_sign=True)
    assert S == 0.0
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    a, _ = oracle.run(d, M[:1].numpy(), G0, s[:1])
    b, _ = oracle.run(d, M[1:].numpy(), G0, s[1:])
    ref = oracle.to_exported(d, a - b)
    err = oracle.errors(ref, out.cpu().numpy())
    assert err["L2"] <= TOL[precision], err
    h.close()


def test_finalize_to_host_buffer():
    torch = cuda()
    p = P(2, 2, 4, 3, 4, 10.0, 9, 8)
    M, G0, s = draw(p)
    g4, h = _handle(p, "mixed")
    G0d = torch.from_numpy(G0).cuda()
    for r in range(p.R):
        h.compute_G(M[r].cuda(), G0d, s[r])
    host = torch.empty((p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc), dtype=torch.complex128)
    out, S = h.finalize(out=host)
    ref, Sref = oracle_full(p, M, G0, s)
    assert S == Sref
    assert oracle.errors(ref, out.numpy())["L2"] <= TOL["mixed"]
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f32pair", "mixed_deferred"])
def test_checkpoint_restore_bitwise(precision, tmp_path):
    """Stop at a batch boundary, save, restore into a fresh handle, finish: the
    result equals an uninterrupted run bit for bit (the mixed path rounds per
    batch, so the boundary matters; the FP64 path updates per measurement)."""
    torch = cuda()
    p = P(2, 2, 4, 3, 4, 10.0, 24, 8)
    M, G0, s = draw(p)
    G0d = torch.from_numpy(G0).cuda()
    Md = M.cuda()   # resident: a deferred handle reads M when the batch accumulates
    g4, h = _handle(p, precision)
    for r in range(p.R):
        h.compute_G(Md[r], G0d, s[r])
    ref, Sref = h.finalize()
    h.close()

    g4, h1 = _handle(p, precision)
    for r in range(16):
        h1.compute_G(Md[r], G0d, s[r])
    h1.checkpoint(tmp_path / "g4.ckpt")
    h1.close()
    g4, h2 = _handle(p, precision)
    h2.restore(tmp_path / "g4.ckpt")
    assert h2.query()[1] == 16
    for r in range(16, p.R):
        h2.compute_G(Md[r], G0d, s[r])
    out, S = h2.finalize()
    assert S == Sref
    assert torch.equal(out, ref)
    # a checkpoint of another problem is rejected
    g4, h3 = _handle(P(2, 2, 4, 2, 4, 10.0, 4, 4), precision)
    with pytest.raises(g4.G4Error) as e:
        h3.restore(tmp_path / "g4.ckpt")
    assert e.value.status == g4.G4_ERR_INVALID
    h2.close()
    h3.close()


@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown"])
def test_accumulate_group_matches_individual(channel):
    """Several problems accumulated round by round with grouped launches: the
    rounds of equal shape relaunch the group's cached graph (the direct-term
    windows advancing as captured), the ragged last rounds capture new ones."""
    torch = cuda()
    g4 = ensure_built()
    probs = [P(2, 2, 4, 2, 4, 5.0, 26, 8), P(4, 2, 2, 3, 8, 10.0, 21, 8), P(3, 3, 3, 4, 9, 20.0, 35, 8)]
    data = [draw(p, problem_index=i) for i, p in enumerate(probs)]
    hs = [g4.G4.for_problem(p, precision="mixed", channel=channel, direct_batches=2) for p in probs]
    G0d = [torch.from_numpy(G0).cuda() for (_, G0, _) in data]
    rounds = max((p.R + p.batch - 1) // p.batch for p in probs)
    for b in range(rounds):
        for i, (p, (M, G0, s)) in enumerate(zip(probs, data)):
            for r in range(b * p.batch, min(p.R, (b + 1) * p.batch)):
                hs[i].compute_G(M[r].cuda(), G0d[i], s[r])
        g4.accumulate_group(hs)
    for i, (p, (M, G0, s)) in enumerate(zip(probs, data)):
        out, S = hs[i].finalize()
        ref, Sref = oracle_full(p, M, G0, s, channel=channel)
        assert S == Sref
        assert oracle.errors(ref, out.cpu().numpy())["L2"] <= TOL["mixed"]
        hs[i].close()


@pytest.mark.slow
def test_group12_all_problems_sampled():
    """The twelve-problem batching workload (Nc in {4, 8, 16, 36} x 2Nw in
    {16, 32, 64}, Nwex = 4, Nkex = Nc, batches of up to 64) accumulated with
    grouped launches as the benchmark runs it, on a prefix of at most 96
    measurements per problem (a full batch and a ragged one, so that the group
    graph is captured for both shapes); every problem checked against the
    oracle on 3 sampled (q, m) slabs (every slab for the small ones)."""
    torch = cuda()
    g4 = ensure_built()
    probs = [inputs.with_(p, R=min(p.R, 96)) for p in inputs.group_problems(seed=0)]
    hs = [g4.G4.for_problem(p, precision="mixed") for p in probs]
    G0s = [inputs.g0(p) for p in probs]
    G0d = [torch.from_numpy(g).cuda() for g in G0s]
    sg = [inputs.signs(p, seed=0, problem_index=i) for i, p in enumerate(probs)]
    rounds = max((p.R + p.batch - 1) // p.batch for p in probs)
    for b in range(rounds):
        for i, p in enumerate(probs):
            for r in range(b * p.batch, min(p.R, (b + 1) * p.batch)):
                M = inputs.measurement_M(p, r, seed=0, problem_index=i)
                hs[i].compute_G(M.cuda(), G0d[i], sg[i][r])
        g4.accumulate_group(hs)
    for i, p in enumerate(probs):
        out, S = hs[i].finalize()
        hs[i].close()
        d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
        if p.NQ <= 16:
            qsel, msel = oracle.all_slabs(d)
        else:
            qsel = np.array([0, p.Nkex - 1, p.Nkex // 2], np.int32)
            msel = np.array([0, 3, 1], np.int32)
        meas = ((inputs.measurement_M(p, r, seed=0, problem_index=i).numpy(), sg[i][r])
                for r in range(p.R))
        ref, Sref = oracle.run_stream(d, meas, G0s[i], qsel, msel)
        assert S == Sref
        sub = oracle.slabs_from_exported(d, out.cpu().numpy(), qsel, msel)
        err = oracle.errors(ref, sub)
        assert err["L2"] <= TOL["mixed"], (i, p, err)
        check_entries(p, ref, sub, msel, TOL["mixed"])


def test_allocation_limit_reports_oom():
    cuda()
    g4 = ensure_built()
    with pytest.raises(g4.G4Error) as e:
        g4.G4(16, 32, 8, 16, precision="mixed", mem_limit=1 << 20)
    assert e.value.status == g4.G4_ERR_OOM


def test_null_arguments_on_live_handle():
    torch = cuda()
    p = P(2, 2, 2, 1, 1, 5.0, 1, 1)
    g4, h = _handle(p, "mixed")
    import ctypes
    st = h.lib.g4_compute_G(h.h, None, None, 1.0)
    assert st == g4.G4_ERR_INVALID
    assert b"NULL" in h.lib.g4_last_error(h.h)
    assert h.lib.g4_profile_read(h.h, 99, None, None) == g4.G4_ERR_INVALID
    h.close()


@pytest.mark.parametrize("precision", ["mixed"])
def test_device_wait_budget_reports_timeout(precision):
    """Give every bounded device-side wait a budget far shorter than a copy
    takes: the kernels give up, record the timeout, drain their own copies and
    return; g4_finalize reports G4_ERR_TIMEOUT and the context stays usable."""
    torch = cuda()
    g4 = ensure_built()
    p = P(4, 4, 8, 4, 16, 10.0, 8, 8)
    M, G0, s = draw(p)
    G0d = torch.from_numpy(G0).cuda()
    h = g4.G4.for_problem(p, precision=precision, timeout_cycles=64)
    for r in range(p.R):
        h.compute_G(M[r].cuda(), G0d, s[r])
    with pytest.raises(g4.G4Error) as e:
        h.finalize()
    assert e.value.status == g4.G4_ERR_TIMEOUT
    h.close()
    # the device is still usable: a normal run on a fresh handle is correct
    got, S, h2 = run_lib(p, M, G0, s, precision)
    ref, Sref = oracle_full(p, M, G0, s)
    assert oracle.errors(ref, got)["L2"] <= TOL[precision]
    h2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown", "ph_density", "ph_transverse"])
def test_transfer_slabs_assemble_the_whole(precision, channel):
    """Handles holding slabs of the transfer frequencies (the partition of G4
    over ranks, Sec. 3.1), fed the same measurements on one GPU: their exported
    arrays are the whole problem's planes m = first .. first+count-1, and
    together they equal the oracle's G4 (and the single handle's)."""
    torch = cuda()
    g4 = ensure_built()
    p = P(3, 2, 4, 5, 6, 8.0, 19, 8)
    M, G0, s = draw(p, seed=6)
    ref, Sref = oracle_full(p, M, G0, s, channel=channel)
    whole, S, h = run_lib(p, M, G0, s, precision, channel=channel)
    h.close()
    parts = []
    for first, count in ((0, 2), (2, 1), (3, 2)):
        hs = g4.G4.for_problem(p, precision=precision, channel=channel, wex_slab=(first, count))
        got, S_s, hs = run_lib(p, M, G0, s, precision, handle=hs, channel=channel)
        hs.close()
        assert S_s == Sref
        assert got.shape[0] == count
        parts.append(got)
        sub = ref.reshape(p.Nwex, -1)[first:first + count]
        assert oracle.errors(sub, got.reshape(count, -1))["L2"] <= TOL[precision]
    joined = np.concatenate(parts, axis=0)
    assert oracle.errors(ref, joined)["L2"] <= TOL[precision]
    # the slabs sum the same products in the same order as the whole handle
    assert np.abs(joined - whole).max() <= TOL[precision] * np.abs(whole).max()


def test_transfer_slab_rejects_bad_ranges():
    cuda()
    g4 = ensure_built()
    for slab in ((3, 2), (-1, 1), (0, 5)):
        with pytest.raises(g4.G4Error) as e:
            g4.G4(4, 2, 4, 4, precision="mixed", wex_slab=slab)
        assert e.value.status == g4.G4_ERR_INVALID
