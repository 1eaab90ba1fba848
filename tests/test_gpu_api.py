"""Behaviour of the C ABI on the GPU: state machine, sign-sum edge cases,
host output, checkpoint/restore, grouped accumulation, allocation limits."""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import TOL, cuda, draw, ensure_built, oracle_full, run_lib

pytestmark = pytest.mark.gpu

P = inputs.Problem


def _handle(p, precision, **kw):
    g4 = ensure_built()
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_restore_bitwise(precision, tmp_path):
    """Stop at a batch boundary, save, restore into a fresh handle, finish: the
    result equals an uninterrupted run bit for bit (the mixed path rounds per
    batch, so the boundary matters; the FP64 path updates per measurement)."""
    torch = cuda()
    p = P(2, 2, 4, 3, 4, 10.0, 24, 8)
    M, G0, s = draw(p)
    G0d = torch.from_numpy(G0).cuda()
    g4, h = _handle(p, precision)
    for r in range(p.R):
        h.compute_G(M[r].cuda(), G0d, s[r])
    ref, Sref = h.finalize()
    h.close()

    g4, h1 = _handle(p, precision)
    for r in range(16):
        h1.compute_G(M[r].cuda(), G0d, s[r])
    h1.checkpoint(tmp_path / "g4.ckpt")
    h1.close()
    g4, h2 = _handle(p, precision)
    h2.restore(tmp_path / "g4.ckpt")
    assert h2.query()[1] == 16
    for r in range(16, p.R):
        h2.compute_G(M[r].cuda(), G0d, s[r])
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


def test_accumulate_group_matches_individual():
    torch = cuda()
    g4 = ensure_built()
    probs = [P(2, 2, 4, 2, 4, 5.0, 10, 8), P(4, 2, 2, 3, 8, 10.0, 7, 8), P(3, 3, 3, 4, 9, 20.0, 5, 8)]
    data = [draw(p, problem_index=i) for i, p in enumerate(probs)]
    hs = [g4.G4.for_problem(p, precision="mixed") for p in probs]
    for i, (p, (M, G0, s)) in enumerate(zip(probs, data)):
        G0d = torch.from_numpy(G0).cuda()
        for r in range(p.R):
            hs[i].compute_G(M[r].cuda(), G0d, s[r])
    g4.accumulate_group(hs)
    for i, (p, (M, G0, s)) in enumerate(zip(probs, data)):
        out, S = hs[i].finalize()
        ref, Sref = oracle_full(p, M, G0, s)
        assert S == Sref
        assert oracle.errors(ref, out.cpu().numpy())["L2"] <= TOL["mixed"]
        hs[i].close()


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
