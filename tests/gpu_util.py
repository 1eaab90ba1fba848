"""Helpers shared by the GPU tests: run the library on seeded inputs and the
oracle on the same bytes."""
import numpy as np

import oracle
from paper_2105_00027_gb300 import inputs

TOL = {"fp64": 1e-11, "mixed": 2e-6}


def cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def ensure_built():
    from paper_2105_00027_gb300 import build, g4
    build.build()
    return g4


def dims_of(p):
    return oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)


def draw(p, seed=0, R=None, problem_index=0):
    R = p.R if R is None else R
    M = inputs.batch_M(p, 0, R, seed=seed, problem_index=problem_index)
    s = inputs.signs(p, seed=seed, problem_index=problem_index)[:R]
    return M, inputs.g0(p), s


def run_lib(p, M, G0, s, precision, batch=None, handle=None, out=None, channel="ph_magnetic",
            exchange="auto", operands="fp16", accum="fp64", deferred=False, own_g0=False,
            **kw):
    """Stage every measurement through g4_compute_G and finalise.  A deferred
    handle reads M (and G0) only when the batch accumulates, so every M stays
    on the device until g4_finalize has returned; own_g0 gives each
    measurement its own device copy of G0 (the handle then reads each slot's
    G0 instead of one shared array)."""
    torch = cuda()
    g4 = ensure_built()
    h = handle or g4.G4.for_problem(p, precision=precision, batch=batch or p.batch, channel=channel,
                                    exchange=exchange, operands=operands, accum=accum,
                                    deferred=deferred, **kw)
    G0d = torch.from_numpy(np.ascontiguousarray(G0)).cuda()
    keep = []
    for r in range(len(s)):
        Md = M[r].cuda()
        g0r = G0d.clone() if own_g0 else G0d
        if deferred:
            keep.append((Md, g0r))
        h.compute_G(Md, g0r, float(s[r]))
    res, S = h.finalize(out=out)
    torch.cuda.synchronize()
    del keep
    return res.cpu().numpy(), S, h


def oracle_full(p, M, G0, s, channel="ph_magnetic"):
    d = dims_of(p)
    Mn = M.numpy().astype(np.complex128)
    slabs, S = oracle.run(d, Mn, G0, s, channel=channel)
    return oracle.to_exported(d, slabs), S


def oracle_slabs(p, M, G0, s, qsel, msel, nthreads=0, channel="ph_magnetic"):
    d = dims_of(p)
    meas = ((M[r].numpy().astype(np.complex128), s[r]) for r in range(len(s)))
    return oracle.run_stream(d, meas, G0, np.asarray(qsel, np.int32), np.asarray(msel, np.int32),
                             nthreads=nthreads, channel=channel)


def structural_zero_mask(Nw2, msel, channel="ph_magnetic"):
    """[s][n2][n1] mask of the entries that the definition makes exactly zero
    in slab s (transfer frequency msel[s]): a G factor whose frequency leaves
    the grid.  Particle-hole channels: n1 + m or n2 + m >= 2Nw; particle-particle
    (Q - K has frequency index m + 2Nw - 1 - n): n1 < m or n2 < m."""
    n = np.arange(Nw2)
    out = []
    for m in msel:
        if channel == "pp_updown":
            bad = n < m
        else:
            bad = n + m >= Nw2
        out.append(bad[:, None] | bad[None, :])
    return np.stack(out)


def check_entries(p, ref_slabs, got_slabs, msel, tol, channel="ph_magnetic"):
    """Element checks beyond the global norm (Eq. 3): per (q, m) slab every
    entry within tol of that slab's largest reference entry, and the entries
    the definition forces to zero exactly zero on both sides.  Slabs are
    [s][n2][n1][k2][k1]."""
    ref = np.asarray(ref_slabs).reshape(len(msel), p.Nw2, p.Nw2, p.Nc, p.Nc)
    got = np.asarray(got_slabs).reshape(ref.shape)
    zero = structural_zero_mask(p.Nw2, msel, channel)
    for s in range(len(msel)):
        scale = np.abs(ref[s]).max()
        dev = np.abs(got[s] - ref[s]).max()
        assert dev <= tol * max(scale, 1e-300), ("slab", s, dev, scale)
        assert np.all(ref[s][zero[s]] == 0), ("oracle non-zero where the definition is zero", s)
        assert np.all(got[s][zero[s]] == 0), ("non-zero where the definition is zero", s)


def exported_to_slabs(p, exported):
    """Exported [m][n2][n1][q][k2][k1] -> slabs [q-major Q][n2][n1][k2][k1] and msel."""
    e = np.asarray(exported).reshape(p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc)
    slabs = np.ascontiguousarray(e.transpose(3, 0, 1, 2, 4, 5)).reshape(
        p.Nkex * p.Nwex, p.Nw2, p.Nw2, p.Nc, p.Nc)
    msel = np.tile(np.arange(p.Nwex), p.Nkex)
    return slabs, msel
