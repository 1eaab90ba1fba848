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
            exchange="auto"):
    torch = cuda()
    g4 = ensure_built()
    h = handle or g4.G4.for_problem(p, precision=precision, batch=batch or p.batch, channel=channel,
                                    exchange=exchange)
    G0d = torch.from_numpy(np.ascontiguousarray(G0)).cuda()
    for r in range(len(s)):
        h.compute_G(M[r].cuda(), G0d, float(s[r]))
    res, S = h.finalize(out=out)
    torch.cuda.synchronize()
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
