"""The allocation-free update entry point, checked on the GPU against the CPU
oracle and against the regular FP64 path of the library.

g4_update_noalloc exists for callers that cannot allocate device memory when
they update G4 -- their GPU memory may belong to another allocator that has
already reserved the device, or their measurement loop may not afford the
implicit device synchronisation of cudaMalloc/cudaFree.  It keeps its only
intermediate (G for both spins) in a fixed array inside the library.

This file is named so that pytest collects it last: a run that stops at the
first failure has then already run every other test.  It must also pass on
its own in a fresh process.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import TOL, cuda, draw, ensure_built, oracle_full

pytestmark = pytest.mark.gpu


def _free_after(torch, fn):
    """Device-wide free memory after fn() has run and the device is idle."""
    fn()
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_noalloc_two_calls_match_oracle_and_handle_path():
    torch = cuda()
    g4 = ensure_built()
    p = inputs.Problem(2, 2, 8, 3, 4, 10.0, 2, 2)      # N = 2*2 * 16 = 64
    M, G0, _ = draw(p, seed=5)
    s = np.array([1.0, -0.5])                          # any finite signs, sum != 0
    G0d = torch.from_numpy(G0).cuda()
    Md = [M[r].cuda() for r in range(2)]
    acc = torch.zeros((p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc), dtype=torch.complex128,
                      device="cuda")

    def call(r):
        return lambda: g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, Md[r], G0d, s[r], acc, lx=p.Lx)

    # The first call on a device may still load the library's device code and
    # look up its array's address (set-up, excluded on purpose); the second
    # call must leave the device's free memory unchanged.  The figure is
    # device-wide, so another process can move it: a change is retried once
    # with both calls repeated on a fresh accumulator before it counts.
    free1 = _free_after(torch, call(0))
    free2 = _free_after(torch, call(1))
    if free2 != free1:
        time.sleep(0.5)
        acc.zero_()
        free1 = _free_after(torch, call(0))
        free2 = _free_after(torch, call(1))
    assert free2 == free1, (free1, free2)   # the second call allocated nothing
    got = (acc / float(s.sum())).cpu().numpy()

    # against the oracle, element by element (relative Frobenius error, Eq. 3)
    ref, S = oracle_full(p, M, G0, s)
    assert S == s.sum()
    err = oracle.errors(ref, got)
    assert err["L2"] <= TOL["fp64"], err
    assert np.abs(got - ref).max() <= TOL["fp64"] * np.abs(ref).max()

    # and against the handle's FP64 path
    h = g4.G4.for_problem(p, precision="fp64", batch=2)
    for r in range(2):
        h.compute_G(Md[r], G0d, s[r])
    ref_h, S_h = h.finalize()
    h.close()
    assert S_h == s.sum()
    err = oracle.errors(ref_h.cpu().numpy(), got)
    assert err["L2"] <= TOL["fp64"], err


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = cuda()
    g4 = ensure_built()
    Nc, Nw = 4, 33                                     # N = 264 > 256
    N = Nc * 2 * Nw
    M = torch.zeros((2, N, N), dtype=torch.complex128, device="cuda")
    G0 = torch.zeros((2, N), dtype=torch.complex128, device="cuda")
    acc = torch.zeros(N * N, dtype=torch.complex128, device="cuda")
    with pytest.raises(g4.G4Error) as e:
        g4.update_noalloc(Nc, Nw, 1, 1, M, G0, 1.0, acc)
    assert e.value.status == g4.G4_ERR_INVALID
    assert "256" in str(e.value)


def test_noalloc_rejects_bad_buffers_before_the_library():
    """A short accumulator, a wrong type or a host tensor is refused by the
    binding (the C entry point receives bare pointers and cannot see sizes);
    an out-of-range Nwex is refused by the library itself."""
    torch = cuda()
    g4 = ensure_built()
    p = inputs.Problem(2, 2, 2, 2, 4, 5.0, 1, 1)
    N, E = p.N, p.entries
    M = torch.zeros((2, N, N), dtype=torch.complex128, device="cuda")
    G0 = torch.zeros((2, N), dtype=torch.complex128, device="cuda")
    acc = torch.zeros(E, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, M, G0, 1.0, acc[:-1], lx=p.Lx)
    with pytest.raises(ValueError):
        g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, M.to(torch.complex64), G0, 1.0, acc, lx=p.Lx)
    with pytest.raises(ValueError):
        g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, M, G0.cpu(), 1.0, acc, lx=p.Lx)
    lib = g4.load()
    import ctypes
    st = lib.g4_update_noalloc(p.Nc, p.Lx, p.Nw, 65, p.Nkex, ctypes.c_void_p(M.data_ptr()),
                               ctypes.c_void_p(G0.data_ptr()), 1.0,
                               ctypes.c_void_p(acc.data_ptr()), None)
    assert st == g4.G4_ERR_INVALID
