"""The allocation-free update entry point, checked on the GPU against the
regular FP64 path of the library.

g4_update_noalloc exists for callers that cannot allocate device memory when
they update G4 -- their GPU memory may belong to another allocator that has
already reserved the device, or their measurement loop may not afford the
implicit device synchronisation of cudaMalloc/cudaFree.  It keeps its only
intermediate (G for both spins) in a fixed array inside the library.

This file is named so that pytest collects it last: a run that stops at the
first failure has then already run every other test.  It must also pass on
its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import TOL, cuda, draw, ensure_built

pytestmark = pytest.mark.gpu


def test_noalloc_two_calls_match_handle_path():
    torch = cuda()
    g4 = ensure_built()
    p = inputs.Problem(2, 2, 8, 3, 4, 10.0, 2, 2)      # N = 2*2 * 16 = 64
    M, G0, _ = draw(p, seed=5)
    s = np.array([1.0, -0.5])                          # any finite signs, sum != 0
    G0d = torch.from_numpy(G0).cuda()
    Md = [M[r].cuda() for r in range(2)]
    acc = torch.zeros((p.Nwex, p.Nw2, p.Nw2, p.Nkex, p.Nc, p.Nc), dtype=torch.complex128,
                      device="cuda")
    g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, Md[0], G0d, s[0], acc, lx=p.Lx)
    torch.cuda.synchronize()
    free_after_first = torch.cuda.mem_get_info()[0]
    g4.update_noalloc(p.Nc, p.Nw, p.Nwex, p.Nkex, Md[1], G0d, s[1], acc, lx=p.Lx)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_after_first   # the second call allocated nothing
    got = (acc / float(s.sum())).cpu().numpy()

    h = g4.G4.for_problem(p, precision="fp64", batch=2)
    for r in range(2):
        h.compute_G(Md[r], G0d, s[r])
    ref, S = h.finalize()
    h.close()
    assert S == s.sum()
    err = oracle.errors(ref.cpu().numpy(), got)
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
