"""The step before the G build on the GPU: M from a vertex configuration (the
non-uniform Fourier transform of Sec. 2) against the oracle's double sum,
element by element, and G4 accumulated from vertex configurations against
the oracle run on the oracle's M."""
import numpy as np
import pytest

import oracle
from paper_2105_00027_gb300 import inputs
from gpu_util import TOL, cuda, ensure_built

pytestmark = pytest.mark.gpu

P = inputs.Problem


def _dev(torch, n_up, n_dn, tau, site, Mt):
    return (torch.from_numpy(tau).cuda(), torch.from_numpy(site).cuda(),
            torch.from_numpy(Mt).cuda())


def _blocks(n_up, n_dn, tau, site, Mt):
    """Per spin (tau, site, Mtau (n, n))."""
    out = []
    for sp, (b, n, mb) in enumerate([(0, n_up, 0), (n_up, n_dn, n_up * n_up)]):
        out.append((tau[b:b + n], site[b:b + n], Mt[mb:mb + n * n].reshape(n, n)))
    return out


def _oracle_M(p, cfg):
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    return np.stack([oracle.nfft(d, p.beta, t, s, m) for t, s, m in _blocks(*cfg)])


def _lib_M(p, cfg, precision):
    torch = cuda()
    g4 = ensure_built()
    h = g4.G4.for_problem(p, precision=precision, batch=1)
    n_up, n_dn = cfg[0], cfg[1]
    M = h.vertex_M(p.beta, n_up, n_dn, *_dev(torch, *cfg))
    out = M.cpu().numpy().astype(np.complex128)
    h.close()
    return out


def _rel(ref, got):
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [
    (2, 2, 4, 13, 7, True),       # ragged counts, independent spins
    (3, 3, 6, 40, 0, True),       # odd cluster, spin down empty
    (4, 2, 4, 1, 1, True),        # non-square cluster, one vertex each
    (1, 1, 1, 5, 5, True),        # Nc = 1, 2Nw = 2
    (2, 2, 16, 100, 100, False),  # 2Nw = 32, many vertices per site
    (5, 3, 3, 37, 50, True),      # 5 x 3 cluster
    (6, 6, 2, 60, 60, False),     # 6 x 6 cluster, more sites than warps
    (9, 2, 1, 40, 33, True),      # 9 x 2 cluster: wider than 8, the fallback kernels
    (8, 7, 1, 60, 45, True),      # 8 x 7 cluster: the longest transform lines (8 and 7)
])
def test_vertex_M_matches_oracle(precision, shape):
    Lx, Ly, Nw, n_up, n_dn, independent = shape
    p = P(Lx, Ly, Nw, 1, 1, 7.5, 1, 1)
    g = np.random.default_rng(Lx * 100 + n_up)
    if independent:
        tau = g.uniform(0.0, p.beta, n_up + n_dn)
        site = g.integers(0, p.Nc, n_up + n_dn).astype(np.int32)
        Mt = np.concatenate([g.normal(size=n_up * n_up), g.normal(size=n_dn * n_dn)])
        cfg = (n_up, n_dn, tau, site, Mt)
    else:
        cfg = inputs.vertex_config(p, 0, seed=3, n=n_up, jitter=False)
    err = _rel(_oracle_M(p, cfg), _lib_M(p, cfg, precision))
    assert err <= TOL[precision], err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vertex_M_one_site_and_wide_times(precision):
    """Every vertex on one site (one group holds all), times outside [0, beta)
    (the phases are antiperiodic, so any real tau is accepted)."""
    p = P(3, 2, 5, 1, 1, 4.0, 1, 1)
    g = np.random.default_rng(7)
    n = 64
    tau = g.uniform(-3 * p.beta, 3 * p.beta, 2 * n)
    site = np.full(2 * n, 4, np.int32)
    Mt = g.normal(size=2 * n * n)
    cfg = (n, n, tau, site, Mt)
    err = _rel(_oracle_M(p, cfg), _lib_M(p, cfg, precision))
    assert err <= TOL[precision], err


def test_vertex_M_c36_w64_sampled():
    """6x6 cluster, 2Nw = 64 at the benchmark's vertex count (1440 per spin,
    beta = 20): 96 entries of each spin's M against the oracle's double sum."""
    p = inputs.workload("c36_w64")
    cfg = inputs.vertex_config(p, 5)
    M = _lib_M(p, cfg, "mixed")
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    g = np.random.default_rng(11)
    K1 = g.integers(0, p.N, 96)
    K2 = np.where(np.arange(96) % 4 == 0, K1, g.integers(0, p.N, 96))   # some diagonal entries
    for sp, (t, s, m) in enumerate(_blocks(*cfg)):
        ref = oracle.nfft_entries(d, p.beta, t, s, m, K1, K2)
        err = _rel(ref, M[sp][K1, K2])
        assert err <= TOL["mixed"], (sp, err)


def test_vertex_M_max_vertices():
    """The largest vertex count the ABI accepts, on a small cluster."""
    from paper_2105_00027_gb300 import g4
    p = P(2, 2, 2, 1, 1, 10.0, 1, 1)
    n = g4.MAX_VERTICES
    g = np.random.default_rng(5)
    tau = g.uniform(0.0, p.beta, n)
    site = g.integers(0, p.Nc, n).astype(np.int32)
    Mt = g.normal(size=n * n) / np.sqrt(n)
    cfg = (n, 0, tau, site, Mt)
    M = _lib_M(p, cfg, "fp64")
    d = oracle.dims(p.Lx, p.Ly, p.Nw, 1, 1)
    K1 = np.array([0, 9], np.int32)
    K2 = np.array([0, 2], np.int32)
    ref = oracle.nfft_entries(d, p.beta, tau, site, Mt.reshape(n, n), K1, K2)
    assert _rel(ref, M[0][K1, K2]) <= TOL["fp64"]
    assert not M[1].any()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("channel", ["ph_magnetic", "pp_updown"])
def test_G4_from_vertices(precision, channel):
    """Whole path from vertex configurations: transform, G build, accumulate."""
    torch = cuda()
    g4 = ensure_built()
    p = P(2, 2, 4, 3, 4, 6.0, 19, 8)
    d = oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)
    G0 = inputs.g0(p)
    s = inputs.signs(p, seed=2)[:p.R]
    cfgs = [inputs.vertex_config(p, r, seed=2, n=30) for r in range(p.R)]
    Ms = np.stack([_oracle_M(p, c) for c in cfgs])
    slabs, S = oracle.run(d, Ms, G0, s, channel=channel)
    ref = oracle.to_exported(d, slabs)
    h = g4.G4.for_problem(p, precision=precision, channel=channel)
    G0d = torch.from_numpy(G0).cuda()
    for r, c in enumerate(cfgs):
        h.compute_G_vertices(p.beta, c[0], c[1], *_dev(torch, *c), G0d, float(s[r]))
    got, Sg = h.finalize()
    h.close()
    assert Sg == S
    err = oracle.errors(ref, got.cpu().numpy())
    assert err["L2"] <= TOL[precision], err


def test_vertex_bad_inputs():
    """Sites outside the cluster and non-finite times are reported as invalid
    (the kernels leave those vertices out); host-side argument errors."""
    torch = cuda()
    g4 = ensure_built()
    p = P(2, 2, 2, 1, 1, 5.0, 1, 1)
    h = g4.G4.for_problem(p, precision="mixed", batch=2)
    tau = torch.tensor([0.5, 1.0, 2.0], dtype=torch.float64, device="cuda")
    Mt = torch.ones(9 + 0, dtype=torch.float64, device="cuda")
    bad_site = torch.tensor([0, 4, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(g4.G4Error) as e:
        h.vertex_M(p.beta, 3, 0, tau, bad_site, Mt)
    assert e.value.status == g4.G4_ERR_INVALID
    h.close()
    h = g4.G4.for_problem(p, precision="fp64", batch=2)
    site = torch.tensor([0, 3, 1], dtype=torch.int32, device="cuda")
    nan_tau = torch.tensor([0.5, float("nan"), 2.0], dtype=torch.float64, device="cuda")
    with pytest.raises(g4.G4Error) as e:
        h.vertex_M(p.beta, 3, 0, nan_tau, site, Mt)
    assert e.value.status == g4.G4_ERR_INVALID
    h.close()
    h = g4.G4.for_problem(p, precision="mixed", batch=2)
    G0 = torch.from_numpy(inputs.g0(p)).cuda()
    h.compute_G_vertices(p.beta, 3, 0, tau, bad_site, Mt, G0, 1.0)
    with pytest.raises(g4.G4Error) as e:
        h.finalize()
    assert e.value.status == g4.G4_ERR_INVALID
    h.close()
    h = g4.G4.for_problem(p, precision="mixed", batch=2)
    for beta, n_up, n_dn in [(0.0, 3, 0), (float("inf"), 3, 0), (5.0, -1, 0),
                             (5.0, g4.MAX_VERTICES + 1, 0)]:
        with pytest.raises(g4.G4Error) as e:
            h.vertex_M(beta, n_up, n_dn, tau, site, Mt)
        assert e.value.status == g4.G4_ERR_INVALID
    with pytest.raises(g4.G4Error):
        h.reserve_vertices(g4.MAX_VERTICES + 1)
    h.reserve_vertices(1000)
    h.close()


def test_vertex_scratch_oom_then_recovers():
    """Growing the vertex scratch past the handle's memory limit fails with
    G4_ERR_OOM part-way; a smaller growth afterwards succeeds and the
    transform is still right."""
    torch = cuda()
    g4 = ensure_built()
    p = P(2, 2, 2, 1, 1, 5.0, 1, 1)
    h = g4.G4.for_problem(p, precision="mixed", batch=1, mem_limit=256 << 20)
    with pytest.raises(g4.G4Error) as e:
        h.reserve_vertices(g4.MAX_VERTICES)      # its Mtau copy alone is 2 GiB
    assert e.value.status == g4.G4_ERR_OOM
    h.reserve_vertices(100)
    cfg = inputs.vertex_config(p, 0, seed=9, n=50, jitter=False)
    M = h.vertex_M(p.beta, cfg[0], cfg[1], *_dev(torch, *cfg)).cpu().numpy().astype(np.complex128)
    h.close()
    assert _rel(_oracle_M(p, cfg), M) <= TOL["mixed"]
