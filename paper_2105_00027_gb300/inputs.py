"""Seeded synthetic inputs for the G4 measurement step.

This module holds no part of the G4 arithmetic: it only describes the
workloads and draws their inputs.  Both the CUDA library (through the tests
and the benchmark) and the CPU oracle consume what it produces.

Input recipe (a stand-in for the Hubbard-model QMC measurements of Sec. 4.3,
which are not available):

* cluster: Lx x Ly square lattice (Nc = Lx*Ly; Nc = 8 is read as 4 x 2),
  momenta k = (2 pi ix / Lx, 2 pi iy / Ly), index k = ix + Lx*iy;
* frequencies: 2*Nw fermionic Matsubara points w_n = (2(n-Nw)+1) pi / beta,
  index n in [0, 2*Nw);
* G0_sigma(k, n) = 1 / (i w_n - (eps_k - sigma*h)), eps_k = -2(cos kx + cos ky),
  h = 0 unless a Zeeman field is asked for;
* M_sigma: per measurement and spin an N x N complex matrix (N = Nc*2*Nw)
  with independent N(0, 1/N) real and imaginary parts;
* sign s_r = +1 with probability 0.9, else -1.

Vertex configurations (the input of the step before, the transform that
turns a configuration into M; see :func:`vertex_config`): n vertices per
spin, shared by both spins as in an auxiliary-field expansion where every
vertex couples to both spin species; n = round(beta U Nc / 2) with U = 4 by
default (the order of magnitude of the mean expansion order of such a
solver on a Hubbard cluster at that coupling), jittered by up to +-10% per
measurement; times tau_i uniform on [0, beta), sites uniform over the
cluster; per spin a real matrix Mtau = diag(d) + X with d_i uniform on
[0.5, 1.5] and X_ij independent N(0, 1/n).

Random streams: signs, per-problem draws and host-side M use numpy's Philox
generator keyed by the seed (M: one generator per measurement, so any
measurement can be regenerated alone); benchmark-sized device-resident M
uses one torch CUDA generator per fill.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Problem:
    """One G4 problem: cluster, frequency grid, transfers and run length."""
    Lx: int
    Ly: int
    Nw: int          # positive frequencies; the grid has 2*Nw points
    Nwex: int        # bosonic transfers m = 0..Nwex-1
    Nkex: int        # transfer momenta q = 0..Nkex-1
    beta: float
    R: int           # measurements
    batch: int       # measurements per accumulate call
    m_dtype: str = "c128"   # storage type of M ("c128" or "c64")
    h: float = 0.0           # Zeeman field (spin splitting of G0)

    @property
    def Nc(self):
        return self.Lx * self.Ly

    @property
    def Nw2(self):
        return 2 * self.Nw

    @property
    def N(self):
        return self.Nc * self.Nw2

    @property
    def NQ(self):
        return self.Nkex * self.Nwex

    @property
    def entries(self):
        """Number of G4 entries E = N^2 * NQ."""
        return self.N * self.N * self.NQ

    @property
    def updates(self):
        """Element-updates of a whole run, E * R."""
        return self.entries * self.R


def cluster_shape(Nc: int):
    """(Lx, Ly) for Nc sites: square when possible; Nc = 8 -> 4 x 2."""
    r = int(round(math.sqrt(Nc)))
    if r * r == Nc:
        return r, r
    for ly in range(int(math.sqrt(Nc)), 0, -1):
        if Nc % ly == 0:
            return Nc // ly, ly
    return Nc, 1


WORKLOADS = ("tiny_2x2", "c16_w64", "c36_w64", "c64_w64")


def workload(name: str) -> Problem:
    """The single-problem workloads, named by cluster and frequency grid.

    tiny_2x2  2x2 cluster, 2Nw = 8, Nwex = Nkex = 1, 16 measurements
    c16_w64   4x4 cluster, 2Nw = 64, Nwex = 8, Nkex = 16, 256 measurements
    c36_w64   6x6 cluster, 2Nw = 64, Nwex = 8, Nkex = 36, 1024 measurements
              in batches of 64 (the mixed-precision form)
    c64_w64   8x8 cluster, 2Nw = 64, Nwex = 4, Nkex = 64, 4096 measurements
              in batches of 128, M stored complex64

    The twelve-problem batching workload is :func:`group_problems`.
    """
    if name == "tiny_2x2":
        return Problem(2, 2, 4, 1, 1, 10.0, 16, 16)
    if name == "c16_w64":
        return Problem(4, 4, 32, 8, 16, 20.0, 256, 64)
    if name == "c36_w64":
        return Problem(6, 6, 32, 8, 36, 20.0, 1024, 64)
    if name == "c64_w64":
        return Problem(8, 8, 32, 4, 64, 40.0, 4096, 128, m_dtype="c64")
    raise ValueError("unknown workload %r" % (name,))


def group_problems(seed: int = 0):
    """Twelve problems: Nc in {4, 8, 16, 36} x 2Nw in {16, 32, 64}, Nwex = 4,
    Nkex = Nc, beta = (5, 10, 20)[p % 3], R_p = 32 + floor(481 u_p)."""
    g = np.random.Generator(np.random.Philox(key=seed + 0x51ED))
    out = []
    p = 0
    for Nc in (4, 8, 16, 36):
        Lx, Ly = cluster_shape(Nc)
        for Nw2 in (16, 32, 64):
            R = 32 + int(math.floor(481 * g.random()))
            out.append(Problem(Lx, Ly, Nw2 // 2, 4, Nc, (5.0, 10.0, 20.0)[p % 3], R,
                               min(64, R)))
            p += 1
    return out


def momenta(Lx: int, Ly: int):
    i = np.arange(Lx * Ly)
    return np.stack([2 * np.pi * (i % Lx) / Lx, 2 * np.pi * (i // Lx) / Ly], axis=1)


def matsubara(Nw: int, beta: float):
    n = np.arange(2 * Nw)
    return (2 * (n - Nw) + 1) * np.pi / beta


def g0(p: Problem) -> np.ndarray:
    """G0[sigma][K] (sigma = 0 is spin up), complex128, K = k*2Nw + n."""
    k = momenta(p.Lx, p.Ly)
    eps = -2.0 * (np.cos(k[:, 0]) + np.cos(k[:, 1]))
    w = matsubara(p.Nw, p.beta)
    out = np.empty((2, p.N), np.complex128)
    for s, sigma in enumerate((+1.0, -1.0)):
        out[s] = (1.0 / (1j * w[None, :] - (eps[:, None] - sigma * p.h))).ravel()
    return out


def signs(p: Problem, seed: int = 0, problem_index: int = 0) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=[seed, 0x5167 + problem_index]))
    u = g.random(p.R)
    return np.where(u < 0.9, 1.0, -1.0)


def _mseed(seed, problem_index, r):
    return (seed * 0x9E3779B1 + problem_index * 0x85EBCA77 + r * 0xC2B2AE3D + 1) % (2 ** 63)


def measurement_M(p: Problem, r: int, seed: int = 0, problem_index: int = 0):
    """M of measurement r as a CPU torch tensor [2][N][N] (complex128 or complex64):
    independent N(0, 1/N) real and imaginary parts from numpy's Philox
    generator keyed by (seed, problem, measurement), drawn directly in the
    storage precision (float64 for complex128 M, float32 for complex64)."""
    import torch
    g = np.random.Generator(np.random.Philox(key=[_mseed(seed, problem_index, r), 0x4D]))
    dt = np.float64 if p.m_dtype == "c128" else np.float32
    x = g.standard_normal((2, p.N, p.N, 2), dtype=dt)
    x *= dt(1.0 / math.sqrt(p.N))
    z = torch.view_as_complex(torch.from_numpy(x))
    return z


def batch_M(p: Problem, r0: int, count: int, seed: int = 0, problem_index: int = 0):
    """M of measurements r0..r0+count-1 stacked as a CPU tensor [count][2][N][N]."""
    import torch
    return torch.stack([measurement_M(p, r, seed, problem_index) for r in range(r0, r0 + count)])


def fill_M_device(out, seed: int = 0):
    """Fill a CUDA complex tensor [..., N, N] with i.i.d. N(0, 1/N) re/im parts
    (benchmark-sized inputs; not reproducible on the host)."""
    import torch
    N = out.shape[-1]
    g = torch.Generator(device=out.device).manual_seed(_mseed(seed, 0xB, 0))
    real = torch.view_as_real(out)
    flat = real.view(-1)
    chunk = 1 << 28
    for i in range(0, flat.numel(), chunk):
        seg = flat[i:i + chunk]
        seg.normal_(0.0, 1.0 / math.sqrt(N), generator=g)
    return out


def with_(p: Problem, **kw) -> Problem:
    return replace(p, **kw)


def vertices_per_spin(p: Problem, U: float = 4.0) -> int:
    """Mean vertex count per spin of the synthetic configurations."""
    return max(1, int(round(p.beta * U * p.Nc / 2)))


def vertex_config(p: Problem, r: int, seed: int = 0, n: int = None, jitter: bool = True,
                  shared: bool = True):
    """Vertex configuration of measurement r.

    Returns (n_up, n_dn, tau [n_up + n_dn] float64, site [n_up + n_dn] int32,
    Mtau [n_up^2 + n_dn^2] float64: the spin-up block, then spin-down, each
    row-major).  ``n`` overrides the mean count; ``shared`` = False draws the
    spin-down vertices independently (with their own count)."""
    g = np.random.Generator(np.random.Philox(key=[seed, (0x7E47 << 32) | r]))
    nbar = n if n is not None else vertices_per_spin(p)

    def count():
        if not jitter or nbar == 0:
            return nbar
        return max(0, int(round(nbar * (1.0 + 0.1 * (2.0 * g.random() - 1.0)))))

    n_up = count()
    tau_up = g.uniform(0.0, p.beta, n_up)
    site_up = g.integers(0, p.Nc, n_up)
    if shared:
        n_dn, tau_dn, site_dn = n_up, tau_up, site_up
    else:
        n_dn = count()
        tau_dn = g.uniform(0.0, p.beta, n_dn)
        site_dn = g.integers(0, p.Nc, n_dn)
    blocks = []
    for m in (n_up, n_dn):
        X = g.normal(0.0, 1.0 / math.sqrt(max(m, 1)), (m, m))
        X[np.diag_indices(m)] += g.uniform(0.5, 1.5, m)
        blocks.append(X.ravel())
    tau = np.concatenate([tau_up, tau_dn]).astype(np.float64)
    site = np.concatenate([site_up, site_dn]).astype(np.int32)
    return n_up, n_dn, tau, site, np.concatenate(blocks)
