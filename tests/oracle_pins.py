"""Pins for the CPU oracle: checks against facts the oracle does not compute.

Each ``pin_*`` function runs the oracle (through a given ctypes library, so
the mutation test can hand it a deliberately broken build) on a small seeded
problem and returns the worst deviation from what mathematics or physics
fixes.  Tolerances are applied by the callers.

Facts used:
* the step before (M from a vertex configuration by the non-uniform Fourier
  transform): time and lattice translation phases, fermionic antiperiodicity,
  momentum completeness, Hermiticity, vertex relabelling, a numpy matrix-product
  evaluation;
* closed forms for a non-interacting configuration (M = 0), with and without
  a spin splitting of G0;
* Wick's theorem written as a 2x2 determinant of spin-resolved propagators,
  evaluated by brute force -- independent of the direct/exchange split;
* exact invariances: lattice-translation and imaginary-time gauge phases of
  M, spin exchange, flipping every sign, splitting the run into batches;
* the frequency-reversal / complex-conjugation relation for a symmetrised M;
* the momentum selection rule for a translation-invariant M;
* numpy's matmul (direct term as A^T diag(s) B) and G as D - D M D.
Momentum sums here use momentum vectors mod 2 pi, never the oracle's table.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2105_00027_gb300 import inputs


def problem(Lx, Ly, Nw, Nwex, Nkex, beta=7.0, R=3, h=0.0):
    return inputs.Problem(Lx, Ly, Nw, Nwex, Nkex, beta, R, R, h=h)


def dims_of(p):
    return oracle.dims(p.Lx, p.Ly, p.Nw, p.Nwex, p.Nkex)


def draw(p, seed=1):
    M = inputs.batch_M(p, 0, p.R, seed=seed).numpy().astype(np.complex128)
    s = inputs.signs(p, seed=seed)
    if s.sum() == 0:
        s[0] = -s[0]
    return M, inputs.g0(p), s


def full(p, M, G0, s, lib, channel=0):
    """Oracle on every slab, in the exported order [m][n2][n1][q][k2][k1]."""
    d = dims_of(p)
    slabs, S = oracle.run(d, M, G0, s, lib=lib, channel=channel)
    return oracle.to_exported(d, slabs), S


# ---- independent momentum arithmetic (vectors mod 2 pi) -------------------

def _kvec(p):
    return inputs.momenta(p.Lx, p.Ly)


def _kindex(p, v):
    k = _kvec(p)
    v = np.mod(v, 2 * np.pi)
    dist = np.abs(np.angle(np.exp(1j * (k - v[None, :])))).sum(axis=1)
    i = int(np.argmin(dist))
    assert dist[i] < 1e-9
    return i


def kplus_vec(p, a, b):
    k = _kvec(p)
    return _kindex(p, k[a] + k[b])


def kneg_vec(p, a):
    return _kindex(p, -_kvec(p)[a])


def kminus_vec(p, a, b):
    k = _kvec(p)
    return _kindex(p, k[a] - k[b])


def freq_index(p, w):
    """Index of the fermionic frequency with value w, or None off the grid."""
    ws = inputs.matsubara(p.Nw, p.beta)
    i = int(np.argmin(np.abs(ws - w)))
    return i if abs(ws[i] - w) < 1e-9 else None


def _rel(a, b):
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


# ---- pins -------------------------------------------------------------------

def pin_closed_form(lib, h=0.0, channel=0):
    """M = 0 (G = G0 on the diagonal), per channel:
    magnetic: d_{Q,0} (G0u-G0d)(K1) (G0u-G0d)(K2) - d_{K1K2} sum_s G0_s(K1) G0_s(K1+Q)
    density:  d_{Q,0} (G0u+G0d)(K1) (G0u+G0d)(K2) - d_{K1K2} sum_s G0_s(K1) G0_s(K1+Q)
    transverse: - d_{K1K2} sum_s G0_-s(K1) G0_s(K1+Q)
    particle-particle: d_{K1K2} sum_s G0_s(Q-K1) G0_-s(K1)."""
    p = problem(2, 2, 2, 3, 4, R=3, h=h)
    M = np.zeros((p.R, 2, p.N, p.N), np.complex128)
    G0 = inputs.g0(p)
    s = np.array([1.0, -1.0, 1.0])
    got, S = full(p, M, G0, s, lib, channel)
    exp = np.zeros_like(got)
    w = inputs.matsubara(p.Nw, p.beta)
    nu = 2 * np.pi / p.beta
    for q in range(p.Nkex):
        for m in range(p.Nwex):
            for n1 in range(p.Nw2):
                for n2 in range(p.Nw2):
                    for k1 in range(p.Nc):
                        for k2 in range(p.Nc):
                            K1, K2 = k1 * p.Nw2 + n1, k2 * p.Nw2 + n2
                            v = 0.0
                            if channel in (0, 2):
                                sg = -1.0 if channel == 0 else 1.0
                                if q == 0 and m == 0:
                                    v += (G0[0][K1] + sg * G0[1][K1]) * (G0[0][K2] + sg * G0[1][K2])
                            if K1 == K2:
                                if channel == 1:
                                    f = freq_index(p, m * nu - w[n1])
                                    if f is not None:
                                        QK = kminus_vec(p, q, k1) * p.Nw2 + f
                                        v += G0[0][QK] * G0[1][K1] + G0[1][QK] * G0[0][K1]
                                elif n1 + m < p.Nw2:
                                    K1Q = kplus_vec(p, k1, q) * p.Nw2 + n1 + m
                                    if channel == 3:
                                        v -= G0[1][K1] * G0[0][K1Q] + G0[0][K1] * G0[1][K1Q]
                                    else:
                                        v -= G0[0][K1] * G0[0][K1Q] + G0[1][K1] * G0[1][K1Q]
                            exp[m, n2, n1, q, k2, k1] = v
    return _rel(got, exp)


def pin_build_G(lib):
    """G = D - D M D with D = diag(G0), by numpy matmul."""
    p = problem(2, 1, 3, 1, 1)
    M, G0, _ = draw(p)
    worst = 0.0
    for sp in range(2):
        D = np.diag(G0[sp])
        exp = D - D @ M[0, sp] @ D
        got = oracle.build_G(M[0, sp], G0[sp], lib)
        worst = max(worst, _rel(got, exp))
    return worst


def wick_bruteforce(p, M, G0, s, channel=0):
    """sum_r s_r sum (weights) det[[G(1,2), G(1,4)], [G(3,2), G(3,4)]] / sum s over the
    channel's operator points (spin-resolved G; K+Q and Q-K from momentum vectors and
    frequency values):
      magnetic / density: 1=(K1+Q,s) 2=(K1,s) 3=(K2,s') 4=(K2+Q,s'), weight s s' / 1
      transverse:         1=(K1+Q,s) 2=(K1,-s) 3=(K2,-s) 4=(K2+Q,s)
      particle-particle:  1=(K2,-s) 2=(K1,-s) 3=(Q-K2,s) 4=(Q-K1,s)"""
    N, Nw2, Nc = p.N, p.Nw2, p.Nc
    w = inputs.matsubara(p.Nw, p.beta)
    nu = 2 * np.pi / p.beta
    out = np.zeros((p.Nwex, Nw2, Nw2, p.Nkex, Nc, Nc), np.complex128)
    for r in range(len(s)):
        Gf = np.zeros((2 * N, 2 * N), np.complex128)
        for sp in range(2):
            D = np.diag(G0[sp])
            Gf[sp * N:(sp + 1) * N, sp * N:(sp + 1) * N] = D - D @ M[r, sp] @ D

        def idx(sp, k, n):
            return None if (n is None or not (0 <= n < Nw2)) else sp * N + k * Nw2 + n

        def g(a, b):
            return 0.0 if a is None or b is None else Gf[a, b]

        for q in range(p.Nkex):
            for m in range(p.Nwex):
                for k1 in range(Nc):
                    k1q, qk1 = kplus_vec(p, k1, q), kminus_vec(p, q, k1)
                    for k2 in range(Nc):
                        k2q, qk2 = kplus_vec(p, k2, q), kminus_vec(p, q, k2)
                        for n1 in range(Nw2):
                            f1 = freq_index(p, m * nu - w[n1])
                            for n2 in range(Nw2):
                                f2 = freq_index(p, m * nu - w[n2])
                                v = 0.0
                                for si, sig in ((0, 1.0), (1, -1.0)):
                                    sb = 1 - si
                                    if channel in (0, 2):
                                        for sj, sig2 in ((0, 1.0), (1, -1.0)):
                                            wt = sig * sig2 if channel == 0 else 1.0
                                            i1, i2 = idx(si, k1q, n1 + m), idx(si, k1, n1)
                                            i3, i4 = idx(sj, k2, n2), idx(sj, k2q, n2 + m)
                                            v += wt * (g(i1, i2) * g(i3, i4) - g(i1, i4) * g(i3, i2))
                                        continue
                                    if channel == 3:
                                        i1, i2 = idx(si, k1q, n1 + m), idx(sb, k1, n1)
                                        i3, i4 = idx(sb, k2, n2), idx(si, k2q, n2 + m)
                                    else:
                                        i1, i2 = idx(sb, k2, n2), idx(sb, k1, n1)
                                        i3, i4 = idx(si, qk2, f2), idx(si, qk1, f1)
                                    v += g(i1, i2) * g(i3, i4) - g(i1, i4) * g(i3, i2)
                                out[m, n2, n1, q, k2, k1] += s[r] * v
    return out / s.sum()


def pin_wick(lib, shape=(2, 2, 2, 3, 4), channel=0):
    p = problem(*shape, R=3)
    M, G0, s = draw(p, seed=3)
    got, _ = full(p, M, G0, s, lib, channel)
    return _rel(got, wick_bruteforce(p, M, G0, s, channel))


def pin_translation_gauge(lib, shape=(4, 2, 2, 2, 8), a=(1, 1), channel=0):
    """M(K1,K2) -> exp(i (k1-k2).a) M(K1,K2) leaves G4 unchanged."""
    p = problem(*shape, R=3)
    M, G0, s = draw(p, seed=4)
    ref, _ = full(p, M, G0, s, lib, channel)
    k = _kvec(p)
    ph_k = np.exp(1j * (k @ np.asarray(a, float)))
    ph = np.repeat(ph_k, p.Nw2)
    M2 = M * ph[None, None, :, None] * np.conj(ph)[None, None, None, :]
    got, _ = full(p, M2, G0, s, lib, channel)
    return _rel(got, ref)


def pin_time_gauge(lib, shape=(2, 2, 3, 3, 4), tau_frac=0.37, channel=0):
    """M(K1,K2) -> exp(i (w1-w2) tau) M(K1,K2) leaves G4 unchanged."""
    p = problem(*shape, R=3)
    M, G0, s = draw(p, seed=5)
    ref, _ = full(p, M, G0, s, lib, channel)
    w = inputs.matsubara(p.Nw, p.beta)
    ph = np.tile(np.exp(1j * w * tau_frac * p.beta), p.Nc)
    M2 = M * ph[None, None, :, None] * np.conj(ph)[None, None, None, :]
    got, _ = full(p, M2, G0, s, lib, channel)
    return _rel(got, ref)


def pin_spin_swap(lib, channel=0):
    p = problem(2, 2, 2, 2, 4, R=3, h=0.3)
    M, G0, s = draw(p, seed=6)
    ref, _ = full(p, M, G0, s, lib, channel)
    got, _ = full(p, M[:, ::-1].copy(), G0[::-1].copy(), s, lib, channel)
    return _rel(got, ref)


def pin_sign_flip(lib):
    p = problem(2, 2, 2, 2, 4, R=3)
    M, G0, s = draw(p, seed=7)
    ref, _ = full(p, M, G0, s, lib)
    got, _ = full(p, M, G0, -s, lib)
    return _rel(got, ref)


def pin_batch_split(lib):
    p = problem(2, 2, 2, 2, 4, R=5)
    M, G0, s = draw(p, seed=8)
    s = np.array([1.0, 1.0, -1.0, 1.0, 1.0])
    ref, S = full(p, M, G0, s, lib)
    a, Sa = full(p, M[:2], G0, s[:2], lib)
    b, Sb = full(p, M[2:], G0, s[2:], lib)
    return _rel((a * Sa + b * Sb) / (Sa + Sb), ref)


def _minusK_perm(p):
    perm = np.empty(p.N, np.int64)
    for k in range(p.Nc):
        for n in range(p.Nw2):
            perm[k * p.Nw2 + n] = kneg_vec(p, k) * p.Nw2 + (p.Nw2 - 1 - n)
    return perm


def pin_conjugation(lib, shape=(4, 2, 2, 3, 8)):
    """For M(-K1,-K2) = conj M(K1,K2): G4(-K2-Q, -K1-Q, Q) = conj G4(K1, K2, Q)."""
    p = problem(*shape, R=3)
    M, G0, s = draw(p, seed=9)
    perm = _minusK_perm(p)
    Ms = 0.5 * (M + np.conj(M[:, :, perm][:, :, :, perm]))
    g4, _ = full(p, Ms, G0, s, lib)
    worst = 0.0
    scale = np.abs(g4).max()
    for q in range(p.Nkex):
        for m in range(p.Nwex):
            for k1 in range(p.Nc):
                for k2 in range(p.Nc):
                    for n1 in range(p.Nw2 - m):
                        for n2 in range(p.Nw2 - m):
                            a = kneg_vec(p, kplus_vec(p, k2, q))
                            b = kneg_vec(p, kplus_vec(p, k1, q))
                            na, nb = p.Nw2 - 1 - (n2 + m), p.Nw2 - 1 - (n1 + m)
                            lhs = g4[m, nb, na, q, b, a]
                            rhs = np.conj(g4[m, n2, n1, q, k2, k1])
                            worst = max(worst, abs(lhs - rhs) / scale)
    return worst


def pin_selection_rule(lib):
    """k-diagonal M: G4 vanishes unless q = 0 or k1 = k2."""
    p = problem(2, 2, 2, 2, 4, R=3)
    M, G0, s = draw(p, seed=10)
    kk = np.repeat(np.arange(p.Nc), p.Nw2)
    M = M * (kk[:, None] == kk[None, :])[None, None]
    g4, _ = full(p, M, G0, s, lib)
    mask = np.zeros(g4.shape, bool)
    for q in range(1, p.Nkex):
        for k1 in range(p.Nc):
            for k2 in range(p.Nc):
                if k1 != k2:
                    mask[:, :, :, q, k2, k1] = True
    return float(np.abs(g4[mask]).max() / np.abs(g4).max())


def numpy_cross(p, M, G0, s):
    """Direct term as A_Q^T diag(s) B_Q (numpy matmul) and the exchange as an
    einsum over (r, spin), assembled in exported order."""
    N, Nw2, Nc = p.N, p.Nw2, p.Nc
    R = len(s)
    G = np.empty((R, 2, N, N), np.complex128)
    for r in range(R):
        for sp in range(2):
            D = np.diag(G0[sp])
            G[r, sp] = D - D @ M[r, sp] @ D
    # pad with a zero frequency block so that n+m >= Nw2 reads zero
    Gp = np.zeros((R, 2, Nc, Nw2 + p.Nwex, Nc, Nw2 + p.Nwex), np.complex128)
    Gp[:, :, :, :Nw2, :, :Nw2] = G.reshape(R, 2, Nc, Nw2, Nc, Nw2)
    sig = np.array([1.0, -1.0])
    out = np.zeros((p.Nwex, Nw2, Nw2, p.Nkex, Nc, Nc), np.complex128)
    n = np.arange(Nw2)
    for q in range(p.Nkex):
        kq = np.array([kplus_vec(p, k, q) for k in range(Nc)])
        for m in range(p.Nwex):
            # a[r, k1, n1] = sum_s s G_s(K1+Q, K1); b[r, k2, n2] = sum_s s G_s(K2, K2+Q)
            a = np.einsum("s,rskn->rkn", sig,
                          Gp[:, :, kq[:, None], (n + m)[None, :], np.arange(Nc)[:, None], n[None, :]])
            b = np.einsum("s,rskn->rkn", sig,
                          Gp[:, :, np.arange(Nc)[:, None], n[None, :], kq[:, None], (n + m)[None, :]])
            A = a.reshape(R, N)
            B = b.reshape(R, N)
            direct = A.T @ np.diag(s) @ B            # [K1, K2]
            # exchange[K1, K2] = sum_r s_r sum_s G_s(K2, K1) G_s(K1+Q, K2+Q)
            Gt = G.transpose(0, 1, 3, 2)              # [r, s, K1, K2] = G(K2, K1)
            sh = Gp[:, :, kq[:, None, None, None], (n + m)[None, :, None, None],
                    kq[None, None, :, None], (n + m)[None, None, None, :]].reshape(R, 2, N, N)
            exch = np.einsum("r,rsij,rsij->ij", s, Gt, sh)
            val = (direct - exch) / s.sum()           # [K1, K2]
            v = val.reshape(Nc, Nw2, Nc, Nw2)         # [k1, n1, k2, n2]
            out[m, :, :, q] = v.transpose(3, 1, 2, 0)  # [n2, n1, k2, k1]
    return out


def pin_numpy_cross(lib):
    p = problem(2, 2, 3, 3, 4, R=4)
    M, G0, s = draw(p, seed=11)
    got, _ = full(p, M, G0, s, lib)
    return _rel(got, numpy_cross(p, M, G0, s))


# name -> (function, tolerance); the other channels' pins follow the magnetic ones
# ---------------------------------------------------------------- the step before:
# M from a vertex configuration by the non-uniform Fourier transform

def _config(n=5, seed=3, hermitian=False, Lx=3, Ly=2, beta=6.0):
    rng = np.random.default_rng(seed)
    tau = rng.uniform(0.0, beta, n)
    site = rng.integers(0, Lx * Ly, n)
    Mt = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    if hermitian:
        Mt = Mt + Mt.conj().T
    return oracle.dims(Lx, Ly, 2, 1, 1), beta, tau, site, Mt


def _kw(d, beta):
    """Per K = k*Nw2 + n: Matsubara frequency and momentum components."""
    K = np.arange(d.N)
    k, n = K // d.Nw2, K % d.Nw2
    w = (2 * (n - d.Nw) + 1) * np.pi / beta
    kx = 2 * np.pi * (k % d.Lx) / d.Lx
    ky = 2 * np.pi * (k // d.Lx) / d.Ly
    return w, kx, ky


def pin_nfft_time_translation(lib, tau0=0.37):
    """Shifting every vertex time by tau0 multiplies M(K1, K2) by e^{i(w1-w2)tau0}."""
    d, beta, tau, site, Mt = _config()
    tau = tau * 0.8                                  # keep tau + tau0 inside [0, beta)
    A = oracle.nfft(d, beta, tau, site, Mt, lib)
    B = oracle.nfft(d, beta, tau + tau0, site, Mt, lib)
    w, _, _ = _kw(d, beta)
    return _rel(B, A * np.exp(1j * (w[:, None] - w[None, :]) * tau0))


def pin_nfft_lattice_translation(lib, a=(1, 1)):
    """Moving every vertex by the lattice vector a multiplies M by e^{-i(k1-k2).a}."""
    d, beta, tau, site, Mt = _config()
    sx, sy = site % d.Lx, site // d.Lx
    moved = (sx + a[0]) % d.Lx + d.Lx * ((sy + a[1]) % d.Ly)
    A = oracle.nfft(d, beta, tau, site, Mt, lib)
    B = oracle.nfft(d, beta, tau, moved, Mt, lib)
    _, kx, ky = _kw(d, beta)
    ka = kx * a[0] + ky * a[1]
    return _rel(B, A * np.exp(-1j * (ka[:, None] - ka[None, :])))


def pin_nfft_antiperiodic(lib):
    """Fermionic frequencies: e^{i w beta} = -1, so moving vertex i by beta and
    negating row i and column i of Mtau (its diagonal entry twice) leaves M unchanged."""
    d, beta, tau, site, Mt = _config()
    i = 2
    tau2 = tau.copy()
    tau2[i] += beta
    Mt2 = Mt.copy()
    Mt2[i, :] *= -1
    Mt2[:, i] *= -1
    return _rel(oracle.nfft(d, beta, tau2, site, Mt2, lib), oracle.nfft(d, beta, tau, site, Mt, lib))


def pin_nfft_momentum_sum(lib):
    """Completeness of the cluster momenta: sum_k M((k,n1),(k,n2)) =
    1/beta sum_{i,j: x_i = x_j} e^{i w1 tau_i} Mtau_ij e^{-i w2 tau_j}."""
    d, beta, tau, site, Mt = _config(n=6, seed=5)
    site = site % 3                                  # several vertices share a site
    M = oracle.nfft(d, beta, tau, site, Mt, lib).reshape(d.Nc, d.Nw2, d.Nc, d.Nw2)
    lhs = np.einsum("knkm->nm", M)
    n = np.arange(d.Nw2)
    w = (2 * (n - d.Nw) + 1) * np.pi / beta
    same = (site[:, None] == site[None, :]).astype(float)
    rhs = np.exp(1j * w[:, None] * tau[None, :]) @ (Mt * same) @ np.exp(-1j * tau[:, None] * w[None, :]) / beta
    return _rel(lhs, rhs)


def pin_nfft_hermitian(lib):
    """A Hermitian Mtau gives a Hermitian M."""
    d, beta, tau, site, Mt = _config(hermitian=True)
    M = oracle.nfft(d, beta, tau, site, Mt, lib)
    return _rel(M, M.conj().T)


def pin_nfft_permutation(lib):
    """Relabelling the vertices (Mtau permuted alike) leaves M unchanged."""
    d, beta, tau, site, Mt = _config()
    perm = np.array([3, 0, 4, 1, 2])
    return _rel(oracle.nfft(d, beta, tau[perm], site[perm], Mt[np.ix_(perm, perm)], lib),
                oracle.nfft(d, beta, tau, site, Mt, lib))


def pin_nfft_numpy(lib):
    """The same transform as two numpy matrix products, Phi Mtau Phi^H / (beta Nc)."""
    d, beta, tau, site, Mt = _config(n=7, seed=11)
    w, kx, ky = _kw(d, beta)
    sx, sy = site % d.Lx, site // d.Lx
    phase = w[:, None] * tau[None, :] - (kx[:, None] * sx[None, :] + ky[:, None] * sy[None, :])
    Phi = np.exp(1j * phase)
    return _rel(oracle.nfft(d, beta, tau, site, Mt, lib), Phi @ Mt @ Phi.conj().T / (beta * d.Nc))


def pin_nfft_entries(lib):
    """Single entries agree with the full transform."""
    d, beta, tau, site, Mt = _config()
    M = oracle.nfft(d, beta, tau, site, Mt, lib)
    K1 = np.array([0, 5, 23, 11]); K2 = np.array([7, 5, 0, 19])
    return _rel(oracle.nfft_entries(d, beta, tau, site, Mt, K1, K2, lib), M[K1, K2])


PINS = {
    "closed_form": (lambda lib: pin_closed_form(lib), 1e-13),
    "closed_form_zeeman": (lambda lib: pin_closed_form(lib, h=0.45), 1e-13),
    "build_G": (pin_build_G, 1e-13),
    "wick_2x2": (lambda lib: pin_wick(lib, (2, 2, 2, 3, 4)), 1e-12),
    "wick_1x1": (lambda lib: pin_wick(lib, (1, 1, 3, 4, 1)), 1e-12),
    "wick_4x2": (lambda lib: pin_wick(lib, (4, 2, 1, 2, 8)), 1e-12),
    "translation_gauge": (pin_translation_gauge, 1e-12),
    "time_gauge": (pin_time_gauge, 1e-12),
    "spin_swap": (pin_spin_swap, 1e-12),
    "sign_flip": (pin_sign_flip, 1e-12),
    "batch_split": (pin_batch_split, 1e-12),
    "conjugation": (pin_conjugation, 1e-12),
    "selection_rule": (pin_selection_rule, 1e-12),
    "numpy_cross": (pin_numpy_cross, 1e-12),
    "nfft_time_translation": (pin_nfft_time_translation, 1e-12),
    "nfft_lattice_translation": (pin_nfft_lattice_translation, 1e-12),
    "nfft_antiperiodic": (pin_nfft_antiperiodic, 1e-12),
    "nfft_momentum_sum": (pin_nfft_momentum_sum, 1e-12),
    "nfft_hermitian": (pin_nfft_hermitian, 1e-12),
    "nfft_permutation": (pin_nfft_permutation, 1e-12),
    "nfft_numpy": (pin_nfft_numpy, 1e-12),
    "nfft_entries": (pin_nfft_entries, 1e-12),
}
for _name, _ch in (("density", 2), ("transverse", 3), ("pp", 1)):
    PINS["closed_form_%s" % _name] = (lambda lib, c=_ch: pin_closed_form(lib, 0.0, c), 1e-13)
    PINS["closed_form_zeeman_%s" % _name] = (lambda lib, c=_ch: pin_closed_form(lib, 0.45, c), 1e-13)
    PINS["wick_2x2_%s" % _name] = (lambda lib, c=_ch: pin_wick(lib, (2, 2, 2, 3, 4), c), 1e-12)
    PINS["wick_4x2_%s" % _name] = (lambda lib, c=_ch: pin_wick(lib, (4, 2, 1, 2, 8), c), 1e-12)
    PINS["translation_gauge_%s" % _name] = (lambda lib, c=_ch: pin_translation_gauge(lib, channel=c), 1e-12)
    PINS["time_gauge_%s" % _name] = (lambda lib, c=_ch: pin_time_gauge(lib, channel=c), 1e-12)
    PINS["spin_swap_%s" % _name] = (lambda lib, c=_ch: pin_spin_swap(lib, c), 1e-12)


def failing_pins(lib, first_only=False):
    bad = []
    for name, (fn, tol) in PINS.items():
        try:
            err = fn(lib)
        except Exception as e:  # a crash counts as a failure
            bad.append((name, repr(e)))
        else:
            if not (err <= tol):
                bad.append((name, err))
        if bad and first_only:
            break
    return bad
