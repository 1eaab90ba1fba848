"""CPU oracle for the G4 measurement step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_2105_00027_gb300``) never imports it, and this package
never imports the product path.

The arithmetic lives in ``g4_oracle.c`` (complex128 loops written as the
definitions read; see its header).  This module compiles it with gcc, loads
it with ctypes and adds numpy-side helpers:

* :func:`build_G` -- G = G0 d - G0 M G0 for one spin (Sec. 2, G_sigma generation).
* :func:`accumulate` / :func:`run` / :func:`run_stream` -- the sign-weighted
  G4 sum evaluated on selected (q, m) slabs, for the particle-hole magnetic
  channel (default), the particle-particle up-down channel printed as Eq. (1)
  (Sec. 2.1), and the particle-hole density and transverse channels.
* :func:`nfft` / :func:`nfft_entries` -- M of one spin's vertex configuration
  by the non-uniform Fourier transform (the step before the G build, Sec. 2).
* :func:`errors` -- the normalised entrywise L1 and L2 errors of Eqs. (2)-(3)
  (Sec. 4.3), plus the real/imaginary split of Table 1.
* :func:`to_exported` -- assemble full slabs into the exported
  [m][n2][n1][q][k2][k1] order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "g4_oracle.c")
LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(src: str = SRC, out: str = LIB, extra_flags=()) -> str:
    """Compile the C oracle into a shared library (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fcx-limited-range", *extra_flags, src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


class Dims(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("Nw", ctypes.c_int),
                ("Nwex", ctypes.c_int), ("Nkex", ctypes.c_int)]

    @property
    def Nc(self):
        return self.Lx * self.Ly

    @property
    def Nw2(self):
        return 2 * self.Nw

    @property
    def N(self):
        return self.Nc * self.Nw2


def _setup(lib):
    P = ctypes.c_void_p
    lib.g4o_build_G.argtypes = [ctypes.c_int, P, P, P]
    lib.g4o_build_G.restype = None
    lib.g4o_accumulate.argtypes = [ctypes.POINTER(Dims), P, P, ctypes.c_double,
                                   P, P, ctypes.c_int, P, ctypes.c_int]
    lib.g4o_accumulate.restype = None
    lib.g4o_run.argtypes = [ctypes.POINTER(Dims), ctypes.c_int, P, P, P, P, P,
                            ctypes.c_int, P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.g4o_run.restype = ctypes.c_int
    lib.g4o_kplus.argtypes = [ctypes.POINTER(Dims), ctypes.c_int, ctypes.c_int]
    lib.g4o_kplus.restype = ctypes.c_int
    lib.g4o_accumulate_ch.argtypes = lib.g4o_accumulate.argtypes + [ctypes.c_int]
    lib.g4o_accumulate_ch.restype = None
    lib.g4o_run_ch.argtypes = lib.g4o_run.argtypes + [ctypes.c_int]
    lib.g4o_run_ch.restype = ctypes.c_int
    lib.g4o_nfft.argtypes = [ctypes.POINTER(Dims), ctypes.c_double, ctypes.c_int, P, P, P, P]
    lib.g4o_nfft.restype = None
    lib.g4o_nfft_entries.argtypes = [ctypes.POINTER(Dims), ctypes.c_double, ctypes.c_int, P, P, P,
                                     ctypes.c_int, P, P, P]
    lib.g4o_nfft_entries.restype = None
    return lib


def load(path: str = LIB, rebuild_if_missing: bool = True):
    """Load (building first if needed) the oracle library."""
    global _lib
    if path == LIB and _lib is not None:
        return _lib
    if not os.path.exists(path) or (path == LIB and os.path.getmtime(path) < os.path.getmtime(SRC)):
        if not rebuild_if_missing:
            raise FileNotFoundError(path)
        build(out=path)
    lib = _setup(ctypes.CDLL(path))
    if path == LIB:
        _lib = lib
    return lib


def dims(Lx, Ly, Nw, Nwex, Nkex) -> Dims:
    return Dims(Lx, Ly, Nw, Nwex, Nkex)


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def build_G(M, G0, lib=None):
    """G = G0 d - G0 M G0 for one spin; M (N, N), G0 (N,) complex128."""
    lib = lib or load()
    M = _c128(M)
    G0 = _c128(G0)
    N = G0.shape[0]
    assert M.shape == (N, N)
    G = np.empty((N, N), np.complex128)
    lib.g4o_build_G(N, _ptr(M), _ptr(G0), _ptr(G))
    return G


def nfft(d: Dims, beta, tau, site, Mtau, lib=None):
    """M(K1, K2) of one spin's vertex configuration by the non-uniform Fourier
    transform (the double sum, see g4o_nfft); tau (n,), site (n,) ints,
    Mtau (n, n) complex128.  Returns (N, N) complex128."""
    lib = lib or load()
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    site = np.ascontiguousarray(site, dtype=np.int32)
    Mtau = _c128(Mtau)
    n = tau.shape[0]
    assert site.shape == (n,) and Mtau.shape == (n, n)
    M = np.empty((d.N, d.N), np.complex128)
    lib.g4o_nfft(ctypes.byref(d), float(beta), n, _ptr(tau), _ptr(site), _ptr(Mtau), _ptr(M))
    return M


def nfft_entries(d: Dims, beta, tau, site, Mtau, K1s, K2s, lib=None):
    """Selected entries M(K1s[e], K2s[e]) of :func:`nfft`."""
    lib = lib or load()
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    site = np.ascontiguousarray(site, dtype=np.int32)
    Mtau = _c128(Mtau)
    K1s = np.ascontiguousarray(K1s, dtype=np.int32)
    K2s = np.ascontiguousarray(K2s, dtype=np.int32)
    out = np.empty(len(K1s), np.complex128)
    lib.g4o_nfft_entries(ctypes.byref(d), float(beta), tau.shape[0], _ptr(tau), _ptr(site), _ptr(Mtau),
                         len(K1s), _ptr(K1s), _ptr(K2s), _ptr(out))
    return out


def all_slabs(d: Dims):
    """(qsel, msel) enumerating every transfer Q = (q, m), q-major."""
    q, m = np.meshgrid(np.arange(d.Nkex), np.arange(d.Nwex), indexing="ij")
    return q.ravel().astype(np.int32), m.ravel().astype(np.int32)


def _sel(d, qsel, msel):
    if qsel is None:
        return all_slabs(d)
    return (np.ascontiguousarray(qsel, dtype=np.int32),
            np.ascontiguousarray(msel, dtype=np.int32))


CHANNELS = {"ph_magnetic": 0, "pp_updown": 1, "ph_density": 2, "ph_transverse": 3}


def _ch(channel):
    return CHANNELS[channel] if isinstance(channel, str) else int(channel)


def accumulate(d: Dims, Gup, Gdn, sign, acc, qsel, msel, nthreads=0, lib=None, channel=0):
    """acc[s] += sign * (the channel's term) of one measurement on slabs s."""
    lib = lib or load()
    Gup, Gdn = _c128(Gup), _c128(Gdn)
    assert acc.dtype == np.complex128 and acc.flags.c_contiguous
    qsel, msel = _sel(d, qsel, msel)
    lib.g4o_accumulate_ch(ctypes.byref(d), _ptr(Gup), _ptr(Gdn), float(sign), _ptr(qsel),
                          _ptr(msel), len(qsel), _ptr(acc), int(nthreads), _ch(channel))


def run(d: Dims, M, G0, signs, qsel=None, msel=None, nthreads=0, lib=None, channel=0):
    """Whole run.  M (R, 2, N, N), G0 (2, N), signs (R,).

    Returns (slabs[nsel][Nw2][Nw2][Nc][Nc] normalised by the sign sum, S).
    If S == 0 the slabs are the unnormalised sums.
    """
    lib = lib or load()
    M = _c128(M)
    G0 = _c128(G0)
    signs = np.ascontiguousarray(signs, dtype=np.float64)
    qsel, msel = _sel(d, qsel, msel)
    R = M.shape[0]
    assert M.shape == (R, 2, d.N, d.N) and G0.shape == (2, d.N) and signs.shape == (R,)
    out = np.empty((len(qsel), d.Nw2, d.Nw2, d.Nc, d.Nc), np.complex128)
    S = ctypes.c_double(0.0)
    rc = lib.g4o_run_ch(ctypes.byref(d), R, _ptr(M), _ptr(G0), _ptr(signs), _ptr(qsel),
                        _ptr(msel), len(qsel), _ptr(out), ctypes.byref(S), int(nthreads),
                        _ch(channel))
    if rc not in (0, 5):
        raise MemoryError("oracle run failed: %d" % rc)
    return out, S.value


def run_stream(d: Dims, measurements, G0, qsel=None, msel=None, nthreads=0, lib=None,
               channel=0):
    """Like :func:`run`, but takes an iterable of (M_r (2,N,N), s_r) pairs so
    that large runs never hold every M at once."""
    lib = lib or load()
    qsel, msel = _sel(d, qsel, msel)
    G0 = _c128(G0)
    acc = np.zeros((len(qsel), d.Nw2, d.Nw2, d.Nc, d.Nc), np.complex128)
    S = 0.0
    for Mr, sr in measurements:
        Gup = build_G(Mr[0], G0[0], lib)
        Gdn = build_G(Mr[1], G0[1], lib)
        accumulate(d, Gup, Gdn, sr, acc, qsel, msel, nthreads, lib, channel)
        S += float(sr)
    if S != 0.0:
        acc /= S
    return acc, S


def to_exported(d: Dims, slabs_all):
    """slabs over every Q (q-major, as :func:`all_slabs`) -> exported order
    [m][n2][n1][q][k2][k1]."""
    s = np.asarray(slabs_all).reshape(d.Nkex, d.Nwex, d.Nw2, d.Nw2, d.Nc, d.Nc)
    return np.ascontiguousarray(s.transpose(1, 2, 3, 0, 4, 5))


def slabs_from_exported(d: Dims, exported, qsel, msel):
    """Pick slabs [s][n2][n1][k2][k1] out of an exported-order array."""
    e = np.asarray(exported).reshape(d.Nwex, d.Nw2, d.Nw2, d.Nkex, d.Nc, d.Nc)
    return np.stack([e[m, :, :, q] for q, m in zip(qsel, msel)])


def errors(ref, test):
    """Normalised entrywise errors of Eqs. (2)-(3) (Sec. 4.3).

    Returns dict with complex-modulus L1 and L2 (L2 = relative Frobenius),
    and the real/imaginary split used by Table 1.
    """
    ref = np.asarray(ref).ravel()
    test = np.asarray(test).ravel()
    diff = test - ref

    def l1(a, b):
        den = np.sum(np.abs(b))
        return float(np.sum(np.abs(a)) / den) if den > 0 else float(np.sum(np.abs(a)))

    def l2(a, b):
        den = np.linalg.norm(b)
        return float(np.linalg.norm(a) / den) if den > 0 else float(np.linalg.norm(a))

    return {
        "L1": l1(diff, ref), "L2": l2(diff, ref),
        "L1_re": l1(diff.real, ref.real), "L1_im": l1(diff.imag, ref.imag),
        "L2_re": l2(diff.real, ref.real), "L2_im": l2(diff.imag, ref.imag),
    }
