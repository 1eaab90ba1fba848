"""Python binding of the C ABI in include/g4.h (argument marshalling only).

Every step of the G4 path runs in the CUDA library; this module only turns
torch tensors into device pointers and status codes into exceptions.  There
is no CPU fallback: if ``_build/libg4.so`` is missing the import of the
library raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libg4.so")

G4_OK, G4_ERR_INVALID, G4_ERR_OOM, G4_ERR_CUDA, G4_ERR_STATE, G4_ERR_ZERO_SIGN, G4_ERR_TIMEOUT = range(7)
G4_PH_MAGNETIC = 0
CHANNELS = {"ph_magnetic": 0, "pp_updown": 1, "ph_density": 2, "ph_transverse": 3}
PRECISION = {"fp64": 0, "mixed": 1}

STATUS_NAMES = {0: "G4_OK", 1: "G4_ERR_INVALID", 2: "G4_ERR_OOM", 3: "G4_ERR_CUDA",
                4: "G4_ERR_STATE", 5: "G4_ERR_ZERO_SIGN", 6: "G4_ERR_TIMEOUT"}

# every entry point declared in include/g4.h
EXPORTS = ["g4_options_init", "g4_create", "g4_compute_G", "g4_accumulate", "g4_accumulate_group",
           "g4_finalize", "g4_reset", "g4_checkpoint", "g4_restore", "g4_query", "g4_last_error",
           "g4_destroy", "g4_build_G", "g4_profile", "g4_profile_read", "g4_update_noalloc",
           "g4_compute_G_vertices", "g4_vertex_M", "g4_reserve_vertices"]
MAX_VERTICES = 16384
NOALLOC_MAX_N = 256
KERNEL_KINDS = {"build_G": 0, "pack": 1, "direct": 2, "exchange": 3, "update_fp64": 4,
                "finalize": 5, "pack_exchange": 6, "nfft": 7, "direct_split": 8,
                "direct_merge": 9}
EXCHANGE_KERNELS = {"auto": 0, "cuda_cores": 1, "tensor_cores": 2}
OPERANDS = {"fp16": 0, "tf32": 1}
ACCUM = {"fp64": 0, "f32pair": 1}


class G4Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("batch", ctypes.c_int), ("lx", ctypes.c_int),
                ("m_complex64", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("timeout_cycles", ctypes.c_longlong), ("mem_limit", ctypes.c_longlong),
                ("autotune", ctypes.c_int), ("exchange", ctypes.c_int),
                ("direct_batches", ctypes.c_int), ("wex_first", ctypes.c_int),
                ("wex_count", ctypes.c_int), ("operands", ctypes.c_int),
                ("accum", ctypes.c_int), ("deferred", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libg4.so (raises OSError with a build hint if it is missing)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise OSError("libg4.so is not built (%s); run paper_2105_00027_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    P = ctypes.c_void_p
    st = ctypes.c_int
    sig = {
        "g4_options_init": ([ctypes.POINTER(Options)], st),
        "g4_create": ([ctypes.c_int] * 4 + [ctypes.c_int, ctypes.POINTER(Options),
                                            ctypes.POINTER(ctypes.c_void_p)], st),
        "g4_compute_G": ([H, P, P, ctypes.c_double], st),
        "g4_compute_G_vertices": ([H, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                   ctypes.c_double], st),
        "g4_vertex_M": ([H, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P], st),
        "g4_reserve_vertices": ([H, ctypes.c_int], st),
        "g4_accumulate": ([H], st),
        "g4_accumulate_group": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int], st),
        "g4_finalize": ([H, P, ctypes.POINTER(ctypes.c_double)], st),
        "g4_reset": ([H], st),
        "g4_checkpoint": ([H, ctypes.c_char_p], st),
        "g4_restore": ([H, ctypes.c_char_p], st),
        "g4_query": ([H, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)], st),
        "g4_last_error": ([H], ctypes.c_char_p),
        "g4_destroy": ([H], None),
        "g4_build_G": ([ctypes.c_int, P, P, P, P], st),
        "g4_profile": ([H, ctypes.c_int], st),
        "g4_update_noalloc": ([ctypes.c_int] * 5 + [P, P, ctypes.c_double, P, P], st),
        "g4_profile_read": ([H, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_longlong)], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path == LIB_PATH:
        _lib = lib
    return lib


def _check(lib, h, status):
    if status != G4_OK:
        msg = lib.g4_last_error(h)
        raise G4Error(status, msg.decode() if msg else "")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _vptr(t):
    """Device pointer of a possibly empty tensor (NULL when empty)."""
    return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() > 0 else None)


def _stream_of(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class G4:
    """One G4 problem (handle of the C ABI).  With deferred=True (mixed path,
    tensor-core exchange) compute_G only records M, G0 and the sign; the
    accumulation forms the operands from M, which must stay on the device,
    unchanged and 16-byte aligned, until its batch has been accumulated."""

    def __init__(self, Nc, Nw, Nwex, Nkex, precision="mixed", batch=64, lx=0,
                 m_complex64=False, stream=None, mem_limit=0, timeout_cycles=0, autotune=True,
                 channel="ph_magnetic", exchange="auto", direct_batches=0, wex_slab=None,
                 operands="fp16", accum="fp64", deferred=False):
        self.lib = load()
        opt = Options()
        self.lib.g4_options_init(ctypes.byref(opt))
        opt.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        opt.batch = batch
        opt.lx = lx
        opt.m_complex64 = int(bool(m_complex64))
        opt.stream = _stream_of(stream)
        opt.mem_limit = mem_limit
        opt.timeout_cycles = timeout_cycles
        opt.autotune = int(bool(autotune))
        opt.exchange = EXCHANGE_KERNELS[exchange] if isinstance(exchange, str) else int(exchange)
        opt.direct_batches = int(direct_batches)
        if wex_slab is not None:
            opt.wex_first, opt.wex_count = int(wex_slab[0]), int(wex_slab[1])
        opt.operands = OPERANDS[operands] if isinstance(operands, str) else int(operands)
        opt.accum = ACCUM[accum] if isinstance(accum, str) else int(accum)
        opt.deferred = int(bool(deferred))
        self.opt = opt
        h = ctypes.c_void_p()
        ch = CHANNELS[channel] if isinstance(channel, str) else int(channel)
        st = self.lib.g4_create(Nc, Nw, Nwex, Nkex, ch, ctypes.byref(opt), ctypes.byref(h))
        _check(self.lib, None, st)
        self.h = h
        self.Nc, self.Nw, self.Nkex = Nc, Nw, Nkex
        self.Nwex = wex_slab[1] if wex_slab is not None and wex_slab[1] > 0 else Nwex
        self.N = Nc * 2 * Nw
        self.E = self.N * self.N * Nkex * self.Nwex

    @classmethod
    def for_problem(cls, p, precision="mixed", batch=None, **kw):
        return cls(p.Nc, p.Nw, p.Nwex, p.Nkex, precision=precision,
                   batch=batch or p.batch, lx=p.Lx, m_complex64=(p.m_dtype == "c64"), **kw)

    def compute_G(self, M, G0, sign):
        """Stage one measurement: M [2][N][N] and G0 [2][N] on the device."""
        _check(self.lib, self.h, self.lib.g4_compute_G(self.h, _ptr(M), _ptr(G0), float(sign)))

    def compute_G_vertices(self, beta, n_up, n_dn, tau, site, Mtau, G0, sign):
        """Stage a measurement from its vertex configuration: tau (float64),
        site (int32), Mtau (float64, both spin blocks) as CUDA tensors."""
        _check(self.lib, self.h, self.lib.g4_compute_G_vertices(
            self.h, float(beta), int(n_up), int(n_dn), _vptr(tau), _vptr(site), _vptr(Mtau),
            _ptr(G0), float(sign)))

    def vertex_M(self, beta, n_up, n_dn, tau, site, Mtau, M=None):
        """M of both spins from a vertex configuration ([2][N][N], complex128 on
        an FP64 handle, complex64 on a mixed one); synchronous."""
        import torch
        if M is None:
            dt = torch.complex128 if self.opt.precision == PRECISION["fp64"] else torch.complex64
            M = torch.empty((2, self.N, self.N), dtype=dt, device=tau.device)
        _check(self.lib, self.h, self.lib.g4_vertex_M(
            self.h, float(beta), int(n_up), int(n_dn), _vptr(tau), _vptr(site), _vptr(Mtau),
            _ptr(M)))
        return M

    def reserve_vertices(self, n_max):
        _check(self.lib, self.h, self.lib.g4_reserve_vertices(self.h, int(n_max)))

    def accumulate(self):
        _check(self.lib, self.h, self.lib.g4_accumulate(self.h))

    def finalize(self, out=None, allow_zero_sign=False):
        """Return (G4 in the exported order [m][n2][n1][q][k2][k1], sign sum)."""
        import torch
        if out is None:
            out = torch.empty((self.Nwex, 2 * self.Nw, 2 * self.Nw, self.Nkex, self.Nc, self.Nc),
                              dtype=torch.complex128, device="cuda")
        S = ctypes.c_double(0.0)
        st = self.lib.g4_finalize(self.h, _ptr(out), ctypes.byref(S))
        if not (allow_zero_sign and st == G4_ERR_ZERO_SIGN):
            _check(self.lib, self.h, st)
        return out, S.value

    def reset(self):
        _check(self.lib, self.h, self.lib.g4_reset(self.h))

    def checkpoint(self, path):
        _check(self.lib, self.h, self.lib.g4_checkpoint(self.h, str(path).encode()))

    def restore(self, path):
        _check(self.lib, self.h, self.lib.g4_restore(self.h, str(path).encode()))

    def query(self):
        e, m = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib, self.h, self.lib.g4_query(self.h, ctypes.byref(e), ctypes.byref(m)))
        return e.value, m.value

    def profile(self, enable=True):
        _check(self.lib, self.h, self.lib.g4_profile(self.h, int(bool(enable))))

    def profile_read(self, kind):
        """(total device ms, launches) recorded for one kernel kind since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        _check(self.lib, self.h, self.lib.g4_profile_read(self.h, k, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.g4_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def accumulate_group(handles):
    lib = load()
    arr = (ctypes.c_void_p * len(handles))(*[h.h.value for h in handles])
    st = lib.g4_accumulate_group(arr, len(handles))
    if st != G4_OK:
        for h in handles:
            msg = lib.g4_last_error(h.h)
            if msg:
                raise G4Error(st, msg.decode())
        raise G4Error(st, "")


def build_G(M, G0, G=None, stream=None):
    """G = G0 d - G0 M G0 for both spins (M [2][N][N], G0 [2][N], complex128)."""
    import torch
    lib = load()
    if G is None:
        G = torch.empty_like(M)
    N = M.shape[-1]
    _check(lib, None, lib.g4_build_G(N, _ptr(M), _ptr(G0), _ptr(G), ctypes.c_void_p(_stream_of(stream))))
    return G


def update_noalloc(Nc, Nw, Nwex, Nkex, M, G0, sign, acc, lx=0, stream=None):
    """acc += sign * (direct - exchange) for one measurement, allocating nothing.

    For callers that cannot allocate device memory at update time: the
    intermediate G lives in a fixed 2 MiB array inside the library, which
    limits N = Nc * 2Nw to NOALLOC_MAX_N.  ``acc`` (complex128, exported
    layout) is owned, zeroed and normalised by the caller.  Calls that can
    overlap on the GPU race on the shared array."""
    import torch
    N = Nc * 2 * Nw
    E = N * N * Nkex * Nwex
    dev = torch.cuda.current_device()
    # the library receives bare pointers: shapes, types and devices are checked here
    for name, t, numel in (("M", M, 2 * N * N), ("G0", G0, 2 * N), ("acc", acc, E)):
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != torch.complex128:
            raise ValueError("%s must be complex128 (got %s)" % (name, t.dtype))
        if not t.is_cuda or t.device.index != dev:
            raise ValueError("%s must be on the current CUDA device (cuda:%d)" % (name, dev))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.numel() != numel:
            raise ValueError("%s has %d entries, expected %d" % (name, t.numel(), numel))
    lib = load()
    _check(lib, None, lib.g4_update_noalloc(Nc, lx, Nw, Nwex, Nkex, _ptr(M), _ptr(G0),
                                            float(sign), _ptr(acc),
                                            ctypes.c_void_p(_stream_of(stream))))
    return acc
