"""The C-ABI library builds, loads and exports every entry point that
include/g4.h declares; argument checks that run before any CUDA call (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2105_00027_gb300 import g4

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "g4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(g4_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(g4.LIB_PATH):
        from paper_2105_00027_gb300 import build
        build.build()
    return g4.load()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert set(names) == set(g4.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_options_defaults(lib):
    o = g4.Options()
    assert lib.g4_options_init(ctypes.byref(o)) == g4.G4_OK
    assert o.precision == g4.PRECISION["mixed"] and o.batch == 64 and o.stream is None
    assert o.autotune == 1 and o.exchange == 0
    assert lib.g4_options_init(None) == g4.G4_ERR_INVALID


@pytest.mark.parametrize("args", [
    (0, 4, 1, 1), (4, 0, 1, 1), (4, 4, 0, 1), (4, 4, 1, 5), (257, 4, 1, 1), (4, 65, 1, 1),
])
def test_create_rejects_bad_sizes(lib, args):
    h = ctypes.c_void_p()
    st = lib.g4_create(*args, 0, None, ctypes.byref(h))
    assert st == g4.G4_ERR_INVALID
    assert h.value is None
    assert lib.g4_last_error(None)


def test_create_rejects_bad_options(lib):
    o = g4.Options()
    lib.g4_options_init(ctypes.byref(o))
    h = ctypes.c_void_p()
    o.batch = 1000
    assert lib.g4_create(4, 2, 1, 1, 0, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
    o.batch = 16
    o.lx = 3  # does not divide Nc = 4
    assert lib.g4_create(4, 2, 1, 1, 0, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
    o.lx = 0
    assert lib.g4_create(8, 2, 1, 1, 0, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
    assert lib.g4_create(4, 2, 1, 1, 7, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
    assert lib.g4_create(4, 2, 1, 1, 4, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
    assert lib.g4_create(4, 2, 1, 1, 0, ctypes.byref(o), None) == g4.G4_ERR_INVALID
    o.exchange = 3
    assert lib.g4_create(4, 2, 1, 1, 0, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID


def test_null_handle_calls(lib):
    assert lib.g4_accumulate(None) == g4.G4_ERR_INVALID
    assert lib.g4_compute_G(None, None, None, 1.0) == g4.G4_ERR_INVALID
    assert lib.g4_finalize(None, None, None) == g4.G4_ERR_INVALID
    assert lib.g4_reset(None) == g4.G4_ERR_INVALID
    assert lib.g4_build_G(0, None, None, None, None) == g4.G4_ERR_INVALID
    assert lib.g4_compute_G_vertices(None, 1.0, 0, 0, None, None, None, None, 1.0) == g4.G4_ERR_INVALID
    assert lib.g4_vertex_M(None, 1.0, 0, 0, None, None, None, None) == g4.G4_ERR_INVALID
    assert lib.g4_reserve_vertices(None, 10) == g4.G4_ERR_INVALID
    lib.g4_destroy(None)


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "g4.h")).read()
    assert int(re.search(r"#define G4_MAX_VERTICES (\d+)", src).group(1)) == g4.MAX_VERTICES
    assert int(re.search(r"#define G4_NOALLOC_MAX_N (\d+)", src).group(1)) == g4.NOALLOC_MAX_N
    kinds = {m.group(1).lower(): int(m.group(2))
             for m in re.finditer(r"G4_K_([A-Z0-9_]+) = (\d+)", src)}
    count = kinds.pop("count")
    assert count == len(g4.KERNEL_KINDS)
    assert sorted(kinds.values()) == sorted(g4.KERNEL_KINDS.values())


def test_options_struct_matches_header():
    """The binding's Options mirrors g4_options field by field, in order."""
    src = open(os.path.join(ROOT, "include", "g4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*g4_options;", src, flags=re.S).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [re.findall(r"[A-Za-z_]\w*", part)[-1] for part in decl.split(",")]
    assert names == [f[0] for f in g4.Options._fields_]


def test_create_rejects_bad_deferred_options(lib):
    """Deferred staging needs the mixed path with the tensor-core exchange."""
    h = ctypes.c_void_p()
    for precision, exchange, deferred in ((g4.PRECISION["mixed"], 0, 2),
                                          (g4.PRECISION["fp64"], 0, 1),
                                          (g4.PRECISION["mixed"], 1, 1)):
        o = g4.Options()
        lib.g4_options_init(ctypes.byref(o))
        o.precision, o.exchange, o.deferred = precision, exchange, deferred
        assert lib.g4_create(4, 2, 1, 1, 0, ctypes.byref(o), ctypes.byref(h)) == g4.G4_ERR_INVALID
        assert h.value is None
