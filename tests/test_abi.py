"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/igg.h declares, and rejects invalid arguments on the host
(before any CUDA call) with the documented status codes."""
import ctypes
import os
import re

import pytest

from paper_2211_15716_gb300 import build as igg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    igg_build.build()
    from paper_2211_15716_gb300 import igg
    return igg.lib()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(igg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("igg_init_global_grid", "igg_finalize_global_grid", "igg_global_size",
              "igg_update_halo", "igg_step", "igg_step_hidden", "igg_run", "igg_reduce"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_abi_version(L):
    L.igg_abi_version.restype = ctypes.c_int
    assert L.igg_abi_version() == 1


def _init(L, n=(8, 8, 8), dims=(1, 1, 1), nsub=1, overlap=(2, 2, 2), periods=(0, 0, 0)):
    h = ctypes.c_void_p()
    I3 = ctypes.c_int * 3
    rc = L.igg_init_global_grid(n[0], n[1], n[2], I3(*dims), nsub, I3(*overlap), I3(*periods),
                                ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("kw,frag", [
    (dict(n=(2, 8, 8)), "local size"),
    (dict(overlap=(1, 2, 2)), "overlap"),
    (dict(overlap=(2, 2, 8)), "overlap"),
    (dict(dims=(2, 2, 2), nsub=6), "differs"),
    (dict(dims=(0, 3, 0), nsub=7), "cannot factor"),
])
def test_invalid_grid_arguments(L, kw, frag):
    rc, h = _init(L, **kw)
    assert rc == -1
    assert frag in L.igg_last_error().decode()
    assert not h.value


def test_null_arguments(L):
    assert L.igg_init_global_grid(8, 8, 8, None, 1, None, None, None) == -1
    ng = (ctypes.c_int * 3)()
    assert L.igg_global_size(None, ng) == -1
    assert L.igg_step(None, None, None, None, 0, 1.0, 1.0, 1.0, 1.0, 1.0, None) == -1
    assert L.igg_finalize_global_grid(None) == 0
    assert L.igg_run_host(None, 1, None, None, None, None, None, None, 0, 1.0, 1.0, 1.0, 1.0, 1.0,
                          None) == -1
    ms, n = (ctypes.c_double * 3)(), ctypes.c_int()
    assert L.igg_phase_times(None, ms, ctypes.byref(n)) == -1
    assert L.igg_fixup_stats(None, (ctypes.c_ulonglong * 2)(), 0) == -1
    out = ctypes.c_double()
    assert L.igg_reduce(9, None, None, 0, 0, ctypes.byref(out), None) == -1
    assert L.igg_reduce(0, None, None, 0, 7, ctypes.byref(out), None) == -1


def test_bounds_checked_build_loads_and_reports_itself(L):
    """The bounds-checked library builds beside the release one, exports the
    same functions and says which build it is; both reject a NULL status."""
    path = igg_build.build(checked=True)
    assert path == igg_build.LIB_CHECKED and path != igg_build.LIB
    C = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(C, name), name
    assert C.igg_bounds_checked() == 1
    assert L.igg_bounds_checked() == 0
    for lib in (C, L):
        lib.igg_bounds_status.argtypes = [ctypes.c_void_p, ctypes.c_int]
        assert lib.igg_bounds_status(None, 0) == -1
