"""The C-ABI library builds, loads and exports every symbol the header
declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(dm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2311_18126_gb300 import ensure_built
    lib = ensure_built()
    names = _declared_functions()
    assert "dm_step" in names and "dm_create_system" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_descriptor_is_rejected_without_gpu_work():
    import numpy as np
    from paper_2311_18126_gb300 import System, DismechError
    bad = dict(nodes_per_rod=[1], x0=np.zeros((1, 3)), E=[1e7], nu=[0.5], rho=[1e3],
               radius=[1e-3])
    with pytest.raises(DismechError) as ei:
        System(bad, dict(dt=1e-3))
    assert ei.value.code == 1


def test_band_solve_batch_rules_are_checked_before_gpu_work():
    # the banded solves update each system's rows in place and accumulate
    # into x: overlapping systems, and an x that overlaps band or rhs, are
    # rejected with DM_ERR_INVALID_ARG before any device call (the pointers
    # below are never dereferenced)
    import ctypes as C
    from paper_2311_18126_gb300 import ensure_built
    lib = ensure_built()
    n = 100
    base = 1 << 40
    band, rhs, x = base, base + 11 * n * 8 + 4096, base + 13 * n * 8 + 8192
    ip = C.POINTER(C.c_int32)

    def call(fn, d0, nd, band=band, rhs=rhs, x=x, extra=()):
        a = (C.c_int32 * len(d0))(*d0)
        b = (C.c_int32 * len(nd))(*nd)
        return fn(len(d0), C.cast(a, ip), C.cast(b, ip), C.c_int64(n), C.c_void_p(band),
                  C.c_void_p(rhs), C.c_void_p(x), *extra, None)

    for name, extra in (("dm_solve_band", ()), ("dm_solve_band_noalloc", ()),
                        ("dm_solve_band_partitioned", (C.c_int32(0),))):
        fn = getattr(lib, name)
        fn.restype = C.c_int
        # systems [0, 50) and [40, 100) share rows 40..49 (given out of order)
        assert call(fn, [40, 0], [60, 50], extra=extra) == 1
        assert b"overlap" in lib.dm_last_error()
        # x == rhs, x inside the band, x straddling the band's end
        assert call(fn, [0], [n], x=rhs, extra=extra) == 1
        assert call(fn, [0], [n], x=band + 5 * n * 8, extra=extra) == 1
        assert call(fn, [0], [n], x=band + 11 * n * 8 - 8, extra=extra) == 1
        assert b"x overlaps" in lib.dm_last_error()
