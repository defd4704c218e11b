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
