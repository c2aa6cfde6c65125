"""The C-ABI library builds, loads and exports every function include/vr.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_1902_01010_gb300 import _build, vr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vr_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    L = ctypes.CDLL(path)
    declared = _declared()
    assert "vr_fof3d" in declared and "vr_find_substructure" in declared
    missing = [s for s in declared if not hasattr(L, s)]
    assert not missing, missing
    assert set(vr.EXPORTS) <= declared


def test_params_default_is_table1():
    p = vr.Params.default()
    assert (p.nse, p.nv, p.nmin) == (256, 32, 20)
    assert p.f_cell == 0.01 and p.ell_th == 2.5 and p.v_ratio == 2.0
    assert abs(p.theta_op - 0.1 * 3.141592653589793) < 1e-15
