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


def _golden():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "table1_defaults.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def test_core_defaults_are_table1():
    """vr_core_params_default and vr_core_grow_params_default give the core-search and
    core-growth defaults the paper prints (Table 1; Table A1 for the growth mode)."""
    g = _golden()
    c = vr.CoreParams.default()
    assert (c.alpha_x, c.alpha_v, c.n_loop, c.f_c, c.alpha_n) == (
        g["alpha_xC"], g["alpha_vC"], g["n_loopC"], g["f_C"], g["alpha_NC"])
    cg = vr.CoreGrowParams.default()
    assert (cg.beta_c, cg.mode) == (g["beta_C"], g["core_growth_mode"])


def test_no_fallback_without_the_library(monkeypatch, tmp_path):
    """With libvr.so missing (and no build), the binding raises instead of computing
    anything on the host."""
    import pytest

    monkeypatch.setattr(vr, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libvr.so"))
    with pytest.raises(RuntimeError):
        vr.lib(build_if_missing=False)


def test_context_needs_a_gpu():
    """Without a usable CUDA device, creating a context fails with a library status."""
    import pytest
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(vr.VrError):
        vr.Context(0)


def test_noalloc_scratch_fits_the_stated_maximum():
    """The 3D FOF scratch for n = VR_FOF3D_NOALLOC_MAX_N fits the static array of
    VR_FOF3D_NOALLOC_BYTES (host-side size function of the library; no GPU needed), so
    every n up to the stated maximum is accepted."""
    src = open(os.path.join(ROOT, "include", "vr.h")).read()
    max_n = int(re.search(r"#define VR_FOF3D_NOALLOC_MAX_N (\d+)", src).group(1))
    m = re.search(r"#define VR_FOF3D_NOALLOC_BYTES \((\d+)u << (\d+)\)", src)
    nbytes = int(m.group(1)) << int(m.group(2))
    L = ctypes.CDLL(_build.build())
    ws = getattr(L, "_ZN2vr8ws_fof3dEl")  # size_t vr::ws_fof3d(int64_t)
    ws.restype = ctypes.c_size_t
    ws.argtypes = [ctypes.c_int64]
    need = ws(max_n)
    assert 0 < need <= nbytes, (need, nbytes)
    assert ws(max_n + 1) >= need  # the size grows with n


def test_log_level_rejects_bad_arguments_without_a_gpu():
    """vr_set_log_level needs a context: NULL (and so any call made here, without a GPU)
    returns VR_ERR_INVALID_ARG instead of touching memory."""
    L = ctypes.CDLL(_build.build())
    f = L.vr_set_log_level
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert f(None, 1) == 1 and f(None, 0) == 1
