"""Thin ctypes binding of libvr.so (include/vr.h) for torch device tensors.

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
PyTorch supplies device memory (inputs, outputs and the workspace) and the stream.
There is no CPU fallback: if libvr.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

from . import _build

VR_OK = 0
STATUS = {0: "VR_OK", 1: "VR_ERR_INVALID_ARG", 2: "VR_ERR_CUDA", 3: "VR_ERR_WORKSPACE_TOO_SMALL",
          4: "VR_ERR_TIMEOUT", 5: "VR_ERR_DEGENERATE_CELL", 6: "VR_ERR_UNSUPPORTED"}
HALO_COLS = 12
H_LABEL, H_NH, H_SEARCHED, H_RBAR, H_SIGR, H_VFX, H_VFY, H_VFZ, H_SIGMA, H_LX2, H_LV2, H_NCELLS = \
    range(12)

# every symbol include/vr.h declares
EXPORTS = ("vr_params_default", "vr_create", "vr_destroy", "vr_last_error", "vr_workspace_size",
           "vr_sync", "vr_fof3d", "vr_velden", "vr_outlier_ratio", "vr_fof6d",
           "vr_fof6d_field", "vr_clean_groups", "vr_grow_params_default", "vr_grow_groups",
           "vr_core_params_default", "vr_core_search", "vr_core_grow_params_default",
           "vr_core_grow", "vr_find_substructure", "vr_autotune", "vr_tuning_force",
           "vr_tuning_report", "vr_set_log_level")


class VrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    """Mirror of vr_params (include/vr.h)."""

    _fields_ = [
        ("nse", ctypes.c_int32), ("nv", ctypes.c_int32), ("f_cell", ctypes.c_double),
        ("ncell_min", ctypes.c_int32), ("nmin", ctypes.c_int32), ("nsearch_min", ctypes.c_int32),
        ("ell_th", ctypes.c_double), ("v_ratio", ctypes.c_double), ("theta_op", ctypes.c_double),
        ("use_lv", ctypes.c_int32), ("use_vr_theta", ctypes.c_int32),
        ("split_rule", ctypes.c_int32), ("fit_nbins_min", ctypes.c_int32),
        ("fit_nbins_max", ctypes.c_int32), ("fit_iters", ctypes.c_int32),
    ]

    @classmethod
    def default(cls, **kw) -> "Params":
        p = cls()
        lib().vr_params_default(ctypes.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class GrowParams(ctypes.Structure):
    """Mirror of vr_grow_params (include/vr.h): gamma factors of the relaxed pass and
    the merge fraction."""

    _fields_ = [("gamma_ell", ctypes.c_double), ("gamma_x", ctypes.c_double),
                ("gamma_vr", ctypes.c_double), ("gamma_theta", ctypes.c_double),
                ("f_merge", ctypes.c_double)]

    @classmethod
    def default(cls, **kw) -> "GrowParams":
        g = cls()
        lib().vr_grow_params_default(ctypes.byref(g))
        for k, v in kw.items():
            setattr(g, k, v)
        return g


class CoreParams(ctypes.Structure):
    """Mirror of vr_core_params (include/vr.h)."""

    _fields_ = [("alpha_x", ctypes.c_double), ("alpha_v", ctypes.c_double),
                ("n_loop", ctypes.c_int32), ("f_c", ctypes.c_double), ("alpha_n", ctypes.c_double)]

    @classmethod
    def default(cls, **kw) -> "CoreParams":
        c = cls()
        lib().vr_core_params_default(ctypes.byref(c))
        for k, v in kw.items():
            setattr(c, k, v)
        return c


class CoreGrowParams(ctypes.Structure):
    """Mirror of vr_core_grow_params (include/vr.h): beta_C of the cleaning and the
    growth mode."""

    _fields_ = [("beta_c", ctypes.c_double), ("mode", ctypes.c_int32)]

    @classmethod
    def default(cls, **kw) -> "CoreGrowParams":
        g = cls()
        lib().vr_core_grow_params_default(ctypes.byref(g))
        for k, v in kw.items():
            setattr(g, k, v)
        return g


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libvr.so, building it first if it is missing or stale (needs nvcc)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libvr.so not found at {_build.LIB}; run _build.build()")
            L = ctypes.CDLL(_build.LIB)
            vp, i64, i32, dbl, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_size_t)
            P = ctypes.POINTER(Params)
            sig = {
                "vr_params_default": (None, [P]),
                "vr_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int]),
                "vr_destroy": (None, [vp]),
                "vr_last_error": (ctypes.c_char_p, [vp]),
                "vr_workspace_size": (ctypes.c_int, [vp, i64, P, ctypes.POINTER(sz)]),
                "vr_sync": (ctypes.c_int, [vp, vp]),
                "vr_fof3d": (ctypes.c_int, [vp, vp, i64, i64, vp, vp, sz, vp]),
                "vr_velden": (ctypes.c_int, [vp, vp, vp, i64, vp, P, vp, vp, sz, vp]),
                "vr_outlier_ratio": (ctypes.c_int, [vp, vp, vp, vp, i64, vp, P, vp, vp, vp,
                                                    ctypes.POINTER(i64), vp, sz, vp]),
                "vr_fof6d": (ctypes.c_int, [vp, vp, vp, vp, i64, vp, vp, i64, P, vp, vp, sz, vp]),
                "vr_fof6d_field": (ctypes.c_int, [vp, vp, vp, i64, vp, dbl, dbl, P, vp, vp,
                                                  ctypes.POINTER(i64), vp, sz, vp]),
                "vr_clean_groups": (ctypes.c_int, [vp, vp, i64, P, dbl, vp, ctypes.POINTER(i64),
                                                   vp, sz, vp]),
                "vr_grow_params_default": (None, [ctypes.POINTER(GrowParams)]),
                "vr_core_params_default": (None, [ctypes.POINTER(CoreParams)]),
                "vr_core_search": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, dbl, dbl, P,
                                                  ctypes.POINTER(CoreParams), vp, vp,
                                                  ctypes.POINTER(i64), vp, ctypes.POINTER(i64),
                                                  vp, sz, vp]),
                "vr_core_grow_params_default": (None, [ctypes.POINTER(CoreGrowParams)]),
                "vr_core_grow": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, dbl, dbl, P,
                                                ctypes.POINTER(CoreParams),
                                                ctypes.POINTER(CoreGrowParams), vp, vp, vp,
                                                ctypes.POINTER(i64), vp, ctypes.POINTER(i64),
                                                vp, sz, vp]),
                "vr_grow_groups": (ctypes.c_int, [vp, vp, vp, vp, i64, vp, vp, i64, P,
                                                  ctypes.POINTER(GrowParams), vp, vp, sz, vp]),
                "vr_find_substructure": (ctypes.c_int, [vp, vp, vp, i64, vp, dbl, dbl, P,
                                                        ctypes.c_int, vp, vp, vp, vp, vp,
                                                        ctypes.POINTER(i64), vp, sz, vp]),
                "vr_autotune": (ctypes.c_int, [vp, ctypes.c_int]),
                "vr_tuning_force": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
                "vr_tuning_report": (ctypes.c_int, [vp, ctypes.c_char_p, sz]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A vr_ctx on one device plus a reusable workspace tensor."""

    def __init__(self, device: int = 0):
        L = lib()
        h = ctypes.c_void_p()
        st = L.vr_create(ctypes.byref(h), device)
        if st != VR_OK:
            raise VrError(st, f"vr_create({device}) failed")
        self.h = h
        self.device = device
        self.ws = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib(False).vr_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def check(self, st):
        if st != VR_OK:
            msg = lib().vr_last_error(self.h)
            raise VrError(st, msg.decode() if msg else "")

    def workspace(self, n: int, params: Params | None = None) -> torch.Tensor:
        sz = ctypes.c_size_t()
        self.check(lib().vr_workspace_size(self.h, n, ctypes.byref(params) if params else None,
                                           ctypes.byref(sz)))
        if self.ws is None or self.ws.numel() < sz.value:
            self.ws = None
            self.ws = torch.empty(sz.value, dtype=torch.uint8, device=f"cuda:{self.device}")
        return self.ws

    def sync(self, stream=None):
        self.check(lib().vr_sync(self.h, _stream(stream)))

    def log_level(self, level: int):
        """stderr logging of this context: 0 silent, 1 errors, 2 errors and one line per
        3D FOF or substructure call (vr_set_log_level)."""
        self.check(lib().vr_set_log_level(self.h, int(level)))

    # ------------------------------------------------------------ launch shapes
    def autotune(self, enable: bool = True):
        """From the next call on, time every candidate launch shape of the f_l kernel (per
        halo-size bin) and of the 6D linker on the caller's data and keep the fastest
        (vr_autotune); False returns to the defaults."""
        self.check(lib().vr_autotune(self.h, 1 if enable else 0))

    def tuning_force(self, velden_shape: int = -1, link_shape: int = -1):
        """Every later launch uses these shape indices (-1: not forced)."""
        self.check(lib().vr_tuning_force(self.h, int(velden_shape), int(link_shape)))

    def tuning_report(self) -> dict:
        """Candidate shapes, the shapes in use and the measured ms (vr_tuning_report)."""
        import json

        buf = ctypes.create_string_buffer(8192)
        self.check(lib().vr_tuning_report(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    # ------------------------------------------------------------------ calls
    def fof3d(self, pos: torch.Tensor, link_d2: int, label: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
        n = pos.shape[0]
        _check(pos, torch.int32, (n, 3))
        if label is None:
            label = torch.empty(n, dtype=torch.int32, device=pos.device)
        ws = self.workspace(n)
        self.check(lib().vr_fof3d(self.h, _ptr(pos), n, int(link_d2), _ptr(label), _ptr(ws),
                                  ws.numel(), _stream(stream)))
        return label

    def velden(self, pos, vel, label, params: Params | None = None, f_l=None, stream=None):
        n = pos.shape[0]
        _check(pos, torch.int32, (n, 3))
        _check(vel, torch.float32, (n, 3))
        _check(label, torch.int32, (n,))
        params = params or Params.default()
        if f_l is None:
            f_l = torch.empty(n, dtype=torch.float32, device=pos.device)
        ws = self.workspace(n, params)
        self.check(lib().vr_velden(self.h, _ptr(pos), _ptr(vel), n, _ptr(label),
                                   ctypes.byref(params), _ptr(f_l), _ptr(ws), ws.numel(),
                                   _stream(stream)))
        return f_l

    def outlier_ratio(self, pos, vel, f_l, label, params: Params | None = None, stream=None):
        n = pos.shape[0]
        params = params or Params.default()
        R = torch.empty(n, dtype=torch.float32, device=pos.device)
        ell = torch.empty(n, dtype=torch.float32, device=pos.device)
        hs = torch.empty((n // max(params.nmin, 1) + 1, HALO_COLS), dtype=torch.float64,
                         device=pos.device)
        nh = ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_outlier_ratio(self.h, _ptr(pos), _ptr(vel), _ptr(f_l), n, _ptr(label),
                                          ctypes.byref(params), _ptr(R), _ptr(ell), _ptr(hs),
                                          ctypes.byref(nh), _ptr(ws), ws.numel(), _stream(stream)))
        return R, ell, hs[: nh.value]

    def fof6d(self, pos, vel, ell, label, halo_params, params: Params | None = None,
              label6=None, stream=None):
        n = pos.shape[0]
        params = params or Params.default()
        if label6 is None:
            label6 = torch.empty(n, dtype=torch.int32, device=pos.device)
        halo_params = halo_params.contiguous()
        ws = self.workspace(n, params)
        self.check(lib().vr_fof6d(self.h, _ptr(pos), _ptr(vel), _ptr(ell), n, _ptr(label),
                                  _ptr(halo_params), halo_params.shape[0], ctypes.byref(params),
                                  _ptr(label6), _ptr(ws), ws.numel(), _stream(stream)))
        return label6

    def fof6d_field(self, pos, vel, label, lx: float, alpha_v: float = 1.25,
                    params: Params | None = None, label6=None, halos=None, stream=None):
        """Field 6DFOF inside every 3DFOF halo (vr_fof6d_field). Returns (label6, halo
        table rows [nhalo, HALO_COLS])."""
        n = pos.shape[0]
        params = params or Params.default()
        if label6 is None:
            label6 = torch.empty(n, dtype=torch.int32, device=pos.device)
        if halos is None:
            halos = torch.empty((n // max(params.nmin, 1) + 1, HALO_COLS), dtype=torch.float64,
                                device=pos.device)
        nh = ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_fof6d_field(self.h, _ptr(pos), _ptr(vel), n, _ptr(label), float(lx),
                                        float(alpha_v), ctypes.byref(params), _ptr(label6),
                                        _ptr(halos), ctypes.byref(nh), _ptr(ws), ws.numel(),
                                        _stream(stream)))
        return label6, halos[: nh.value]

    def grow_groups(self, pos, vel, ell, label, halo_params, label6,
                    params: Params | None = None, grow: GrowParams | None = None, stream=None):
        """Two-stage linking (vr_grow_groups): grows the groups of label6 in place."""
        n = pos.shape[0]
        params = params or Params.default()
        grow = grow or GrowParams.default()
        halo_params = halo_params.contiguous()
        ws = self.workspace(n, params)
        self.check(lib().vr_grow_groups(self.h, _ptr(pos), _ptr(vel), _ptr(ell), n, _ptr(label),
                                        _ptr(halo_params), halo_params.shape[0],
                                        ctypes.byref(params), ctypes.byref(grow), _ptr(label6),
                                        _ptr(ws), ws.numel(), _stream(stream)))
        return label6

    def core_search(self, pos, vel, label, label6, lx: float, alpha_v: float = 1.25,
                    params: Params | None = None, cores: CoreParams | None = None, out=None,
                    stream=None):
        """Core search (vr_core_search). label6 may be None. Returns a dict with core,
        level, ncores, halos (rows) and nhalo."""
        n = pos.shape[0]
        params = params or Params.default()
        cores = cores or CoreParams.default()
        if out is None:
            dev = pos.device
            out = dict(core=torch.empty(n, dtype=torch.int32, device=dev),
                       level=torch.empty(n, dtype=torch.int32, device=dev),
                       halos=torch.empty((n // max(params.nmin, 1) + 1, HALO_COLS),
                                         dtype=torch.float64, device=dev))
        nc, nh = ctypes.c_int64(), ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_core_search(self.h, _ptr(pos), _ptr(vel), n, _ptr(label),
                                        _ptr(label6) if label6 is not None else None, float(lx),
                                        float(alpha_v), ctypes.byref(params), ctypes.byref(cores),
                                        _ptr(out["core"]), _ptr(out["level"]), ctypes.byref(nc),
                                        _ptr(out["halos"]), ctypes.byref(nh), _ptr(ws), ws.numel(),
                                        _stream(stream)))
        out["ncores"], out["nhalo"] = nc.value, nh.value
        return out

    def core_grow(self, pos, vel, label, label6, lx: float, alpha_v: float = 1.25,
                  params: Params | None = None, cores: CoreParams | None = None,
                  grow: CoreGrowParams | None = None, out=None, stream=None):
        """Core search, core cleaning and core growth (vr_core_grow). label6 may be None.
        Returns a dict with core, level, grown, nkept, halos (rows) and nhalo."""
        n = pos.shape[0]
        params = params or Params.default()
        cores = cores or CoreParams.default()
        grow = grow or CoreGrowParams.default()
        if out is None:
            dev = pos.device
            out = dict(core=torch.empty(n, dtype=torch.int32, device=dev),
                       level=torch.empty(n, dtype=torch.int32, device=dev),
                       grown=torch.empty(n, dtype=torch.int32, device=dev),
                       halos=torch.empty((n // max(params.nmin, 1) + 1, HALO_COLS),
                                         dtype=torch.float64, device=dev))
        nk, nh = ctypes.c_int64(), ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_core_grow(self.h, _ptr(pos), _ptr(vel), n, _ptr(label),
                                      _ptr(label6) if label6 is not None else None, float(lx),
                                      float(alpha_v), ctypes.byref(params), ctypes.byref(cores),
                                      ctypes.byref(grow), _ptr(out["core"]), _ptr(out["level"]),
                                      _ptr(out["grown"]), ctypes.byref(nk), _ptr(out["halos"]),
                                      ctypes.byref(nh), _ptr(ws), ws.numel(), _stream(stream)))
        out["nkept"], out["nhalo"] = nk.value, nh.value
        return out

    def clean_groups(self, ell, label6, params: Params | None = None, beta: float = 1.0,
                     stream=None):
        """Significance cleaning of the groups in label6, in place (vr_clean_groups).
        Returns the number of groups kept."""
        n = label6.shape[0]
        params = params or Params.default()
        ng = ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_clean_groups(self.h, _ptr(ell), n, ctypes.byref(params), float(beta),
                                         _ptr(label6), ctypes.byref(ng), _ptr(ws), ws.numel(),
                                         _stream(stream)))
        return ng.value

    def find_substructure(self, pos, vel, label, lx_sub: float, alpha_lv: float = 1.0,
                          params: Params | None = None, batched: int = 1, out=None, stream=None):
        n = pos.shape[0]
        params = params or Params.default()
        if out is None:
            out = alloc_outputs(n, params, pos.device)
        nh = ctypes.c_int64()
        ws = self.workspace(n, params)
        self.check(lib().vr_find_substructure(
            self.h, _ptr(pos), _ptr(vel), n, _ptr(label), float(lx_sub), float(alpha_lv),
            ctypes.byref(params), int(batched), _ptr(out["f_l"]), _ptr(out["R"]), _ptr(out["ell"]),
            _ptr(out["label6"]), _ptr(out["halos"]), ctypes.byref(nh), _ptr(ws), ws.numel(),
            _stream(stream)))
        out["nhalo"] = nh.value
        return out


def alloc_outputs(n, params, device):
    return dict(
        f_l=torch.empty(n, dtype=torch.float32, device=device),
        R=torch.empty(n, dtype=torch.float32, device=device),
        ell=torch.empty(n, dtype=torch.float32, device=device),
        label6=torch.empty(n, dtype=torch.int32, device=device),
        halos=torch.empty((n // max(params.nmin, 1) + 1, HALO_COLS), dtype=torch.float64,
                          device=device),
    )


def _check(t, dtype, shape):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise TypeError(f"expected contiguous {dtype} of shape {shape}, got {t.dtype} {tuple(t.shape)}")


def theta_op_default() -> float:
    return 0.1 * math.pi
