"""GB300 (sm_103a) VELOCIraptor substructure hot path: CUDA library + thin binding.

The compute lives in libvr.so (include/vr.h); ``vr`` wraps it for torch device tensors.
"""
from . import _build  # noqa: F401
from .vr import Context, CoreGrowParams, CoreParams, GrowParams, Params, VrError, lib  # noqa: F401
