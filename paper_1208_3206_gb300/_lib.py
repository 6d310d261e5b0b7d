"""ctypes view of include/lt.h. Argument marshalling only: every step of the
projection runs in liblt.so's CUDA kernels."""
from __future__ import annotations

import ctypes as C
import os

from . import _build

_lib = None


class LtCamera(C.Structure):
    _fields_ = [
        ("type", C.c_int),
        ("eye", C.c_double * 3),
        ("fwd", C.c_double * 3),
        ("up", C.c_double * 3),
        ("fov_y_deg", C.c_double),
        ("lo", C.c_double * 2),
        ("hi", C.c_double * 2),
        ("W", C.c_int),
        ("H", C.c_int),
        ("wrap", C.c_int),
        ("near_radius", C.c_double),
    ]


class LtConfig(C.Structure):
    _fields_ = [
        ("tile", C.c_int),
        ("raster_threads", C.c_int),
        ("ctas_per_sm", C.c_int),
        ("frac_bits", C.c_int),
    ]


class LtStats(C.Structure):
    _fields_ = [
        ("tets", C.c_longlong),
        ("entries", C.c_longlong),
        ("capacity", C.c_longlong),
        ("degenerate", C.c_longlong),
        ("fp64_fallbacks", C.c_longlong),
        ("inverted", C.c_longlong),
        ("nonfinite", C.c_longlong),
        ("behind_eye", C.c_longlong),
        ("range_overflow", C.c_longlong),
        ("exact_fragments", C.c_longlong),
        ("queue_overflow", C.c_longlong),
        ("resample_intervals", C.c_longlong),
        ("resample_pieces", C.c_longlong),
        ("area_pairs", C.c_longlong),
        ("area_fp64_pairs", C.c_longlong),
        ("exact_tile_max", C.c_longlong),
        ("n_frames", C.c_int),
        ("tile", C.c_int),
        ("graph_kernels", C.c_int),
        ("pad", C.c_int),
    ]


STATUS = {
    0: "LT_OK",
    1: "LT_ERR_ARG",
    2: "LT_ERR_CUDA",
    3: "LT_ERR_CAPACITY",
    4: "LT_ERR_NONFINITE",
    5: "LT_ERR_BEHIND_EYE",
    6: "LT_ERR_RANGE",
    7: "LT_ERR_STATE",
    8: "LT_ERR_NOMEM",
    9: "LT_ERR_BOUNDS",
}

# every symbol declared in include/lt.h
EXPORTS = [
    "lt_create", "lt_destroy", "lt_set_config", "lt_get_config", "lt_build_tets", "lt_project_bin",
    "lt_render_tiles", "lt_render_atomic", "lt_count_fragments", "lt_render_backward", "lt_graph_build",
    "lt_graph_launch", "lt_autotune", "lt_sync", "lt_get_stats", "lt_status_str", "lt_frame_mass_static",
    "lt_resample", "lt_slice", "lt_render_centroids", "lt_render_area", "lt_render_hybrid",
]


class LtError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        self.name = STATUS.get(code, str(code))
        msg = _lib.lt_status_str(code).decode() if _lib is not None else self.name
        super().__init__(f"{fn}: {self.name} ({msg})")


def lib_path() -> str:
    return _build.LIB


def build_flags() -> str:
    """Extra compiler flags liblt.so was built with ("" for the default build)."""
    try:
        with open(_build.STAMP) as fh:
            return fh.read().strip()
    except OSError:
        return ""


def load(build_if_missing: bool = False):
    """Load liblt.so. Raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(
                f"liblt.so not found at {path}: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    flags = build_flags()
    if flags and os.environ.get("LT_ALLOW_DEBUG_BUILD") != "1":
        # a debugging build (bounds checks, ptxas report) must not be timed
        # or tested by mistake: rebuild the default one
        _build.build(force=True)
    lib = C.CDLL(path)
    vp, ip, fp, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_double)
    cam_p = C.POINTER(LtCamera)
    cfg_p = C.POINTER(LtConfig)
    sigs = {
        "lt_create": ([C.POINTER(vp), cfg_p], C.c_int),
        "lt_destroy": ([vp], None),
        "lt_set_config": ([vp, cfg_p], C.c_int),
        "lt_get_config": ([vp, cfg_p], C.c_int),
        "lt_build_tets": ([vp, vp, C.c_int, C.c_int, C.c_float, C.c_double, C.c_int, vp, vp], C.c_int),
        "lt_project_bin": ([vp, cam_p, C.c_int, ip, vp], C.c_int),
        "lt_render_tiles": ([vp, vp, vp, vp], C.c_int),
        "lt_render_atomic": ([vp, cam_p, C.c_int, ip, vp, vp], C.c_int),
        "lt_count_fragments": ([vp, C.POINTER(C.c_longlong), vp], C.c_int),
        "lt_render_backward": ([vp, vp, vp, vp], C.c_int),
        "lt_graph_build": ([vp, cam_p, C.c_int, ip, vp, vp, vp], C.c_int),
        "lt_graph_launch": ([vp, vp], C.c_int),
        "lt_autotune": ([vp, cam_p, C.c_int, ip, vp, C.c_int, cfg_p, vp], C.c_int),
        "lt_sync": ([vp, vp], C.c_int),
        "lt_get_stats": ([vp, C.POINTER(LtStats)], C.c_int),
        "lt_status_str": ([C.c_int], C.c_char_p),
        "lt_frame_mass_static": ([vp, C.c_int, C.c_int, C.c_int, C.c_double, vp, vp], C.c_int),
        "lt_resample": ([vp, C.c_int, C.c_int, C.c_int, vp, vp], C.c_int),
        "lt_slice": ([vp, C.c_int, C.c_int, C.c_int, C.c_double, vp, vp], C.c_int),
        "lt_render_centroids": ([vp, cam_p, C.c_int, vp, vp], C.c_int),
        "lt_render_area": ([vp, cam_p, C.c_int, vp, vp], C.c_int),
        "lt_render_hybrid": ([vp, cam_p, C.c_int, C.c_double, vp, vp], C.c_int),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(fn: str, code: int) -> None:
    if code != 0:
        raise LtError(fn, code)
