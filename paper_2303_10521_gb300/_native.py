"""ctypes binding of libemrt.so (argument marshalling only).

The structures mirror ``include/emrt.h`` field by field.  Loading fails
loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemrt.so")

MAX_DEPTH = 4
PATH_WORDS = 8
NO_FACE = 0xFFFFFFFF
PATH_VALID = 0x100
PATH_MARGINAL = 0x200
TRACE_KEEP_REJECTED = 0x1
TRACE_SORT_RAYS = 0x2
TRACE_WIDE_BVH = 0x4
TRACE_STATIC_CACHE = 0x8
TRACE_BREADTH_FIRST = 0x10
TRACE_REVALIDATE_FIRST = 0x20
REVALIDATE_KEEP = 0x1
NOALLOC_MAX_PATHS = 65536
BATCH_AUTOTUNE = 0x1
BATCH_BREADTH_FIRST = 0x2

vp, u32, u64, dbl = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double


class SceneDesc(C.Structure):
    _fields_ = [("n_static_faces", u32), ("face_off", vp), ("face_xyz", vp),
                ("face_mat", vp), ("n_tris", u32), ("tri_xyz", vp), ("tri_face", vp),
                ("n_vehicles", u32), ("veh_half", vp), ("veh_mat", u32),
                ("max_rx", u32), ("max_tx", u32), ("rebuild_every", u32)]


class TraceParams(C.Structure):
    _fields_ = [("max_depth", u32), ("n_rays", u64), ("ray_offset", u64),
                ("ray_stride", u64), ("ray_count", u64), ("flags", u32)]


class PathsC(C.Structure):
    _fields_ = [("rec", vp), ("capacity", u32), ("count", vp)]


class Materials(C.Structure):
    _fields_ = [("n_mat", u32), ("eps_r", vp), ("sigma", vp), ("gamma", vp),
                ("const_gamma", u32)]


class ChannelOut(C.Structure):
    _fields_ = [("path_out", vp), ("pair_out", vp), ("rx_out", vp)]


class Stats(C.Structure):
    _fields_ = [("segments", u64 * (MAX_DEPTH + 1)), ("candidates", u64),
                ("unique_candidates", u64), ("accepted", u64), ("occlusion_rays", u64),
                ("node_visits", u64), ("tri_tests", u64), ("dyn_node_visits", u64),
                ("box_tests", u64), ("rx_node_visits", u64), ("rx_tests", u64),
                ("error_bits", u32), ("required_candidates", u32), ("required_paths", u32),
                ("pad", u32), ("traverse_ms", C.c_float), ("dedup_ms", C.c_float),
                ("accept_ms", C.c_float), ("trace_ms", C.c_float), ("bounce_ms", C.c_float),
                ("pad2", u32), ("static_reused", u64), ("deferred", u64)]


STATUS = {0: "EMRT_OK", 1: "EMRT_ERR_INVALID_ARG", 2: "EMRT_ERR_OOM", 3: "EMRT_ERR_CUDA",
          4: "EMRT_ERR_CAPACITY", 5: "EMRT_ERR_TIMEOUT", 6: "EMRT_ERR_STATE",
          7: "EMRT_ERR_DEVICE"}

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "emrt_scene_create": (C.c_int, [C.POINTER(SceneDesc), vp, C.POINTER(vp)]),
    "emrt_scene_destroy": (None, [vp]),
    "emrt_scene_update_dynamic": (C.c_int, [vp, vp, vp, vp, vp, u32, vp, vp, u32, vp]),
    "emrt_trace": (C.c_int, [vp, C.POINTER(TraceParams), C.POINTER(PathsC), vp]),
    "emrt_trace_backward": (C.c_int, [vp, C.POINTER(TraceParams), vp, C.c_uint32,
                                      C.POINTER(PathsC), vp]),
    "emrt_revalidate": (C.c_int, [vp, C.POINTER(PathsC), u32, vp]),
    "emrt_revalidate_cache": (C.c_int, [vp, C.POINTER(PathsC), vp, vp]),
    "emrt_trace_batched": (C.c_int, [C.POINTER(vp), u32, C.POINTER(TraceParams),
                                     C.POINTER(PathsC), vp]),
    "emrt_cache_merge": (C.c_int, [vp, C.POINTER(PathsC), C.POINTER(PathsC), vp]),
    "emrt_rediscover": (C.c_int, [vp, C.POINTER(TraceParams), C.POINTER(PathsC), vp]),
    "emrt_channel": (C.c_int, [vp, C.POINTER(PathsC), C.POINTER(Materials), dbl, dbl,
                               C.POINTER(ChannelOut), vp]),
    "emrt_channel_multi": (C.c_int, [vp, C.POINTER(PathsC), C.POINTER(Materials),
                                     C.POINTER(dbl), C.c_uint32, dbl, C.POINTER(ChannelOut),
                                     vp]),
    "emrt_channel_backward": (C.c_int, [vp, C.POINTER(PathsC), C.POINTER(Materials), dbl, vp,
                                        vp, vp, vp, vp]),
    "emrt_channel_backward_noalloc": (C.c_int, [vp, C.POINTER(PathsC), C.POINTER(Materials),
                                                dbl, vp, vp, vp, vp, vp]),
    "emrt_sync": (C.c_int, [vp, vp, C.POINTER(Stats)]),
    "emrt_channel_correlation": (C.c_int, [vp, u32, u32, u32, vp, vp]),
    "emrt_coherence_time": (C.c_int, [vp, dbl, dbl, vp, vp]),
    "emrt_refresh_schedule": (C.c_int, [vp, vp, vp, dbl, dbl, dbl, C.c_float, u32, vp, vp,
                                        vp]),
    "emrt_batch_create": (C.c_int, [C.POINTER(vp), u32, C.POINTER(TraceParams),
                                    C.POINTER(PathsC), u32, vp, C.POINTER(vp)]),
    "emrt_batch_trace": (C.c_int, [vp, vp]),
    "emrt_batch_sync": (C.c_int, [vp, vp, C.POINTER(Stats)]),
    "emrt_batch_config": (C.c_int, [vp, C.c_char_p, u32]),
    "emrt_batch_destroy": (None, [vp]),
    "emrt_status_string": (C.c_char_p, [C.c_int]),
    "emrt_kernel_launches": (u64, []),
    "emrt_selftest_grid_barrier": (C.c_int, [u32, C.POINTER(u32), C.POINTER(u32)]),
}

_lib = None


class EmrtError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{where}: {self.name}")


def load():
    """Load libemrt.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libemrt.so not found at {LIB_PATH}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(nvcc for sm_103a is required; there is no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code, where):
    if code != 0:
        raise EmrtError(code, where)
