"""ctypes declarations of the C ABI in ``include/rtsdf.h`` (marshalling only).

The shared library is built in-tree (``build.py``) and is required: there is
no CPU fallback.  Importing this module does not touch the GPU; the first
function call loads ``librtsdf.so`` and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librtsdf.so")

c_f, c_i32, c_i64, c_u64, c_vp, c_sz = (ctypes.c_float, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_size_t)
c_int = ctypes.c_int
status_t = ctypes.c_int


class Config(ctypes.Structure):
    _fields_ = [("bmin", c_f * 3), ("extent", c_f), ("coarse_n", c_i32), ("beta_vox", c_f),
                ("alpha", c_f), ("seed", c_u64), ("stream", c_vp)]


class Grids(ctypes.Structure):
    _fields_ = [("coarse_n", c_i32), ("fine_n", c_i32), ("seeds", c_vp), ("coarse", c_vp), ("fine", c_vp),
                ("accum", c_vp), ("counts", c_vp), ("masked", c_vp)]


STAGES = ("voxelize", "jfa", "mask", "trace", "bvh", "shadow", "shadow_bwd", "motion")


class Stats(ctypes.Structure):
    _fields_ = [("launches", c_i64), ("n_masked_texels", c_i64), ("jfa_passes", c_i32), ("bvh_depth", c_i32),
                ("stage_ms", c_f * len(STAGES)), ("stage_calls", c_i32 * len(STAGES)), ("rays", c_i64),
                ("node_visits", c_i64), ("tri_tests", c_i64), ("lane_slots", c_i64), ("leaf_slots", c_i64)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", c_i32), ("refill_min", c_i32), ("ray_chunk", c_i32), ("use_graph", c_i32),
                ("barrier_spins", c_i32), ("leaf_min", c_i32), ("split_trace", c_i32)]


class Tuning(ctypes.Structure):
    _fields_ = [("jfa_tile", c_i32), ("trace_blocks_per_sm", c_i32), ("refill_min", c_i32), ("ray_chunk", c_i32),
                ("leaf_min", c_i32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_scenes", c_i32), ("grid", c_i32), ("graph", c_i32), ("frames", c_i64), ("launches", c_i64),
                ("last_frame_ms", c_f), ("stage_ms", c_f * 7)]


F3 = c_f * 3
ctx_t = c_vp

# name -> (restype, argtypes); the order follows include/rtsdf.h
SIGNATURES = {
    "rtsdf_create": (status_t, [ctypes.POINTER(Config), ctypes.POINTER(c_vp)]),
    "rtsdf_destroy": (status_t, [ctx_t]),
    "rtsdf_set_stream": (status_t, [ctx_t, c_vp]),
    "rtsdf_upload_mesh": (status_t, [ctx_t, c_vp, c_i64, c_vp, c_i64, c_int]),
    "rtsdf_set_objects": (status_t, [ctx_t, c_vp, c_i32, c_int]),
    "rtsdf_move_objects": (status_t, [ctx_t, c_vp, c_int]),
    "rtsdf_transform_objects": (status_t, [ctx_t, c_vp, c_int]),
    "rtsdf_set_reset": (status_t, [ctx_t, c_i32]),
    "rtsdf_debug_fail_allocation": (None, [c_i64]),
    "rtsdf_debug_bvh_cycle": (status_t, [ctx_t]),
    "rtsdf_debug_texture_fetch": (None, [c_i32]),
    "rtsdf_get_reset": (status_t, [ctx_t, ctypes.POINTER(c_i32)]),
    "rtsdf_build_bvh": (status_t, [ctx_t, c_int]),
    "rtsdf_voxelize": (status_t, [ctx_t]),
    "rtsdf_jfa": (status_t, [ctx_t]),
    "rtsdf_trace": (status_t, [ctx_t, c_f, c_i32, c_i32]),
    "rtsdf_shadow": (status_t, [ctx_t, c_vp, c_vp, c_vp, c_i64, F3, c_f, c_i32, c_f, c_f, c_vp]),
    "rtsdf_shadow_jittered": (status_t, [ctx_t, c_vp, c_vp, c_vp, c_i64, F3, c_f, c_i32, c_f, c_f, c_f, c_i32, c_vp]),
    "rtsdf_taa_resolve": (status_t, [ctx_t, c_vp, c_vp, c_i32, c_i32, c_f]),
    "rtsdf_shadow_fallback": (status_t, [ctx_t, c_vp, c_vp, c_i64, F3, c_f, c_vp, c_vp]),
    "rtsdf_set_sign_mode": (status_t, [ctx_t, c_i32]),
    "rtsdf_get_sign_mode": (status_t, [ctx_t, ctypes.POINTER(c_i32)]),
    "rtsdf_set_bvh_builder": (status_t, [ctx_t, c_i32]),
    "rtsdf_get_bvh_builder": (status_t, [ctx_t, ctypes.POINTER(c_i32)]),
    "rtsdf_get_bvh_topology": (status_t, [ctx_t, c_vp, c_vp, ctypes.POINTER(c_i32)]),
    "rtsdf_shadow_backward": (status_t, [ctx_t, c_vp, c_vp, c_vp, c_i64, F3, c_f, c_i32, c_f, c_f, c_vp, c_vp,
                                         c_vp]),
    "rtsdf_jfa_noalloc": (status_t, [c_vp, c_vp, c_vp, c_i32, c_f, c_f, c_vp]),
    "rtsdf_batch_create": (status_t, [ctypes.POINTER(Config), c_i32, ctypes.POINTER(c_vp)]),
    "rtsdf_batch_destroy": (status_t, [c_vp]),
    "rtsdf_batch_context": (status_t, [c_vp, c_i32, ctypes.POINTER(c_vp)]),
    "rtsdf_batch_frame": (status_t, [c_vp, c_f, c_i32, c_i32]),
    "rtsdf_batch_sync": (status_t, [c_vp]),
    "rtsdf_batch_set_tuning": (status_t, [c_vp, ctypes.POINTER(BatchTuning)]),
    "rtsdf_batch_get_tuning": (status_t, [c_vp, ctypes.POINTER(BatchTuning)]),
    "rtsdf_batch_stats": (status_t, [c_vp, ctypes.POINTER(BatchInfo)]),
    "rtsdf_set_tuning": (status_t, [ctx_t, ctypes.POINTER(Tuning)]),
    "rtsdf_get_tuning": (status_t, [ctx_t, ctypes.POINTER(Tuning)]),
    "rtsdf_autotune": (status_t, [ctx_t, c_f, c_i32, c_i32, c_i32, ctypes.POINTER(Tuning)]),
    "rtsdf_batch_autotune": (status_t, [c_vp, c_f, c_i32, c_i32, c_i32, ctypes.POINTER(BatchTuning)]),
    "rtsdf_get_grids": (status_t, [ctx_t, ctypes.POINTER(Grids)]),
    "rtsdf_get_masked_count": (status_t, [ctx_t, ctypes.POINTER(c_i64)]),
    "rtsdf_get_stats": (status_t, [ctx_t, ctypes.POINTER(Stats)]),
    "rtsdf_set_profiling": (status_t, [ctx_t, c_int]),
    "rtsdf_set_counting": (status_t, [ctx_t, c_int]),
    "rtsdf_state_size": (status_t, [ctx_t, ctypes.POINTER(c_sz)]),
    "rtsdf_save_state": (status_t, [ctx_t, c_vp, c_sz]),
    "rtsdf_load_state": (status_t, [ctx_t, c_vp, c_sz]),
    "rtsdf_sync": (status_t, [ctx_t]),
    "rtsdf_status_str": (ctypes.c_char_p, [c_int]),
    "rtsdf_version": (ctypes.c_char_p, []),
}

STATUS_NAMES = {0: "RTSDF_OK", 1: "RTSDF_E_ARG", 2: "RTSDF_E_STATE", 3: "RTSDF_E_OOM", 4: "RTSDF_E_CUDA",
                5: "RTSDF_E_MESH", 6: "RTSDF_E_OVERFLOW", 7: "RTSDF_E_TIMEOUT"}

_lib = None
_lock = threading.Lock()


class RtsdfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = STATUS_NAMES.get(code, str(code))
        msg = lib().rtsdf_status_str(code).decode()
        super().__init__(f"{where}: {self.name} ({msg})")


def lib() -> ctypes.CDLL:
    """The loaded librtsdf.so; raises when it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def check(code: int, where: str) -> None:
    if code != 0:
        raise RtsdfError(code, where)


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args), name)
