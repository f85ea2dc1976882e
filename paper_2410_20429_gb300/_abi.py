"""ctypes binding of libmars (include/mars.h).  Argument marshalling only: every
step of the path tracer runs in the CUDA library; there is no CPU fallback.
The entry points keep the C names."""
from __future__ import annotations

import ctypes as ct
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmars.so")

MARS_OK, MARS_ERR_INVALID_ARG, MARS_ERR_OOM, MARS_ERR_CUDA, MARS_ERR_TIMEOUT, MARS_ERR_BUSY, MARS_ERR_NOT_FOUND = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "BUSY", 6: "NOT_FOUND"}
MARS_TECH_BSDF, MARS_TECH_NEE, MARS_TECH_GUIDED, MARS_TECH_LIGHT = 1, 2, 4, 8
MARS_LIGHT_MAX = 5
MARS_MODE_WARMUP, MARS_MODE_MARS, MARS_MODE_FIXED = 0, 1, 2
MARS_WEIGHTS_AWARE, MARS_WEIGHTS_UNAWARE = 0, 1
MARS_JOB_QUEUED, MARS_JOB_RUNNING, MARS_JOB_DONE, MARS_JOB_FAILED = range(4)
MARS_CACHE_FP32_STATISTICS = 1
MARS_CACHE_OCTREE = 2
MARS_CACHE_NO_GRAPHS = 4
MARS_CACHE_ONE_LANE = 8
MARS_BVH_SAH = 0
MARS_MAX_DROP_BRIGHTEST = 16
MARS_INJECT_ALLOC, MARS_INJECT_LAUNCH = 0, 1
MARS_BVH_LBVH = 1
NUM_SLOTS, NUM_STATS, GUIDE_BINS, MAX_DEPTH = 3, 8, 256, 16


class MarsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where} failed with MARS_ERR_{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mars_scene_desc(ct.Structure):
    _fields_ = [
        ("n_quads", ct.c_int32), ("n_spheres", ct.c_int32), ("n_tris", ct.c_int32), ("n_materials", ct.c_int32),
        ("quads", ct.POINTER(ct.c_double)), ("quad_mat", ct.POINTER(ct.c_int32)),
        ("spheres", ct.POINTER(ct.c_double)), ("sphere_mat", ct.POINTER(ct.c_int32)),
        ("tris", ct.POINTER(ct.c_double)), ("tri_mat", ct.POINTER(ct.c_int32)),
        ("materials", ct.POINTER(ct.c_double)),
        ("camera", ct.c_double * 10),
        ("width", ct.c_int32), ("height", ct.c_int32), ("bvh", ct.c_int32), ("reserved", ct.c_int32),
    ]


class mars_cache_desc(ct.Structure):
    _fields_ = [("grid_n", ct.c_int32), ("techniques", ct.c_int32), ("max_depth", ct.c_int32),
                ("flags", ct.c_int32), ("arena_capacity", ct.c_uint64), ("max_leaves", ct.c_int32),
                ("split_samples", ct.c_float)]


class mars_iter_params(ct.Structure):
    _fields_ = [
        ("seed", ct.c_uint32), ("job", ct.c_uint32), ("iteration", ct.c_uint32),
        ("mode", ct.c_int32), ("weights", ct.c_int32),
        ("clamp_lo", ct.c_float), ("clamp_hi", ct.c_float), ("outlier", ct.c_float),
        ("collect", ct.c_int32), ("image_on_host", ct.c_int32), ("update_estimate", ct.c_int32),
        ("profile", ct.c_int32), ("max_multiplicity", ct.c_float),
        ("vi_drop_brightest", ct.c_int32), ("combine", ct.c_int32),
        ("px_begin", ct.c_int32), ("px_end", ct.c_int32),
    ]


class mars_iter_stats(ct.Structure):
    _fields_ = [
        ("VI", ct.c_double), ("CI", ct.c_double), ("rays", ct.c_uint64), ("vertices", ct.c_uint64),
        ("estimator_vertices", ct.c_uint64), ("mean_beta", ct.c_double * 3), ("tiles", ct.c_uint32),
        ("retries", ct.c_uint32), ("arena_demand", ct.c_uint64), ("launches", ct.c_uint32),
        ("wave_launches", ct.c_uint32), ("trace_ms", ct.c_double), ("shade_ms", ct.c_double),
        ("shadow_ms", ct.c_double), ("reverse_ms", ct.c_double), ("image_ms", ct.c_double),
        ("wave_entries", ct.c_uint64), ("shadow_entries", ct.c_uint64), ("shadow_traced", ct.c_uint64),
        ("wave_ms", (ct.c_float * 16) * 4), ("wave_rays", ct.c_uint64 * 16),
        ("trace_work", (ct.c_uint64 * 4) * 2), ("check_flags", ct.c_uint32), ("reserved", ct.c_uint32),
        ("light_rays", ct.c_uint64), ("connection_rays", ct.c_uint64), ("light_samples", ct.c_uint64),
        ("light_ms", ct.c_double),
    ]


class mars_cache_state(ct.Structure):
    _fields_ = [
        ("q_rr", ct.POINTER(ct.c_float)), ("q_s", ct.POINTER(ct.c_float)), ("valid", ct.POINTER(ct.c_uint8)),
        ("stats", ct.POINTER(ct.c_double)), ("guide_hist", ct.POINTER(ct.c_float)),
        ("guide_cdf", ct.POINTER(ct.c_float)), ("pixel_estimate", ct.POINTER(ct.c_float)),
        ("run_sum", ct.POINTER(ct.c_float)), ("n_iterations", ct.c_int32), ("has_estimate", ct.c_int32),
        ("VI", ct.c_double), ("CI", ct.c_double),
        ("oct_nodes", ct.POINTER(ct.c_int32)), ("oct_leaf_level", ct.POINTER(ct.c_int32)),
        ("oct_n_nodes", ct.c_int32), ("oct_n_leaves", ct.c_int32),
        ("pixel_rays", ct.POINTER(ct.c_float)), ("image_iterations", ct.c_int32),
    ]


class mars_cache_info(ct.Structure):
    _fields_ = [
        ("n_cells", ct.c_int64), ("n_pixels", ct.c_int64), ("grid_n", ct.c_int32), ("techniques", ct.c_int32),
        ("max_depth", ct.c_int32), ("n_prims", ct.c_int32), ("arena_capacity", ct.c_uint64),
        ("device_bytes", ct.c_uint64), ("device", ct.c_int32), ("n_lights", ct.c_int32),
        ("oct_n_nodes", ct.c_int32), ("oct_n_leaves", ct.c_int32), ("oct_cap_nodes", ct.c_int32),
        ("graph_captures", ct.c_int32),
    ]


class mars_launch_config(ct.Structure):
    _fields_ = [("threads", ct.c_int32 * 4), ("blocks_per_sm", ct.c_int32 * 4), ("max_registers", ct.c_int32 * 4),
                ("lanes", ct.c_int32), ("lane_min_pixels", ct.c_int32)]


class mars_job_desc(ct.Structure):
    _fields_ = [("scene", ct.POINTER(mars_scene_desc)), ("cache", mars_cache_desc), ("seed", ct.c_uint32),
                ("iterations", ct.c_int32), ("warmup", ct.c_int32), ("key", ct.c_uint32),
                ("timeout_s", ct.c_double)]


class mars_job_status(ct.Structure):
    _fields_ = [("state", ct.c_int32), ("iterations_done", ct.c_int32), ("error", ct.c_int32),
                ("reserved", ct.c_int32), ("submit_s", ct.c_double), ("start_s", ct.c_double),
                ("end_s", ct.c_double), ("iter_ms_p50", ct.c_double), ("iter_ms_p99", ct.c_double),
                ("device_bytes", ct.c_uint64), ("vertices", ct.c_uint64)]


_VP = ct.c_void_p
# name -> (argtypes, restype); every entry point declared in include/mars.h
SIGNATURES = {
    "mars_scene_create": ([ct.POINTER(mars_scene_desc), _VP, ct.POINTER(_VP)], ct.c_int),
    "mars_scene_destroy": ([_VP], ct.c_int),
    "mars_cache_create": ([_VP, ct.POINTER(mars_cache_desc), _VP, ct.POINTER(_VP)], ct.c_int),
    "mars_cache_destroy": ([_VP], ct.c_int),
    "mars_cache_info_get": ([_VP, ct.POINTER(mars_cache_info)], ct.c_int),
    "mars_render_iteration": ([_VP, ct.POINTER(mars_iter_params), _VP, ct.POINTER(mars_iter_stats), _VP], ct.c_int),
    "mars_update_counts": ([_VP, _VP], ct.c_int),
    "mars_cache_combined_image": ([_VP, _VP, ct.POINTER(ct.c_double), _VP], ct.c_int),
    "mars_debug_inject_failure": ([ct.c_int32, ct.c_int32], ct.c_int),
    "mars_cache_get_state": ([_VP, ct.POINTER(mars_cache_state), _VP], ct.c_int),
    "mars_cache_set_state": ([_VP, ct.POINTER(mars_cache_state), _VP], ct.c_int),
    "mars_cache_get_launch": ([_VP, ct.POINTER(mars_launch_config)], ct.c_int),
    "mars_cache_set_launch": ([_VP, ct.POINTER(mars_launch_config)], ct.c_int),
    "mars_cache_autotune": ([_VP, ct.POINTER(mars_iter_params), ct.c_int32, ct.POINTER(mars_launch_config), _VP],
                            ct.c_int),
    "mars_server_create": ([ct.c_uint64, ct.c_int32, ct.POINTER(_VP)], ct.c_int),
    "mars_server_destroy": ([_VP], ct.c_int),
    "mars_submit": ([_VP, ct.POINTER(mars_job_desc), ct.POINTER(ct.c_uint64)], ct.c_int),
    "mars_poll": ([_VP, ct.c_uint64, ct.POINTER(mars_job_status), _VP], ct.c_int),
    "mars_job_latencies": ([_VP, ct.c_uint64, _VP, ct.c_int32, ct.POINTER(ct.c_int32)], ct.c_int),
    "mars_image_stats_static": ([_VP, _VP, _VP, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_float, ct.c_double, _VP,
                                 _VP], ct.c_int),
    "mars_last_error_string": ([], ct.c_char_p),
    "mars_version": ([], ct.c_char_p),
    "mars_training_step_ends": ([ct.c_int32, ct.c_int32, ct.c_int32], ct.c_int32),
}

_lib = None


def load(path: str | None = None):
    """Load libmars.so (built in-tree by ``__graft_entry__.build()``).  Raises if
    the library is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libmars.so not found at {p}; build it with paper_2410_20429_gb300.build.build()")
    L = ct.CDLL(p)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != MARS_OK:
        msg = load().mars_last_error_string()
        raise MarsError(status, where, msg.decode() if msg else "")
