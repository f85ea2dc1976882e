"""Python front end of libmars: objects that own a mars_scene / mars_cache and
marshal numpy / torch buffers into the C ABI.  Device memory and streams come
from PyTorch; all rendering work runs in the CUDA library."""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _abi as A


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dp(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


def scene_desc(desc):
    """Build a mars_scene_desc over contiguous copies of the description's arrays;
    returns the struct and the arrays that must stay alive while it is used."""
    keep = [
        np.ascontiguousarray(desc.quads, np.float64).reshape(-1, 9),
        np.ascontiguousarray(desc.quad_mat, np.int32).reshape(-1),
        np.ascontiguousarray(desc.spheres, np.float64).reshape(-1, 4),
        np.ascontiguousarray(desc.sphere_mat, np.int32).reshape(-1),
        np.ascontiguousarray(desc.tris, np.float64).reshape(-1, 9),
        np.ascontiguousarray(desc.tri_mat, np.int32).reshape(-1),
        np.ascontiguousarray(desc.materials, np.float64).reshape(-1, 8),
    ]
    q, qm, s, sm, t, tm, m = keep
    d = A.mars_scene_desc()
    d.n_quads, d.n_spheres, d.n_tris, d.n_materials = len(q), len(s), len(t), len(m)
    d.quads, d.quad_mat = _dp(q, ct.c_double), _dp(qm, ct.c_int32)
    d.spheres, d.sphere_mat = _dp(s, ct.c_double), _dp(sm, ct.c_int32)
    d.tris, d.tri_mat = _dp(t, ct.c_double), _dp(tm, ct.c_int32)
    d.materials = _dp(m, ct.c_double)
    for i in range(10):
        d.camera[i] = float(desc.camera[i])
    d.width, d.height = int(desc.width), int(desc.height)
    d.bvh = int(getattr(desc, "bvh", A.MARS_BVH_SAH))
    return d, keep


class Scene:
    """Device-resident scene (primitives, materials, lights, LBVH).  ``desc`` is
    any object with the numpy fields of a scene description (quads, quad_mat,
    spheres, sphere_mat, tris, tri_mat, materials, camera, width, height)."""

    def __init__(self, desc, stream=None):
        self._lib = A.load()
        self.desc, self._keep = scene_desc(desc)
        self.width, self.height = self.desc.width, self.desc.height
        h = ct.c_void_p()
        A.check(self._lib.mars_scene_create(ct.byref(self.desc), _stream_handle(stream), ct.byref(h)),
                "mars_scene_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mars_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cache:
    """Statistics cache, count fields, guide and image accumulators of one job."""

    def __init__(self, scene: Scene, grid_n: int, techniques: int, max_depth: int, arena_capacity: int = 0,
                 fp32_statistics: bool = False, octree: bool = False, max_leaves: int = 0,
                 split_samples: float = 0.0, graphs: bool = True, lanes: int = 2, stream=None):
        self._lib = A.load()
        self.scene = scene
        flags = ((A.MARS_CACHE_FP32_STATISTICS if fp32_statistics else 0) | (A.MARS_CACHE_OCTREE if octree else 0)
                 | (0 if graphs else A.MARS_CACHE_NO_GRAPHS) | (A.MARS_CACHE_ONE_LANE if lanes == 1 else 0))
        d = A.mars_cache_desc(int(grid_n), int(techniques), int(max_depth), flags, int(arena_capacity),
                              int(max_leaves), float(split_samples))
        h = ct.c_void_p()
        A.check(self._lib.mars_cache_create(scene.handle, ct.byref(d), _stream_handle(stream), ct.byref(h)),
                "mars_cache_create")
        self.handle = h
        self.grid_n, self.techniques, self.max_depth = int(grid_n), int(techniques), int(max_depth)
        self.octree = bool(octree)
        info = self.info()
        self.n_cells = int(info["n_cells"])   # grid_n^3, or the octree's leaf capacity
        self.oct_cap_nodes = int(info["oct_cap_nodes"])
        self.n_pixels = scene.width * scene.height

    def info(self) -> dict:
        i = A.mars_cache_info()
        A.check(self._lib.mars_cache_info_get(self.handle, ct.byref(i)), "mars_cache_info_get")
        return {f: getattr(i, f) for f, _ in A.mars_cache_info._fields_}

    def render_iteration(self, image, *, seed=0, job=0, iteration=0, mode=A.MARS_MODE_WARMUP,
                         weights=A.MARS_WEIGHTS_AWARE, clamp_lo=0.05, clamp_hi=20.0, outlier=50.0, collect=True,
                         update_estimate=True, profile=False, max_multiplicity=0.0, vi_drop_brightest=0,
                         combine=0, px_range=None, stream=None) -> dict:
        """Render one iteration into ``image``: a CUDA float32 tensor with
        height*width*3 elements, or a host numpy float32 array of that size (the
        library then copies the image back).  ``vi_drop_brightest`` and
        ``combine`` select the bidirectional application's image-variance
        rejection and progressive combination (see mars.h).  ``px_range``
        (begin, end) renders only those pixels (a shard of a multi-GPU job)."""
        on_host = isinstance(image, np.ndarray)
        if on_host:
            if image.dtype != np.float32 or not image.flags.c_contiguous or image.size != 3 * self.n_pixels:
                raise ValueError("host image must be a contiguous float32 array of height*width*3")
            ptr = image.ctypes.data
        elif image is None:
            ptr = None
        else:
            if (not image.is_cuda or image.dtype.__str__() != "torch.float32" or not image.is_contiguous()
                    or image.numel() != 3 * self.n_pixels):
                raise ValueError("device image must be a contiguous CUDA float32 tensor of height*width*3")
            ptr = image.data_ptr()
        p = A.mars_iter_params(int(seed), int(job), int(iteration), int(mode), int(weights), float(clamp_lo),
                               float(clamp_hi), float(outlier), int(bool(collect)), int(on_host),
                               int(bool(update_estimate)), int(bool(profile)), float(max_multiplicity),
                               int(vi_drop_brightest), int(combine),
                               *((0, 0) if px_range is None else (int(px_range[0]), int(px_range[1]))))
        st = A.mars_iter_stats()
        A.check(self._lib.mars_render_iteration(self.handle, ct.byref(p), ptr, ct.byref(st), _stream_handle(stream)),
                "mars_render_iteration")
        return {"VI": st.VI, "CI": st.CI, "rays": st.rays, "vertices": st.vertices,
                "estimator_vertices": st.estimator_vertices, "mean_beta": list(st.mean_beta),
                "tiles": st.tiles, "retries": st.retries, "arena_demand": st.arena_demand,
                "launches": st.launches, "wave_launches": st.wave_launches, "trace_ms": st.trace_ms,
                "shade_ms": st.shade_ms, "shadow_ms": st.shadow_ms, "reverse_ms": st.reverse_ms,
                "image_ms": st.image_ms, "wave_entries": st.wave_entries, "shadow_entries": st.shadow_entries,
                "shadow_traced": st.shadow_traced,
                "wave_ms": [[st.wave_ms[k][d] for d in range(self.max_depth)] for k in range(4)],
                "wave_rays": [st.wave_rays[d] for d in range(self.max_depth)],
                "trace_work": [[st.trace_work[k][q] for q in range(4)] for k in range(2)],
                "check_flags": st.check_flags, "light_rays": st.light_rays,
                "connection_rays": st.connection_rays, "light_samples": st.light_samples,
                "light_ms": st.light_ms}

    def combined_image(self, stream=None):
        """(image [height][width][3] float32, weight sum) of the progressive
        inverse-variance combination."""
        img = np.zeros((self.scene.height, self.scene.width, 3), np.float32)
        w = ct.c_double(0.0)
        A.check(self._lib.mars_cache_combined_image(self.handle, img.ctypes.data, ct.byref(w), _stream_handle(stream)),
                "mars_cache_combined_image")
        return img, w.value

    def get_launch(self) -> dict:
        """Launch shape of the wave kernels (trace, shade, shadow, reverse)."""
        cfg = A.mars_launch_config()
        A.check(self._lib.mars_cache_get_launch(self.handle, ct.byref(cfg)), "mars_cache_get_launch")
        return {"threads": list(cfg.threads), "blocks_per_sm": list(cfg.blocks_per_sm),
                "max_registers": list(cfg.max_registers), "lanes": cfg.lanes, "lane_min_pixels": cfg.lane_min_pixels}

    def set_launch(self, threads, blocks_per_sm, max_registers=(0, 0, 0, 0), lanes=0, lane_min_pixels=0) -> None:
        """Launch shape of the wave kernels; ``lanes`` / ``lane_min_pixels`` (0:
        unchanged) set how many concurrent tile lanes an iteration may use and
        the smallest image split over them."""
        cfg = A.mars_launch_config()
        for k in range(4):
            cfg.threads[k] = int(threads[k])
            cfg.blocks_per_sm[k] = int(blocks_per_sm[k])
            cfg.max_registers[k] = int(max_registers[k])
        cfg.lanes = int(lanes)
        cfg.lane_min_pixels = int(lane_min_pixels)
        A.check(self._lib.mars_cache_set_launch(self.handle, ct.byref(cfg)), "mars_cache_set_launch")

    def autotune(self, *, seed=0, job=0, iteration=0, mode=A.MARS_MODE_WARMUP, weights=A.MARS_WEIGHTS_AWARE,
                 clamp_lo=0.05, clamp_hi=20.0, outlier=50.0, repeats=2, max_multiplicity=0.0, stream=None) -> dict:
        """Pick the fastest launch shape of every wave kernel on this iteration,
        then one or all tile lanes by whole-iteration time (rendered without
        statistics, so the learned state is unchanged)."""
        p = A.mars_iter_params(int(seed), int(job), int(iteration), int(mode), int(weights), float(clamp_lo),
                               float(clamp_hi), float(outlier), 0, 0, 0, 1, float(max_multiplicity))
        cfg = A.mars_launch_config()
        A.check(self._lib.mars_cache_autotune(self.handle, ct.byref(p), int(repeats), ct.byref(cfg),
                                              _stream_handle(stream)), "mars_cache_autotune")
        return {"threads": list(cfg.threads), "blocks_per_sm": list(cfg.blocks_per_sm),
                "max_registers": list(cfg.max_registers), "lanes": cfg.lanes, "lane_min_pixels": cfg.lane_min_pixels}

    def update_counts(self, stream=None) -> None:
        A.check(self._lib.mars_update_counts(self.handle, _stream_handle(stream)), "mars_update_counts")

    def get_state(self, stream=None) -> dict:
        c, px = self.n_cells, self.n_pixels
        out = {
            "q_rr": np.zeros((c, 3, 3), np.float32), "q_s": np.zeros((c, 3, 3), np.float32),
            "valid": np.zeros((c, 3), np.uint8), "stats": np.zeros((c, 3, 8), np.float64),
            "pixel_estimate": np.zeros((px, 3), np.float32), "run_sum": np.zeros((px, 3), np.float32),
            "pixel_rays": np.zeros(px, np.float32),
        }
        guided = bool(self.techniques & A.MARS_TECH_GUIDED)
        if guided:
            out["guide_hist"] = np.zeros((c, A.GUIDE_BINS), np.float32)
            out["guide_cdf"] = np.zeros((c, A.GUIDE_BINS), np.float32)
        s = A.mars_cache_state()
        s.q_rr, s.q_s = _dp(out["q_rr"], ct.c_float), _dp(out["q_s"], ct.c_float)
        s.valid, s.stats = _dp(out["valid"], ct.c_uint8), _dp(out["stats"], ct.c_double)
        s.pixel_estimate, s.run_sum = _dp(out["pixel_estimate"], ct.c_float), _dp(out["run_sum"], ct.c_float)
        s.pixel_rays = _dp(out["pixel_rays"], ct.c_float)
        if guided:
            s.guide_hist, s.guide_cdf = _dp(out["guide_hist"], ct.c_float), _dp(out["guide_cdf"], ct.c_float)
        if self.octree:
            nodes = np.zeros(self.oct_cap_nodes, np.int32)
            levels = np.zeros(c, np.int32)
            s.oct_nodes, s.oct_leaf_level = _dp(nodes, ct.c_int32), _dp(levels, ct.c_int32)
        A.check(self._lib.mars_cache_get_state(self.handle, ct.byref(s), _stream_handle(stream)),
                "mars_cache_get_state")
        out.update(n_iterations=s.n_iterations, has_estimate=bool(s.has_estimate), VI=s.VI, CI=s.CI,
                   image_iterations=s.image_iterations)
        if self.octree:
            out.update(oct_nodes=nodes[:s.oct_n_nodes].copy(), oct_leaf_level=levels[:s.oct_n_leaves].copy(),
                       oct_n_nodes=s.oct_n_nodes, oct_n_leaves=s.oct_n_leaves)
        return out

    def set_state(self, *, q_rr=None, q_s=None, valid=None, stats=None, guide_hist=None, guide_cdf=None,
                  pixel_estimate=None, run_sum=None, n_iterations=0, has_estimate=False, VI=0.0, CI=0.0,
                  image_iterations=0, oct_nodes=None, oct_leaf_level=None, stream=None) -> None:
        c, px = self.n_cells, self.n_pixels
        keep = []

        def arr(x, dtype, shape, ctype):
            if x is None:
                return ct.POINTER(ctype)()
            a = np.ascontiguousarray(x, dtype).reshape(shape)
            keep.append(a)
            return _dp(a, ctype)

        s = A.mars_cache_state()
        s.q_rr = arr(q_rr, np.float32, (c, 3, 3), ct.c_float)
        s.q_s = arr(q_s, np.float32, (c, 3, 3), ct.c_float)
        s.valid = arr(valid, np.uint8, (c, 3), ct.c_uint8)
        s.stats = arr(stats, np.float64, (c, 3, 8), ct.c_double)
        s.guide_hist = arr(guide_hist, np.float32, (c, A.GUIDE_BINS), ct.c_float)
        s.guide_cdf = arr(guide_cdf, np.float32, (c, A.GUIDE_BINS), ct.c_float)
        s.pixel_estimate = arr(pixel_estimate, np.float32, (px, 3), ct.c_float)
        s.run_sum = arr(run_sum, np.float32, (px, 3), ct.c_float)
        s.n_iterations, s.has_estimate = int(n_iterations), int(bool(has_estimate))
        s.VI, s.CI = float(VI), float(CI)
        s.image_iterations = int(image_iterations)
        if oct_nodes is not None:
            on = np.ascontiguousarray(oct_nodes, np.int32)
            ol = np.ascontiguousarray(oct_leaf_level, np.int32)
            keep += [on, ol]
            s.oct_nodes, s.oct_leaf_level = _dp(on, ct.c_int32), _dp(ol, ct.c_int32)
            s.oct_n_nodes, s.oct_n_leaves = len(on), len(ol)
        A.check(self._lib.mars_cache_set_state(self.handle, ct.byref(s), _stream_handle(stream)),
                "mars_cache_set_state")

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mars_cache_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching render server (mars_server_create / mars_submit / mars_poll)."""

    def __init__(self, memory_budget_bytes: int, max_slots: int):
        self._lib = A.load()
        h = ct.c_void_p()
        A.check(self._lib.mars_server_create(int(memory_budget_bytes), int(max_slots), ct.byref(h)),
                "mars_server_create")
        self.handle = h
        self._descs = {}

    def submit(self, desc, *, grid_n, techniques, max_depth, iterations, warmup, seed=0, key=0,
               arena_capacity=0, graphs=True, timeout_s=0.0) -> int:
        d, keep = scene_desc(desc)
        j = A.mars_job_desc()
        j.scene = ct.pointer(d)
        j.cache = A.mars_cache_desc(int(grid_n), int(techniques), int(max_depth),
                                    0 if graphs else A.MARS_CACHE_NO_GRAPHS, int(arena_capacity), 0, 0.0)
        j.seed, j.iterations, j.warmup, j.key = int(seed), int(iterations), int(warmup), int(key)
        j.timeout_s = float(timeout_s)
        jid = ct.c_uint64()
        A.check(self._lib.mars_submit(self.handle, ct.byref(j), ct.byref(jid)), "mars_submit")
        self._descs[jid.value] = (desc.width, desc.height)
        return jid.value

    def poll(self, job_id: int, want_image: bool = False):
        s = A.mars_job_status()
        img = None
        ptr = None
        if want_image:
            w, h = self._descs[job_id]
            img = np.zeros((h, w, 3), np.float32)
            ptr = img.ctypes.data
        A.check(self._lib.mars_poll(self.handle, ct.c_uint64(job_id), ct.byref(s), ptr), "mars_poll")
        st = {f: getattr(s, f) for f, _ in A.mars_job_status._fields_}
        if s.state == A.MARS_JOB_FAILED:
            msg = self._lib.mars_last_error_string()
            st["message"] = msg.decode() if msg else ""
        return st, img

    def latencies(self, job_id: int) -> np.ndarray:
        """Per-iteration latencies (ms) of a job, in iteration order."""
        n = ct.c_int32()
        A.check(self._lib.mars_job_latencies(self.handle, ct.c_uint64(job_id), None, 0, ct.byref(n)),
                "mars_job_latencies")
        out = np.zeros(max(n.value, 1), np.float64)
        A.check(self._lib.mars_job_latencies(self.handle, ct.c_uint64(job_id), out.ctypes.data, n.value,
                                             ct.byref(n)), "mars_job_latencies")
        return out[:n.value]

    def close(self):
        if getattr(self, "handle", None):
            self._lib.mars_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def training_step_ends(iteration: int, warmup: int, iterations: int) -> bool:
    """Whether render `iteration` of a job of `iterations` one-sample renders
    (the first `warmup` warm-up renders) closes a training iteration, so that
    update_counts follows it (mars_training_step_ends in mars.h)."""
    return bool(A.load().mars_training_step_ends(int(iteration), int(warmup), int(iterations)))


def training_schedule(iterations: int, warmup: int) -> list:
    """Renders per training iteration of such a job, e.g. 3 warm-up renders and
    32 in all: [1, 1, 1, 1, 2, 4, 8, 14]; 35 in all: [1, 1, 1, 1, 2, 4, 8, 17]."""
    out, n = [], 0
    for k in range(iterations):
        n += 1
        if training_step_ends(k, warmup, iterations):
            out.append(n)
            n = 0
    return out


def inject_failure(kind: int, n: int) -> None:
    """Testing hook: the n-th next device allocation (kind MARS_INJECT_ALLOC) or
    render / update call (kind MARS_INJECT_LAUNCH) of the library fails; n = 0
    cancels (see mars_debug_inject_failure in mars.h)."""
    A.check(A.load().mars_debug_inject_failure(int(kind), int(n)), "mars_debug_inject_failure")
