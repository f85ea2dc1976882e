"""ctypes front end of the CPU oracle for MARS (Meyer et al. 2024).

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA path; only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import it.
It shares no code with the CUDA path (``paper_2410_20429_gb300``).

The C source is ``mars_oracle.c`` (plain C, float64, single thread), compiled
with ``gcc -O2 -ffp-contract=off`` into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mars_oracle.c")
_HDR = os.path.join(_HERE, "mars_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmars_oracle.so")
_lock = threading.Lock()
_lib = None

NT = 3
NSTAT = 8
GUIDE_BINS = 256
MODE_WARMUP, MODE_MARS, MODE_FIXED = 0, 1, 2
WEIGHTS_AWARE, WEIGHTS_UNAWARE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or force or any(
        os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR))
    if stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class SceneDesc(ct.Structure):
    _fields_ = [
        ("n_quads", ct.c_int), ("n_spheres", ct.c_int), ("n_tris", ct.c_int), ("n_materials", ct.c_int),
        ("quads", ct.POINTER(ct.c_double)), ("quad_mat", ct.POINTER(ct.c_int32)),
        ("spheres", ct.POINTER(ct.c_double)), ("sphere_mat", ct.POINTER(ct.c_int32)),
        ("tris", ct.POINTER(ct.c_double)), ("tri_mat", ct.POINTER(ct.c_int32)),
        ("materials", ct.POINTER(ct.c_double)),
        ("camera", ct.c_double * 10),
        ("width", ct.c_int), ("height", ct.c_int),
    ]


class Params(ct.Structure):
    _fields_ = [
        ("grid_n", ct.c_int), ("techniques", ct.c_int), ("max_depth", ct.c_int),
        ("mode", ct.c_int), ("weights", ct.c_int),
        ("seed", ct.c_uint32), ("job", ct.c_uint32), ("iteration", ct.c_uint32),
        ("clamp_lo", ct.c_double), ("clamp_hi", ct.c_double), ("outlier", ct.c_double),
        ("has_estimate", ct.c_int), ("collect", ct.c_int), ("max_mult", ct.c_float),
    ]


class State(ct.Structure):
    _fields_ = [
        ("q_rr", ct.POINTER(ct.c_float)), ("q_s", ct.POINTER(ct.c_float)),
        ("valid", ct.POINTER(ct.c_uint8)), ("guide_cdf", ct.POINTER(ct.c_float)),
        ("est", ct.POINTER(ct.c_float)), ("oct_nodes", ct.POINTER(ct.c_int32)),
        ("image", ct.POINTER(ct.c_double)), ("stats", ct.POINTER(ct.c_double)),
        ("hist", ct.POINTER(ct.c_double)), ("counters", ct.POINTER(ct.c_double)),
        ("px_rays", ct.POINTER(ct.c_double)),
    ]


def _p(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype)) if a is not None else ct.POINTER(ctype)()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            L.orc_render.argtypes = [ct.POINTER(SceneDesc), ct.POINTER(Params), ct.POINTER(State),
                                     ct.c_int, ct.c_int]
            L.orc_render.restype = ct.c_int
            L.orc_image_stats.argtypes = [ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                          ct.c_int, ct.c_double, ct.POINTER(ct.c_double)]
            L.orc_image_stats.restype = ct.c_double
            L.orc_image_stats_k.argtypes = [ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                            ct.c_int, ct.c_double, ct.c_int, ct.POINTER(ct.c_double)]
            L.orc_image_stats_k.restype = ct.c_double
            L.orc_update_counts.argtypes = [ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.c_double,
                                            ct.c_double, ct.POINTER(ct.c_float), ct.POINTER(ct.c_float),
                                            ct.POINTER(ct.c_uint8)]
            L.orc_update_counts.restype = None
            L.orc_guide_update.argtypes = [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_float)]
            L.orc_guide_update.restype = None
            L.orc_philox4x32_10.argtypes = [ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint32),
                                            ct.POINTER(ct.c_uint32)]
            L.orc_philox4x32_10.restype = None
            L.orc_stochastic_round.argtypes = [ct.c_int, ct.POINTER(ct.c_float), ct.c_float,
                                               ct.POINTER(ct.c_int32)]
            L.orc_stochastic_round.restype = None
            L.orc_vertex_count.argtypes = [ct.POINTER(ct.c_float), ct.POINTER(ct.c_float),
                                           ct.POINTER(ct.c_double), ct.POINTER(ct.c_float),
                                           ct.c_double, ct.c_double]
            L.orc_vertex_count.restype = ct.c_double
            L.orc_balance_weight.argtypes = [ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                             ct.POINTER(ct.c_int), ct.c_int, ct.c_int]
            L.orc_balance_weight.restype = ct.c_double
            L.orc_bsdf_eval_local.argtypes = [ct.POINTER(SceneDesc), ct.c_int, ct.POINTER(ct.c_double),
                                              ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                                              ct.POINTER(ct.c_double)]
            L.orc_bsdf_eval_local.restype = None
            L.orc_bsdf_sample_local.argtypes = [ct.POINTER(SceneDesc), ct.c_int, ct.POINTER(ct.c_double),
                                                ct.c_double, ct.c_double, ct.POINTER(ct.c_double),
                                                ct.POINTER(ct.c_double)]
            L.orc_bsdf_sample_local.restype = ct.c_int
            I32 = ct.POINTER(ct.c_int32)
            D = ct.POINTER(ct.c_double)
            L.orc_debug_light_emit.argtypes = [ct.POINTER(SceneDesc), ct.POINTER(Params), ct.c_int, D, ct.c_int, D,
                                               D, I32]
            L.orc_debug_light_emit.restype = ct.c_int
            L.orc_debug_light_bounce.argtypes = [ct.POINTER(SceneDesc), ct.POINTER(Params), ct.c_int, D, D,
                                                 ct.c_int, D, D, I32]
            L.orc_debug_light_bounce.restype = ct.c_int
            L.orc_debug_light_density.argtypes = [ct.POINTER(SceneDesc), ct.POINTER(Params), ct.c_int, D, D, D, D]
            L.orc_debug_light_density.restype = ct.c_int
            L.orc_octree_init.argtypes = [ct.c_int, I32, I32, I32]
            L.orc_octree_init.restype = ct.c_int
            L.orc_octree_refine.argtypes = [ct.c_int, ct.c_double, ct.POINTER(ct.c_double), I32, I32, I32, I32, I32,
                                            ct.POINTER(ct.c_float), ct.POINTER(ct.c_float), ct.POINTER(ct.c_uint8),
                                            ct.POINTER(ct.c_double), ct.POINTER(ct.c_float)]
            L.orc_octree_refine.restype = ct.c_int
            L.orc_octree_cell.argtypes = [ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), I32,
                                          ct.POINTER(ct.c_double)]
            L.orc_octree_cell.restype = ct.c_int
            L.orc_guide_pdf.argtypes = [ct.POINTER(ct.c_float), ct.POINTER(ct.c_double)]
            L.orc_guide_pdf.restype = ct.c_double
            L.orc_guide_sample.argtypes = [ct.POINTER(ct.c_float), ct.c_double, ct.c_double, ct.c_double,
                                           ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            L.orc_guide_sample.restype = None
            _lib = L
    return _lib


class _SceneHolder:
    """Keeps the numpy arrays alive while the C descriptor points at them."""

    def __init__(self, scene):
        self.arrays = [
            np.ascontiguousarray(scene.quads, dtype=np.float64),
            np.ascontiguousarray(scene.quad_mat, dtype=np.int32),
            np.ascontiguousarray(scene.spheres, dtype=np.float64),
            np.ascontiguousarray(scene.sphere_mat, dtype=np.int32),
            np.ascontiguousarray(scene.tris, dtype=np.float64),
            np.ascontiguousarray(scene.tri_mat, dtype=np.int32),
            np.ascontiguousarray(scene.materials, dtype=np.float64),
        ]
        q, qm, s, sm, t, tm, m = self.arrays
        d = SceneDesc()
        d.n_quads, d.n_spheres, d.n_tris, d.n_materials = len(q), len(s), len(t), len(m)
        d.quads, d.quad_mat = _p(q, ct.c_double), _p(qm, ct.c_int32)
        d.spheres, d.sphere_mat = _p(s, ct.c_double), _p(sm, ct.c_int32)
        d.tris, d.tri_mat = _p(t, ct.c_double), _p(tm, ct.c_int32)
        d.materials = _p(m, ct.c_double)
        for i in range(10):
            d.camera[i] = float(scene.camera[i])
        d.width, d.height = scene.width, scene.height
        self.desc = d


class RenderResult:
    def __init__(self, image, stats, hist, counters, px_rays=None):
        self.image = image          # [pixels, 3] float64
        self.stats = stats          # [cells, 3, 8] float64
        self.hist = hist            # [cells, 256] float64
        self.counters = counters    # rays, traced vertices, estimator vertices, sum beta x3
        self.px_rays = px_rays      # [pixels] rays of each pixel's path tree (rendered pixels)

    @property
    def rays(self) -> float:
        return float(self.counters[0])

    @property
    def vertices(self) -> float:
        return float(self.counters[1])


def render(scene, *, grid_n, techniques, max_depth, mode=MODE_WARMUP, weights=WEIGHTS_AWARE,
           seed=0, job=0, iteration=0, clamp_lo=0.05, clamp_hi=20.0, outlier=50.0,
           q_rr=None, q_s=None, valid=None, guide_cdf=None, est=None, collect=True,
           px_begin=0, px_end=None, max_mult=0.0, octree=None) -> RenderResult:
    """One iteration of the MARS path tracer over pixels [px_begin, px_end).
    ``octree``: (nodes int32 array, cells) to use an adaptive octree cache with
    that many cells instead of the uniform grid_n^3 grid."""
    L = lib()
    cells = grid_n ** 3 if octree is None else int(octree[1])
    oct_nodes = None if octree is None else np.ascontiguousarray(octree[0], np.int32)
    npx = scene.width * scene.height
    if px_end is None:
        px_end = npx
    if q_rr is None:
        q_rr = np.zeros((cells, NT, 3), np.float32)
    if q_s is None:
        q_s = np.zeros((cells, NT, 3), np.float32)
    if valid is None:
        valid = np.zeros((cells, NT), np.uint8)
    if guide_cdf is None and (techniques & 4):
        guide_cdf = np.tile((np.arange(1, GUIDE_BINS + 1, dtype=np.float64) / GUIDE_BINS).astype(np.float32),
                            (cells, 1))
    has_est = est is not None
    if est is None:
        est = np.ones((npx, 3), np.float32)
    q_rr = np.ascontiguousarray(q_rr, np.float32).reshape(cells, NT, 3)
    q_s = np.ascontiguousarray(q_s, np.float32).reshape(cells, NT, 3)
    valid = np.ascontiguousarray(valid, np.uint8).reshape(cells, NT)
    est = np.ascontiguousarray(est, np.float32).reshape(npx, 3)
    if guide_cdf is not None:
        guide_cdf = np.ascontiguousarray(guide_cdf, np.float32).reshape(cells, GUIDE_BINS)
    image = np.zeros((npx, 3), np.float64)
    stats = np.zeros((cells, NT, NSTAT), np.float64)
    hist = np.zeros((cells, GUIDE_BINS), np.float64)
    counters = np.zeros(8, np.float64)
    px_rays = np.zeros(npx, np.float64)
    sh = _SceneHolder(scene)
    P = Params(grid_n, techniques, max_depth, mode, weights, seed, job, iteration,
               clamp_lo, clamp_hi, outlier, int(has_est), int(bool(collect)), float(max_mult))
    S = State(_p(q_rr, ct.c_float), _p(q_s, ct.c_float), _p(valid, ct.c_uint8),
              _p(guide_cdf, ct.c_float), _p(est, ct.c_float), _p(oct_nodes, ct.c_int32), _p(image, ct.c_double),
              _p(stats, ct.c_double), _p(hist, ct.c_double), _p(counters, ct.c_double), _p(px_rays, ct.c_double))
    rc = L.orc_render(ct.byref(sh.desc), ct.byref(P), ct.byref(S), int(px_begin), int(px_end))
    if rc != 0:
        raise ValueError(f"orc_render failed with {rc}")
    return RenderResult(image, stats, hist, counters, px_rays)


def render_samples(scene, n, *, grid_n, techniques, max_depth, mode=MODE_WARMUP, weights=WEIGHTS_AWARE,
                   seed=0, px=0, clamp_lo=0.05, clamp_hi=20.0, outlier=50.0, q_rr=None, q_s=None, valid=None,
                   est=None, collect=True):
    """Pixel ``px`` rendered in n independent iterations (Philox iteration k,
    k < 65536): one call of orc_render per iteration on reused buffers, so that
    many samples of one pixel are cheap.  Returns (values [n, 3] float64, the
    statistics summed over the n iterations [cells, 3, 8], the counters summed
    over them)."""
    L = lib()
    if n > 65536:
        raise ValueError("at most 65536 iterations per key")
    cells = grid_n ** 3
    npx = scene.width * scene.height
    q_rr = np.ascontiguousarray(np.zeros((cells, NT, 3)) if q_rr is None else q_rr, np.float32).reshape(cells, NT, 3)
    q_s = np.ascontiguousarray(np.zeros((cells, NT, 3)) if q_s is None else q_s, np.float32).reshape(cells, NT, 3)
    valid = np.ascontiguousarray(np.zeros((cells, NT)) if valid is None else valid, np.uint8).reshape(cells, NT)
    has_est = est is not None
    est = np.ascontiguousarray(np.ones((npx, 3)) if est is None else est, np.float32).reshape(npx, 3)
    image = np.zeros((npx, 3), np.float64)
    stats = np.zeros((cells, NT, NSTAT), np.float64)
    hist = np.zeros((cells, GUIDE_BINS), np.float64)
    counters = np.zeros(8, np.float64)
    sh = _SceneHolder(scene)
    P = Params(grid_n, techniques, max_depth, mode, weights, seed, 0, 0, clamp_lo, clamp_hi, outlier,
               int(has_est), int(bool(collect)), 0.0)
    S = State(_p(q_rr, ct.c_float), _p(q_s, ct.c_float), _p(valid, ct.c_uint8), ct.POINTER(ct.c_float)(),
              _p(est, ct.c_float), ct.POINTER(ct.c_int32)(), _p(image, ct.c_double), _p(stats, ct.c_double),
              _p(hist, ct.c_double), _p(counters, ct.c_double), ct.POINTER(ct.c_double)())
    out = np.zeros((n, 3), np.float64)
    for k in range(n):
        P.iteration = k
        rc = L.orc_render(ct.byref(sh.desc), ct.byref(P), ct.byref(S), int(px), int(px) + 1)
        if rc != 0:
            raise ValueError(f"orc_render failed with {rc}")
        out[k] = image[px]
    return out, stats, counters


def image_stats(width, height, img, run_sum, n_prev, outlier=50.0, drop_k=0):
    """Returns (V_I, new run_sum, pixel estimate).  drop_k > 0: the rejection of
    the bidirectional application (Sec. 5.1) instead of the outlier clamp."""
    L = lib()
    img = np.ascontiguousarray(img, np.float64).reshape(-1, 3)
    rs = np.array(run_sum, dtype=np.float64).reshape(-1, 3).copy()
    est = np.zeros_like(rs)
    vi = L.orc_image_stats_k(int(width), int(height), _p(img, ct.c_double), _p(rs, ct.c_double),
                             int(n_prev), float(outlier), int(drop_k), _p(est, ct.c_double))
    return float(vi), rs, est


def combine(images, vis):
    """Progressive combination of Sec. 5.1 ("the inverse-variance weighted
    combination of all iterations"): sum_i w_i I_i / sum_i w_i with
    w_i = 1 / max(V_I of iteration i, 1e-12).  Returns (image, sum of weights)."""
    acc = None
    wsum = 0.0
    for img, vi in zip(images, vis):
        w = 1.0 / max(float(vi), 1e-12)
        a = np.asarray(img, np.float64) * w
        acc = a if acc is None else acc + a
        wsum += w
    return acc / wsum, wsum


def update_counts(stats, VI, CI, techniques, q_rr, q_s, valid):
    """One fixed-point step; returns new (q_rr, q_s, valid)."""
    L = lib()
    stats = np.ascontiguousarray(stats, np.float64)
    cells = stats.shape[0]
    q_rr = np.array(q_rr, np.float32).reshape(cells, NT, 3).copy()
    q_s = np.array(q_s, np.float32).reshape(cells, NT, 3).copy()
    valid = np.array(valid, np.uint8).reshape(cells, NT).copy()
    L.orc_update_counts(cells, int(techniques), _p(stats, ct.c_double), float(VI), float(CI),
                        _p(q_rr, ct.c_float), _p(q_s, ct.c_float), _p(valid, ct.c_uint8))
    return q_rr, q_s, valid


OCT_LMAX = 10


def octree_init(grid_n, max_leaves):
    """The adaptive octree equal to the uniform grid: (nodes, n_nodes, n_leaves,
    leaf_level, leaf_node) with arrays sized for max_leaves cells."""
    L = lib()
    cap_nodes = 2 * max_leaves + 8 ** 4
    nodes = np.zeros(cap_nodes, np.int32)
    level = np.zeros(max_leaves, np.int32)
    lnode = np.zeros(max_leaves, np.int32)
    n = L.orc_octree_init(int(grid_n), _p(nodes, ct.c_int32), _p(level, ct.c_int32), _p(lnode, ct.c_int32))
    if n < 0:
        raise ValueError("grid_n must be a power of two up to 2^10")
    return nodes, n, grid_n ** 3, level, lnode


def octree_refine(max_leaves, split_samples, stats, nodes, n_nodes, n_leaves, level, lnode, q_rr, q_s, valid,
                  hist=None, cdf=None):
    """One refinement step (in place on copies); returns the new
    (nodes, n_nodes, n_leaves, level, lnode, q_rr, q_s, valid, hist, cdf, splits)."""
    L = lib()
    nodes, level, lnode = nodes.copy(), level.copy(), lnode.copy()
    q_rr = np.array(q_rr, np.float32).copy()
    q_s = np.array(q_s, np.float32).copy()
    valid = np.array(valid, np.uint8).copy()
    hist = None if hist is None else np.array(hist, np.float64).copy()
    cdf = None if cdf is None else np.array(cdf, np.float32).copy()
    nn, nl = ct.c_int32(n_nodes), ct.c_int32(n_leaves)
    stats = np.ascontiguousarray(stats, np.float64)
    sp = L.orc_octree_refine(int(max_leaves), float(split_samples), _p(stats, ct.c_double), _p(nodes, ct.c_int32),
                             ct.byref(nn), ct.byref(nl), _p(level, ct.c_int32), _p(lnode, ct.c_int32),
                             _p(q_rr, ct.c_float), _p(q_s, ct.c_float), _p(valid, ct.c_uint8),
                             _p(hist, ct.c_double), _p(cdf, ct.c_float))
    return nodes, nn.value, nl.value, level, lnode, q_rr, q_s, valid, hist, cdf, sp


def octree_cell(lo, ext, nodes, p):
    L = lib()
    lo = np.ascontiguousarray(lo, np.float64)
    ext = np.ascontiguousarray(ext, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    nodes = np.ascontiguousarray(nodes, np.int32)
    return int(L.orc_octree_cell(_p(lo, ct.c_double), _p(ext, ct.c_double), _p(nodes, ct.c_int32),
                                 _p(p, ct.c_double)))


def guide_update(hist):
    L = lib()
    hist = np.ascontiguousarray(hist, np.float64)
    cdf = np.zeros(hist.shape, np.float32)
    L.orc_guide_update(hist.shape[0], _p(hist, ct.c_double), _p(cdf, ct.c_float))
    return cdf


def philox(ctr, key):
    L = lib()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    L.orc_philox4x32_10(_p(c, ct.c_uint32), _p(k, ct.c_uint32), _p(o, ct.c_uint32))
    return o


def stochastic_round(beta, r):
    L = lib()
    b = np.ascontiguousarray(beta, np.float32)
    g = np.zeros(len(b), np.int32)
    L.orc_stochastic_round(len(b), _p(b, ct.c_float), ct.c_float(float(r)), _p(g, ct.c_int32))
    return g


def vertex_count(q_rr, q_s, T, I, lo=0.05, hi=20.0):
    L = lib()
    a = np.ascontiguousarray(q_rr, np.float32)
    b = np.ascontiguousarray(q_s, np.float32)
    t = np.ascontiguousarray(T, np.float64)
    i = np.ascontiguousarray(I, np.float32)
    return L.orc_vertex_count(_p(a, ct.c_float), _p(b, ct.c_float), _p(t, ct.c_double), _p(i, ct.c_float),
                              float(lo), float(hi))


def balance_weight(beta, pdf, participates, t, aware=True):
    L = lib()
    b = np.ascontiguousarray(beta, np.float64)
    p = np.ascontiguousarray(pdf, np.float64)
    q = np.ascontiguousarray(participates, np.int32)
    return L.orc_balance_weight(len(b), _p(b, ct.c_double), _p(p, ct.c_double), _p(q, ct.c_int), int(t),
                                int(bool(aware)))


def _debug_params(techniques=7, max_depth=6):
    return Params(4, techniques, max_depth, MODE_WARMUP, WEIGHTS_AWARE, 0, 0, 0, 0.05, 20.0, 50.0, 0, 0, 0.0)


def light_emit(scene, light, y0, u):
    """Test hook: the first hits of cosine emission directions from point y0 of
    light ``light`` drawn by u[i] = (u0, u1); returns (hits [n, 3], prims [n],
    -1 on a miss)."""
    L = lib()
    sh = _SceneHolder(scene)
    P = _debug_params()
    y = np.ascontiguousarray(y0, np.float64)
    uu = np.ascontiguousarray(u, np.float64).reshape(-1, 2)
    hit = np.zeros((len(uu), 3), np.float64)
    prim = np.zeros(len(uu), np.int32)
    rc = L.orc_debug_light_emit(ct.byref(sh.desc), ct.byref(P), int(light), _p(y, ct.c_double), len(uu),
                                _p(uu, ct.c_double), _p(hit, ct.c_double), _p(prim, ct.c_int32))
    if rc != 0:
        raise ValueError(f"orc_debug_light_emit failed with {rc}")
    return hit, prim


def light_bounce(scene, light, y0, d1, u):
    """Test hook: the light subpath vertex y_1 hit from y0 along d1, and the next
    vertex of bounces there drawn by u[i] = (u0, u1, u2) (BSDF sampling and the
    roulette); returns (hits [n, 3], prims [n], -1 when the subpath ended)."""
    L = lib()
    sh = _SceneHolder(scene)
    P = _debug_params()
    y = np.ascontiguousarray(y0, np.float64)
    d = np.ascontiguousarray(d1, np.float64)
    uu = np.ascontiguousarray(u, np.float64).reshape(-1, 3)
    hit = np.zeros((len(uu), 3), np.float64)
    prim = np.zeros(len(uu), np.int32)
    rc = L.orc_debug_light_bounce(ct.byref(sh.desc), ct.byref(P), int(light), _p(y, ct.c_double),
                                  _p(d, ct.c_double), len(uu), _p(uu, ct.c_double), _p(hit, ct.c_double),
                                  _p(prim, ct.c_int32))
    if rc != 0:
        raise ValueError(f"orc_debug_light_bounce failed with {rc}")
    return hit, prim


def light_density(scene, light, y0, d1, x):
    """Test hook: (P<- of y_1, the first hit from y0 along d1; P<- of the first
    hit from y_1 towards x, the light arriving from y0), the light-side area
    densities of the whole-path weights."""
    L = lib()
    sh = _SceneHolder(scene)
    P = _debug_params()
    y = np.ascontiguousarray(y0, np.float64)
    d = np.ascontiguousarray(d1, np.float64)
    xx = np.ascontiguousarray(x, np.float64)
    out = np.zeros(2, np.float64)
    rc = L.orc_debug_light_density(ct.byref(sh.desc), ct.byref(P), int(light), _p(y, ct.c_double),
                                   _p(d, ct.c_double), _p(xx, ct.c_double), _p(out, ct.c_double))
    if rc != 0:
        raise ValueError(f"orc_debug_light_density failed with {rc}")
    return float(out[0]), float(out[1])


def bsdf_eval_local(scene, mat, wo, wi):
    L = lib()
    sh = _SceneHolder(scene)
    a = np.ascontiguousarray(wo, np.float64)
    b = np.ascontiguousarray(wi, np.float64)
    f = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    L.orc_bsdf_eval_local(ct.byref(sh.desc), int(mat), _p(a, ct.c_double), _p(b, ct.c_double),
                          _p(f, ct.c_double), _p(pdf, ct.c_double))
    return f, float(pdf[0])


def bsdf_sample_local(scene, mat, wo, u0, u1):
    L = lib()
    sh = _SceneHolder(scene)
    a = np.ascontiguousarray(wo, np.float64)
    wi = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    ok = L.orc_bsdf_sample_local(ct.byref(sh.desc), int(mat), _p(a, ct.c_double), float(u0), float(u1),
                                 _p(wi, ct.c_double), _p(pdf, ct.c_double))
    return bool(ok), wi, float(pdf[0])


def guide_pdf(cdf, w):
    L = lib()
    c = np.ascontiguousarray(cdf, np.float32)
    d = np.ascontiguousarray(w, np.float64)
    return L.orc_guide_pdf(_p(c, ct.c_float), _p(d, ct.c_double))


def guide_sample(cdf, u0, u1, u2):
    L = lib()
    c = np.ascontiguousarray(cdf, np.float32)
    w = np.zeros(3, np.float64)
    pdf = np.zeros(1, np.float64)
    L.orc_guide_sample(_p(c, ct.c_float), float(u0), float(u1), float(u2), _p(w, ct.c_double),
                       _p(pdf, ct.c_double))
    return w, float(pdf[0])
