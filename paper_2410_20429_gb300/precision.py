"""Precision study: float32 versus float64 statistics.

The statistics cache accumulates, per (cell, technique), the sample count, the
sums of the sample values and of their squares (per channel) and the sum of the
sample costs; the fixed-point update turns them into the count factors q^RR and
q^S, and the image pass reduces V_I and C_I.  ``compare`` renders the same
iteration from the same state (same count fields, pixel estimate and random
numbers) on a float64 cache and on a float32-statistics cache, runs the update
on both, and states the relative error of every statistic of the float32 run
against the float64 one.  Everything is computed by the CUDA library; this
module only reads the two caches' states back and summarises the differences.
"""
from __future__ import annotations

import numpy as np

from . import _abi as A
from .renderer import Cache, Scene

STATISTICS = ["n", "sum_v", "sum_v2", "sum_cost", "m1", "m2", "var", "C_t", "q_rr", "q_s", "V_I", "C_I"]


def _rel(a64, a32, floor):
    a64 = np.asarray(a64, np.float64)
    a32 = np.asarray(a32, np.float64)
    return np.abs(a32 - a64) / np.maximum(np.abs(a64), floor)


def _summary(r):
    r = np.asarray(r, np.float64).ravel()
    if r.size == 0:
        return {"max": 0.0, "p99": 0.0, "median": 0.0, "count": 0}
    return {"max": float(r.max()), "p99": float(np.percentile(r, 99)), "median": float(np.median(r)),
            "count": int(r.size)}


def compare(scene_desc, grid_n, techniques, max_depth, q_rr, q_s, valid, pixel_estimate, run_sum, n_prev,
            iteration=1, seed=0, min_samples=2, stream=None, cache_kw=None, tree=None, guide_cdf=None):
    """Render one MARS iteration on a float64 and a float32-statistics cache
    from the same state; returns {statistic: {max, p99, median, count}} of the
    float32 run's relative error over the populated (cell, technique) entries
    with at least ``min_samples`` samples (per channel for the rgb sums), plus
    the two images' agreement.  ``cache_kw`` (e.g. the octree settings) and
    ``tree`` = (oct_nodes, oct_leaf_level) configure both caches alike."""
    scene = Scene(scene_desc, stream=stream)
    res = {}
    for fp32 in (False, True):
        cache = Cache(scene, grid_n, techniques, max_depth, fp32_statistics=fp32, stream=stream, **(cache_kw or {}))
        extra = {} if tree is None else dict(oct_nodes=tree[0], oct_leaf_level=tree[1])
        if guide_cdf is not None:
            extra["guide_cdf"] = guide_cdf
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=pixel_estimate, run_sum=run_sum,
                        n_iterations=n_prev, has_estimate=True, stream=stream, **extra)
        img = np.zeros(3 * cache.n_pixels, np.float32)
        st = cache.render_iteration(img, seed=seed, iteration=iteration, mode=A.MARS_MODE_MARS,
                                    update_estimate=True, stream=stream)
        before = cache.get_state(stream=stream)
        cache.update_counts(stream=stream)
        after = cache.get_state(stream=stream)
        res[fp32] = (img, st, before, after)
        cache.close()
    scene.close()
    (i64, st64, b64, a64), (i32, st32, b32, a32) = res[False], res[True]
    s64, s32 = b64["stats"], b32["stats"]
    n = s64[..., 0]
    pop = n >= min_samples
    out = {}
    out["n"] = _summary(_rel(s64[..., 0][pop], s32[..., 0][pop], 1.0))
    out["sum_cost"] = _summary(_rel(s64[..., 7][pop], s32[..., 7][pop], 1.0))
    m = pop[..., None]
    for k, name in ((1, "sum_v"), (4, "sum_v2")):
        v64, v32 = s64[..., k:k + 3], s32[..., k:k + 3]
        sel = np.broadcast_to(m, v64.shape) & (v64 > 0)
        out[name] = _summary(_rel(v64[sel], v32[sel], 1e-30))

    def moments(s):
        nn = np.maximum(s[..., 0:1], 1.0)
        m1 = s[..., 1:4] / nn
        m2 = s[..., 4:7] / nn
        var = np.maximum(m2 - m1 * m1, 0.0)
        ct = s[..., 7] / np.maximum(s[..., 0], 1.0)
        return m1, m2, var, ct

    m1a, m2a, vara, cta = moments(s64)
    m1b, m2b, varb, ctb = moments(s32)
    sel = np.broadcast_to(m, m1a.shape)
    out["m1"] = _summary(_rel(m1a[sel & (m1a > 0)], m1b[sel & (m1a > 0)], 1e-30))
    out["m2"] = _summary(_rel(m2a[sel & (m2a > 0)], m2b[sel & (m2a > 0)], 1e-30))
    # the variance loses digits to cancellation where it is small against m2:
    # report it where var > 1e-3 m2, and the worst cancellation case separately
    good = sel & (vara > 1e-3 * m2a)
    out["var"] = _summary(_rel(vara[good], varb[good], 1e-30))
    out["C_t"] = _summary(_rel(cta[pop], ctb[pop], 1e-30))
    upd = (a64["valid"] > 0) & pop
    mq = np.broadcast_to(upd[..., None], a64["q_rr"].shape)
    out["q_rr"] = _summary(_rel(a64["q_rr"][mq & (a64["q_rr"] > 0)], a32["q_rr"][mq & (a64["q_rr"] > 0)], 1e-30))
    gq = mq & np.broadcast_to(good, mq.shape)
    out["q_s"] = _summary(_rel(a64["q_s"][gq & (a64["q_s"] > 0)], a32["q_s"][gq & (a64["q_s"] > 0)], 1e-30))
    out["V_I"] = _summary(_rel([st64["VI"]], [st32["VI"]], 1e-30))
    out["C_I"] = _summary(_rel([st64["CI"]], [st32["CI"]], 1e-30))
    out["images_equal"] = bool(np.array_equal(i64, i32))
    out["cells_compared"] = int(pop.sum())
    return out
