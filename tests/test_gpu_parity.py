"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs and the same Philox streams.

Bars (floating point; the oracle is float64, the CUDA path float32):
* images: at least 99.9 % of pixels agree within 1e-4 relative in every channel
  (a rare pixel may take a different discrete branch -- a rounding decision of
  Alg. 1 or a grazing hit -- because float32 and float64 differ in the last bits);
* per-cell statistics: every (cell, technique) entry that no disagreeing
  pixel's path reaches agrees within 1e-3 relative in all 8 sums (the cells a
  disagreeing pixel reaches are found by rendering that pixel alone, on both
  sides, from the same state); the fraction of all populated entries that
  agree is printed; the sums over all cells agree within 1e-3 relative;
* integer counters (rays, traced vertices) within 0.1 %.
"""
import math

import numpy as np
import pytest

import mars_workloads as W

pytestmark = pytest.mark.gpu

PIX_TOL = 1e-4
STAT_TOL = 1e-3


@pytest.fixture(scope="module")
def mars():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2410_20429_gb300 import build as B
    B.build()
    import paper_2410_20429_gb300 as M
    return M


def _gpu_iteration(M, cache, *, iteration=0, seed=0, mode=0, weights=0, update_estimate=False, collect=True):
    import torch
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    st = cache.render_iteration(img, seed=seed, iteration=iteration, mode=mode, weights=weights, collect=collect,
                                update_estimate=update_estimate)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(-1, 3).astype(np.float64), st


def _pixel_agreement(g, o):
    ok = np.abs(g - o) <= PIX_TOL * np.abs(o) + 1e-7
    return ok.all(axis=1).mean()


def _stat_agreement(gs, os_):
    """fraction of populated (cell, technique) entries whose 8 statistics agree"""
    n_g, n_o = gs[..., 0], os_[..., 0]
    pop = (n_g > 0) | (n_o > 0)
    close = np.abs(gs - os_) <= STAT_TOL * np.abs(os_) + 1e-9
    agree = close.all(axis=-1) & pop
    return agree.sum() / pop.sum() if pop.any() else 1.0   # no samples (D = 1): nothing to disagree


def _touched_cells(M, orc, cache, sc, gpu_kw, orc_kw, pixels):
    """Cells in which any of `pixels`' path trees recorded a sample, on the CUDA
    path (the pixel rendered alone through a pixel range, from the cache's
    state) or in the oracle (the pixel alone): where a pixel took a different
    discrete branch on the two sides, its samples land in different cells."""
    import torch
    touched = np.zeros(cache.n_cells, bool)
    if len(pixels) == 0:
        return touched
    full = cache.get_state()
    saved = full["stats"]
    keep = dict(has_estimate=full["has_estimate"], n_iterations=full["n_iterations"])
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    for px in pixels:
        px = int(px)
        cache.set_state(stats=np.zeros_like(saved), **keep)
        cache.render_iteration(img, update_estimate=False, px_range=(px, px + 1), **gpu_kw)
        torch.cuda.synchronize()
        touched |= cache.get_state()["stats"][..., 0].sum(-1) > 0
        o = orc.render(sc, px_begin=px, px_end=px + 1, **orc_kw)
        touched[: o.stats.shape[0]] |= o.stats[..., 0].sum(-1) > 0
    cache.set_state(stats=saved, **keep)
    return touched


def _stat_tolerance(o_stats):
    """Per-entry tolerance of the 8 sums: the sample count and the summed cost
    are integers and must be equal; the value sums agree within STAT_TOL
    relative, with an absolute floor of STAT_TOL times the technique's mean
    per-sample value (or squared value) times the entry's sample count -- as the
    pixel bar has a floor: a single grazing NEE sample of value 1e-6 carries a
    1 % float32 error that is 1e-4 of a typical sample."""
    tol = STAT_TOL * np.abs(o_stats)
    n = o_stats[..., 0]
    for t in range(o_stats.shape[1]):
        nt = max(n[:, t].sum(), 1.0)
        v1 = np.abs(o_stats[:, t, 1:4]).sum() / (3 * nt)
        v2 = np.abs(o_stats[:, t, 4:7]).sum() / (3 * nt)
        tol[:, t, 1:4] += STAT_TOL * v1 * n[:, t, None]
        tol[:, t, 4:7] += STAT_TOL * v2 * n[:, t, None]
    tol[..., 0] = 0.0
    tol[..., 7] = 0.0
    return tol


def _strict_stats(g_stats, o_stats, touched, what, sensitive=None):
    """Every populated (cell, technique) entry outside the cells reached by a
    disagreeing pixel (and outside the `sensitive` entries, if given) agrees in
    all 8 sums (see _stat_tolerance); returns the fraction of all populated
    entries that agree."""
    g_stats = g_stats[: o_stats.shape[0]]
    pop = (g_stats[..., 0] > 0) | (o_stats[..., 0] > 0)
    close = (np.abs(g_stats - o_stats) <= _stat_tolerance(o_stats) + 1e-12).all(axis=-1)
    keep = pop & ~touched[: o_stats.shape[0], None]
    if sensitive is not None:
        keep &= ~sensitive
    bad = np.argwhere(keep & ~close)
    assert bad.size == 0, f"{what}: {len(bad)} (cell, technique) entries outside the disagreeing pixels' " \
                          f"cells differ, e.g. {bad[:3].tolist()}: " + \
                          "; ".join(f"gpu {g_stats[c, t].tolist()} oracle {o_stats[c, t].tolist()}" for c, t in bad[:2])
    frac = (close & pop).sum() / max(pop.sum(), 1)
    print(f"{what}: {frac:.5f} of {int(pop.sum())} populated entries agree; "
          f"{int(touched.sum())} cells reached by disagreeing pixels")
    return frac


def _check(g_img, o_img, g_state, o_res, g_st, what, touch=None):
    """Image, statistics and counter bars.  touch(pixels) -> the cells those
    pixels reach (see _touched_cells); without it the per-cell bar is 99 % of
    the populated entries."""
    frac = _pixel_agreement(g_img, o_img)
    assert frac >= 0.999, f"{what}: only {frac:.5f} of pixels agree"
    if touch is not None:
        # disagreeing pixels: off by more than the pixel bar, or a path tree of
        # another size (a discrete branch taken differently, even where the
        # extra sample's value is zero)
        off = ~(np.abs(g_img - o_img) <= PIX_TOL * np.abs(o_img) + 1e-7).all(axis=1)
        rays_off = g_state["pixel_rays"].astype(np.float64) != o_res.px_rays
        print(f"{what}: {int(off.sum())} pixels off, {int(rays_off.sum())} with another path-tree size")
        _strict_stats(g_state["stats"], o_res.stats, touch(np.flatnonzero(off | rays_off)), what)
    else:
        sa = _stat_agreement(g_state["stats"], o_res.stats)
        assert sa >= 0.99, f"{what}: only {sa:.4f} of cell statistics agree"
    tot_g = g_state["stats"].sum(axis=0)
    tot_o = o_res.stats.sum(axis=0)
    assert np.allclose(tot_g, tot_o, rtol=STAT_TOL, atol=1e-6), f"{what}: total statistics differ"
    assert abs(g_st["rays"] - o_res.rays) <= 1e-3 * o_res.rays + 1
    assert abs(g_st["vertices"] - o_res.vertices) <= 1e-3 * o_res.vertices + 1


def _make(M, cfg, **kw):
    scene = M.Scene(cfg.scene)
    cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, **kw)
    return scene, cache


def test_box_warmup_iteration_parity(mars, orc):
    cfg = W.config_box(64, 64)
    scene, cache = _make(mars, cfg)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=0, seed=0, mode=0)
    g_state = cache.get_state()
    okw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=0)
    o = orc.render(cfg.scene, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, cfg.scene, dict(iteration=0, seed=0, mode=0), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "box warm-up", touch)
    assert g_st["estimator_vertices"] == pytest.approx(o.counters[2], rel=1e-3)


@pytest.mark.parametrize("weights", [0, 1])
def test_box_mars_iteration_parity(mars, orc, weights):
    """Teacher-forced MARS iteration: random count fields and pixel estimate set
    on both sides; splitting and Russian roulette both occur."""
    cfg = W.config_box(64, 64)
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=101, lo=0.05, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=102, lo=0.05, hi=1.0)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=3, seed=5, mode=1, weights=weights)
    g_state = cache.get_state()
    okw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=3, seed=5,
               mode=orc.MODE_MARS, weights=weights, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
    o = orc.render(cfg.scene, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, cfg.scene,
                                      dict(iteration=3, seed=5, mode=1, weights=weights), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "box MARS", touch)
    # splitting and roulette really happened
    assert o.counters[3] / o.counters[2] != pytest.approx(1.0, abs=0.05)
    for t in range(2):
        assert g_st["mean_beta"][t] == pytest.approx(o.counters[3 + t] / o.counters[2], rel=1e-3)


def test_multiplicity_cap_parity(mars, orc):
    """Teacher-forced MARS iteration with large count factors (splitting at the
    clamp) and a path multiplicity cap that binds: the capped budgets, the
    children's multiplicities and everything downstream agree with the oracle."""
    cfg = W.config_box(48, 40)
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=111, lo=2.0, hi=30.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=112, lo=0.02, hi=0.3)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
    import torch
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    g_st = cache.render_iteration(img, seed=6, iteration=2, mode=1, update_estimate=False, max_multiplicity=6.0)
    torch.cuda.synchronize()
    g_img = img.cpu().numpy().reshape(-1, 3).astype(np.float64)
    g_state = cache.get_state()
    okw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=2, seed=6,
               mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est, max_mult=6.0)
    o = orc.render(cfg.scene, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, cfg.scene,
                                      dict(iteration=2, seed=6, mode=1, max_multiplicity=6.0), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "box MARS, multiplicity cap", touch)
    free = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                      iteration=2, seed=6, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
    assert free.vertices > 2 * o.vertices   # the cap binds


def test_heightfield_triangles_parity(mars, orc):
    """Triangle geometry through the LBVH: a small seeded heightfield (12 x 12
    quads, 288 triangles) with spheres and the hidden emitter, warm-up and a
    teacher-forced MARS iteration with all three techniques."""
    sc = W.heightfield_scene(5, n=12, width=40, height=32, n_spheres=20)
    cfg = W.WorkloadConfig(sc, max_depth=5, grid_n=8, techniques=7, iterations=2, warmup=1, name="hf")
    scene, cache = _make(mars, cfg)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=0, seed=8, mode=0)
    g_state = cache.get_state()
    okw = dict(grid_n=8, techniques=7, max_depth=5, iteration=0, seed=8, collect=True)
    o = orc.render(sc, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, sc, dict(iteration=0, seed=8, mode=0), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "heightfield warm-up", touch)
    assert o.image.mean() > 0
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=121, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=122, lo=0.01, hi=0.5)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=123)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                    guide_cdf=cdf, stats=np.zeros((cfg.n_cells, 3, 8)))
    g_img, g_st = _gpu_iteration(mars, cache, iteration=1, seed=8, mode=1)
    g_state = cache.get_state()
    okw = dict(grid_n=8, techniques=7, max_depth=5, iteration=1, seed=8, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s,
               valid=valid, est=est, guide_cdf=cdf)
    o = orc.render(sc, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, sc, dict(iteration=1, seed=8, mode=1), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "heightfield MARS", touch)


def test_guided_room_crop_parity(mars, orc):
    """Three techniques (BSDF, NEE, guided) on a 64 x 64 render of the guided room
    with 16 spheres, GGX and Lambert, random guide CDFs and random counts."""
    sc = W.guided_room_scene(seed=0, width=64, height=64, n_spheres=16)
    cfg = W.WorkloadConfig(sc, max_depth=6, grid_n=8, techniques=7, iterations=1, warmup=0, name="guided crop")
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=201, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=202, lo=0.05, hi=2.0)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=203)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, guide_cdf=cdf, has_estimate=True,
                    n_iterations=2)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=2, seed=9, mode=1)
    g_state = cache.get_state()
    okw = dict(grid_n=cfg.grid_n, techniques=7, max_depth=cfg.max_depth, iteration=2, seed=9, mode=orc.MODE_MARS,
               q_rr=q_rr, q_s=q_s, valid=valid, est=est, guide_cdf=cdf)
    o = orc.render(sc, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, sc, dict(iteration=2, seed=9, mode=1), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "guided room", touch)
    gh, oh = g_state["guide_hist"].astype(np.float64), o.hist
    pop = (gh > 0) | (oh > 0)
    close = np.abs(gh - oh) <= STAT_TOL * np.abs(oh) + 1e-9
    assert (close & pop).sum() >= 0.99 * pop.sum()
    assert gh.sum() == pytest.approx(oh.sum(), rel=STAT_TOL)


def test_update_and_guide_parity(mars, orc):
    """Fixed-point update and guide CDF from the same synthetic statistics."""
    cfg = W.config_guided(16, 16)
    scene, cache = _make(mars, cfg)
    rng = np.random.default_rng(301)
    cells = cfg.n_cells
    stats = np.zeros((cells, 3, 8))
    n = rng.integers(0, 40, size=(cells, 3)).astype(float)
    stats[..., 0] = n
    m1 = rng.exponential(0.5, size=(cells, 3, 3))
    stats[..., 1:4] = n[..., None] * m1
    stats[..., 4:7] = n[..., None] * (m1 ** 2 + rng.exponential(0.3, size=(cells, 3, 3)))
    stats[..., 7] = n * rng.uniform(1.0, 6.0, size=(cells, 3))
    stats[rng.uniform(size=(cells, 3)) < 0.05, 7] = 0.0
    hist = rng.exponential(1.0, size=(cells, 256)).astype(np.float32)
    hist[rng.uniform(size=hist.shape) < 0.6] = 0.0
    hist[:7] = 0.0
    q_rr0, q_s0, valid0 = W.random_count_fields(cells, seed=302)
    VI, CI = 0.37, 4.25
    cache.set_state(q_rr=q_rr0, q_s=q_s0, valid=valid0, stats=stats, guide_hist=hist, VI=VI, CI=CI,
                    has_estimate=True, n_iterations=3)
    cache.update_counts()
    g = cache.get_state()
    q_rr, q_s, valid = orc.update_counts(stats, VI, CI, cfg.techniques, q_rr0, q_s0, valid0)
    assert np.array_equal(g["valid"], valid)
    np.testing.assert_allclose(g["q_rr"], q_rr, rtol=1e-6)
    np.testing.assert_allclose(g["q_s"], q_s, rtol=1e-6, atol=1e-30)
    assert np.all(g["stats"] == 0.0)
    cdf = orc.guide_update(hist.astype(np.float64))
    np.testing.assert_allclose(g["guide_cdf"], cdf, atol=2e-7)


def test_guide_update_edge_cases(mars, orc):
    """The guide CDF rebuild (float-float arithmetic on the GPU, float64 in the
    oracle) on histograms at the edges: empty, one bin, two bins 40 orders of
    magnitude apart, uniform, every bin tiny or huge, a geometric ramp over 256
    bins, and seeded random rows; every CDF value within 2e-7 of the oracle's,
    the last exactly 1."""
    cfg = W.config_guided(16, 16)
    scene, cache = _make(mars, cfg)
    cells = cfg.n_cells
    rng = np.random.default_rng(311)
    hist = rng.exponential(1.0, size=(cells, 256)).astype(np.float32)
    hist[rng.uniform(size=hist.shape) < 0.3] = 0.0
    hist[0] = 0.0
    hist[1] = 0.0
    hist[1, 17] = 3.0
    hist[2] = 0.0
    hist[2, 0], hist[2, 255] = 1e20, 1e-20
    hist[3] = 1.0
    hist[4] = 1e-20
    hist[5] = 1e20
    hist[6] = (1.07 ** np.arange(256)).astype(np.float32)
    hist[7] = 0.0
    hist[7, 255] = 5.0
    cache.set_state(guide_hist=hist, has_estimate=True, n_iterations=1)
    cache.update_counts()
    g = cache.get_state()
    cdf = orc.guide_update(hist.astype(np.float64))
    np.testing.assert_allclose(g["guide_cdf"], cdf, atol=2e-7, rtol=0)
    assert np.all(g["guide_cdf"][:, -1] == 1.0)
    assert np.all(np.diff(g["guide_cdf"], axis=1) >= 0.0)


def test_training_iteration_update_takes_the_mean_image_statistics(mars, orc):
    """A training iteration of three renders (Sec. 4.1 "Fixed-point iteration":
    the iterations grow in duration): the statistics of all three accumulate,
    the state reports the mean of their V_I and C_I over three image
    iterations, and the update equals the oracle's update of the accumulated
    statistics with those means; the next training iteration starts afresh."""
    cfg = W.config_box(32, 24)
    scene, cache = _make(mars, cfg)
    sts = [_gpu_iteration(mars, cache, iteration=k, seed=5, mode=0, update_estimate=True)[1] for k in range(3)]
    g = cache.get_state()
    vi = np.mean([s["VI"] for s in sts])
    ci = np.mean([s["CI"] for s in sts])
    assert g["image_iterations"] == 3
    assert g["VI"] == pytest.approx(vi, rel=1e-12) and g["CI"] == pytest.approx(ci, rel=1e-12)
    assert g["stats"][..., 0].sum() > 0
    cache.update_counts()
    u = cache.get_state()
    q_rr, q_s, valid = orc.update_counts(g["stats"], g["VI"], g["CI"], cfg.techniques, g["q_rr"], g["q_s"],
                                         g["valid"])
    assert np.array_equal(u["valid"], valid)
    np.testing.assert_allclose(u["q_rr"], q_rr, rtol=1e-6)
    np.testing.assert_allclose(u["q_s"], q_s, rtol=1e-6, atol=1e-30)
    assert u["image_iterations"] == 0 and u["VI"] == 0.0 and u["CI"] == 0.0
    # a checkpoint in the middle of a training iteration resumes it exactly
    st = _gpu_iteration(mars, cache, iteration=3, seed=5, mode=1, update_estimate=True)[1]
    _gpu_iteration(mars, cache, iteration=4, seed=5, mode=1, update_estimate=True)
    s = cache.get_state()
    assert s["image_iterations"] == 2
    other = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    other.set_state(VI=st["VI"], CI=st["CI"], image_iterations=1)
    assert other.get_state()["image_iterations"] == 1
    other.set_state(VI=s["VI"], CI=s["CI"], image_iterations=2)
    o = other.get_state()
    assert o["image_iterations"] == 2 and o["VI"] == pytest.approx(s["VI"], rel=1e-15)


def test_image_statistics_parity(mars, orc):
    """Running mean, pixel estimate and V_I after one rendered iteration, from a
    seeded running sum; the oracle uses its own image of the same iteration."""
    cfg = W.config_box(48, 40)
    scene, cache = _make(mars, cfg)
    rs = W.random_pixel_estimate(cfg.scene.n_pixels, seed=401, lo=0.1, hi=3.0) * 2.0
    cache.set_state(run_sum=rs, n_iterations=2, has_estimate=True,
                    pixel_estimate=np.ones((cfg.scene.n_pixels, 3), np.float32))
    g_img, g_st = _gpu_iteration(mars, cache, iteration=2, seed=3, mode=0, update_estimate=True)
    g = cache.get_state()
    o = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=2,
                   seed=3, est=np.ones((cfg.scene.n_pixels, 3), np.float32))
    vi, o_rs, o_est = orc.image_stats(48, 40, o.image, rs.astype(np.float64), 2)
    assert _pixel_agreement(g["run_sum"].astype(np.float64), o_rs) >= 0.999
    est_ok = np.abs(g["pixel_estimate"] - o_est) <= 1e-4 * np.abs(o_est) + 1e-7
    assert est_ok.all(axis=1).mean() >= 0.99
    assert g_st["VI"] == pytest.approx(vi, rel=1e-2)
    assert g_st["CI"] == pytest.approx(o.rays / cfg.scene.n_pixels, rel=1e-3)
    assert g["n_iterations"] == 3


def test_pixel_ranges_shard_the_frame(mars, orc):
    """The partitioning of a multi-GPU job (one pixel range per rank): two
    caches from the same state render the two halves of the frame (split at a
    pixel that is not warp-aligned); their pixels are bitwise those of the
    whole-frame render, their statistics, rays, vertices and budget sums add up
    to the whole frame's (up to the order of float64 sums), the image
    statistics of the assembled frame (the library's allocation-free image pass
    on caller buffers, with the summed rays) equal the whole-frame cache's, and
    the fixed-point update on the summed statistics equals the update on the
    whole.  Argument errors: an empty or out-of-frame range, or a range with
    update_estimate."""
    import torch
    cfg = W.WorkloadConfig(W.guided_room_scene(seed=2, width=64, height=48, n_spheres=24), max_depth=6, grid_n=8,
                           techniques=7, iterations=1, warmup=0, name="guided 64x48")
    npx = cfg.scene.n_pixels
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=501, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(npx, seed=502, lo=0.05, hi=2.0)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=503)
    rs = W.random_pixel_estimate(npx, seed=504, lo=0.1, hi=3.0) * 2.0
    state = dict(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, guide_cdf=cdf, run_sum=rs,
                 has_estimate=True, n_iterations=2)
    scene = mars.Scene(cfg.scene)
    caches = [mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth) for _ in range(3)]
    for c in caches:
        c.set_state(**state)
    kw = dict(seed=13, iteration=4, mode=mars.MARS_MODE_MARS)
    full = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    st_full = caches[0].render_iteration(full, update_estimate=True, **kw)
    split = 1337
    part = torch.full((npx * 3,), -1.0, dtype=torch.float32, device="cuda")
    st_a = caches[1].render_iteration(part, update_estimate=False, px_range=(0, split), **kw)
    st_b = caches[2].render_iteration(part, update_estimate=False, px_range=(split, npx), **kw)
    torch.cuda.synchronize()
    assert torch.equal(part, full)
    g_full, g_a, g_b = (c.get_state() for c in caches)
    assert st_a["rays"] + st_b["rays"] == st_full["rays"]
    assert st_a["vertices"] + st_b["vertices"] == st_full["vertices"]
    assert st_a["estimator_vertices"] + st_b["estimator_vertices"] == st_full["estimator_vertices"]
    for t in range(3):
        sb = st_a["mean_beta"][t] * st_a["estimator_vertices"] + st_b["mean_beta"][t] * st_b["estimator_vertices"]
        assert sb == pytest.approx(st_full["mean_beta"][t] * st_full["estimator_vertices"], rel=1e-9)
    summed = g_a["stats"] + g_b["stats"]
    np.testing.assert_allclose(summed, g_full["stats"], rtol=1e-6, atol=1e-9)
    assert np.array_equal(summed[..., 0], g_full["stats"][..., 0])
    assert np.array_equal(summed[..., 7], g_full["stats"][..., 7])
    np.testing.assert_allclose(g_a["guide_hist"].astype(np.float64) + g_b["guide_hist"],
                               g_full["guide_hist"], rtol=1e-4, atol=1e-6)
    # the oracle over the same two ranges agrees with the shards' sum
    okw = dict(grid_n=cfg.grid_n, techniques=7, max_depth=cfg.max_depth, iteration=4, seed=13, mode=orc.MODE_MARS,
               q_rr=q_rr, q_s=q_s, valid=valid, est=est, guide_cdf=cdf)
    o = [orc.render(cfg.scene, px_begin=b, px_end=e, **okw) for b, e in ((0, split), (split, npx))]
    assert np.allclose(summed.sum(0), (o[0].stats + o[1].stats).sum(0), rtol=STAT_TOL, atol=1e-6)
    # image statistics of the assembled frame on caller buffers, rays summed over the shards
    L = mars.load()
    run_sum = torch.tensor(rs.reshape(-1), dtype=torch.float32, device="cuda")
    est_out = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    vi_ci = torch.zeros(2, dtype=torch.float64, device="cuda")
    rc = L.mars_image_stats_static(part.data_ptr(), run_sum.data_ptr(), est_out.data_ptr(), 64, 48, 2, 50.0,
                                   float(st_a["rays"] + st_b["rays"]), vi_ci.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    VI, CI = vi_ci.cpu().tolist()
    assert VI == pytest.approx(st_full["VI"], rel=1e-6) and CI == pytest.approx(st_full["CI"], rel=1e-12)
    np.testing.assert_allclose(est_out.cpu().numpy().reshape(-1, 3), g_full["pixel_estimate"], rtol=1e-6)
    # the update on the summed statistics equals the update on the whole
    caches[1].set_state(stats=summed, VI=VI, CI=CI, has_estimate=True, n_iterations=3)
    caches[0].update_counts()
    caches[1].update_counts()
    u_full, u_sum = caches[0].get_state(), caches[1].get_state()
    assert np.array_equal(u_full["valid"], u_sum["valid"])
    np.testing.assert_allclose(u_sum["q_rr"], u_full["q_rr"], rtol=1e-5)
    # q^S = sqrt(var) amplifies the regrouped float32 partial sums by m2 / var
    # where the variance is small against the second moment
    close = np.abs(u_sum["q_s"] - u_full["q_s"]) <= 1e-4 * np.abs(u_full["q_s"]) + 1e-12
    assert close.mean() >= 0.999
    np.testing.assert_allclose(u_sum["q_s"], u_full["q_s"], rtol=1e-2, atol=1e-9)
    # argument errors
    for bad in ((0, 0 - 1), (5, 5), (0, npx + 1), (-3, 10)):
        with pytest.raises(mars.MarsError) as e:
            caches[2].render_iteration(part, update_estimate=False, px_range=bad, **kw)
        assert e.value.status == mars.MARS_ERR_INVALID_ARG
    with pytest.raises(mars.MarsError) as e:
        caches[2].render_iteration(part, update_estimate=True, px_range=(0, 10), **kw)
    assert e.value.status == mars.MARS_ERR_INVALID_ARG


def test_arena_overflow_tiles_reproduce_the_image(mars):
    """A small queue arena forces pixel tiles; the image is bitwise identical and
    the statistics equal up to summation order (runs of equal cells are summed
    in float32 within a warp before the float64 atomics, and tiling changes
    which vertices share a warp)."""
    cfg = W.config_box(32, 32)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=501, lo=0.5, hi=6.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=502, lo=0.05, hi=0.5)
    res = []
    for cap in (0, 6000):
        scene, cache = _make(mars, cfg, arena_capacity=cap)
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
        img, st = _gpu_iteration(mars, cache, iteration=1, seed=2, mode=1)
        res.append((img, st, cache.get_state()["stats"]))
    (a, sa, ta), (b, sb, tb) = res
    assert sa["retries"] == 0 and sb["retries"] > 0 and sb["tiles"] > 1
    assert np.array_equal(a, b)
    np.testing.assert_allclose(ta, tb, rtol=1e-6, atol=1e-9)
    assert sa["rays"] == sb["rays"] and sa["vertices"] == sb["vertices"]


def test_launch_shape_does_not_change_results(mars):
    """Every wave kernel strides over its wave in chunks of 32 slots, so threads
    per block and grid size change the speed only: the image is bitwise equal
    and the statistics equal up to the order of the float64 atomics.  The
    autotuner leaves the learned state untouched."""
    cfg = W.config_guided(48, 40)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=601, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=602, lo=0.05, hi=0.5)
    scene, cache = _make(mars, cfg)
    base = cache.get_launch()
    assert base["threads"] == [128, 128, 128, 128] and min(base["blocks_per_sm"]) >= 1
    assert base["max_registers"] == [0, 0, 0, 0]
    res = []
    for threads, bps, regs in (([128] * 4, [0] * 4, [0] * 4), ([64, 256, 32, 256], [3, 1, 7, 2], [40, 80, 0, 64]),
                               ([256, 64, 256, 64], [9, 5, 1, 4], [0, 64, 40, 80])):
        cache.set_launch(threads, bps, regs)
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                        stats=np.zeros((cfg.n_cells, 3, 8)))
        img, st = _gpu_iteration(mars, cache, iteration=1, seed=4, mode=1)
        res.append((img, st, cache.get_state()["stats"]))
    for img, st, stats in res[1:]:
        assert np.array_equal(img, res[0][0])
        assert st["rays"] == res[0][1]["rays"] and st["vertices"] == res[0][1]["vertices"]
        np.testing.assert_allclose(stats, res[0][2], rtol=1e-6, atol=1e-9)
    before = cache.get_state()
    chosen = cache.autotune(iteration=1, seed=4, mode=1, repeats=1)
    assert all(t in (64, 128, 256) for t in chosen["threads"]) and min(chosen["blocks_per_sm"]) >= 1
    after = cache.get_state()
    for k in ("q_rr", "q_s", "valid", "stats", "run_sum", "pixel_estimate", "guide_cdf", "guide_hist"):
        assert np.array_equal(before[k], after[k]), k
    img, st = _gpu_iteration(mars, cache, iteration=1, seed=4, mode=1)
    assert np.array_equal(img, res[0][0])
    with pytest.raises(mars.MarsError):
        cache.set_launch([100, 128, 128, 128], [0] * 4)
    with pytest.raises(mars.MarsError):
        cache.set_launch([128] * 4, [0] * 4, [0, 0, 0, 48])


@pytest.mark.parametrize("albedo,D", [(0.5, 3), (0.8, 5)])
def test_gpu_furnace_closed_form(mars, albedo, D):
    """The CUDA path alone against the closed furnace Le (1 - a^D) / (1 - a)
    under a random count field (unbiasedness, App. A.1)."""
    sc = W.furnace_scene(albedo=albedo, radiance=1.5, width=64, height=64)
    cfg = W.WorkloadConfig(sc, max_depth=D, grid_n=4, techniques=3, iterations=1, warmup=0, name="furnace")
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=601, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=602, lo=0.5, hi=4.0)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
    means = []
    for it in range(40):
        img, _ = _gpu_iteration(mars, cache, iteration=it, seed=1, mode=1, collect=False)
        means.append(img.mean())
    m, se = np.mean(means), np.std(means, ddof=1) / math.sqrt(len(means))
    expected = 1.5 * (1 - albedo ** D) / (1 - albedo)
    assert abs(m - expected) < 3.5 * se


def test_state_roundtrip(mars):
    cfg = W.config_guided(8, 8)
    scene, cache = _make(mars, cfg)
    rng = np.random.default_rng(701)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=702)
    stats = rng.normal(size=(cfg.n_cells, 3, 8))
    hist = rng.exponential(size=(cfg.n_cells, 256)).astype(np.float32)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=703)
    est = W.random_pixel_estimate(64, seed=704)
    rs = W.random_pixel_estimate(64, seed=705)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, stats=stats, guide_hist=hist, guide_cdf=cdf,
                    pixel_estimate=est, run_sum=rs, n_iterations=5, has_estimate=True, VI=0.5, CI=3.0)
    g = cache.get_state()
    for k, v in dict(q_rr=q_rr, q_s=q_s, valid=valid, stats=stats, guide_hist=hist, guide_cdf=cdf,
                     pixel_estimate=est, run_sum=rs).items():
        assert np.array_equal(g[k], v), k
    assert g["n_iterations"] == 5 and g["has_estimate"] and g["VI"] == 0.5 and g["CI"] == 3.0


def test_invalid_arguments_are_reported(mars):
    from paper_2410_20429_gb300 import _abi as A
    cfg = W.config_box(8, 8)
    scene = mars.Scene(cfg.scene)
    with pytest.raises(mars.MarsError) as e:
        mars.Cache(scene, 0, 3, 5)
    assert e.value.status == A.MARS_ERR_INVALID_ARG
    with pytest.raises(mars.MarsError):
        mars.Cache(scene, 4, 2, 5)        # BSDF missing
    cache = mars.Cache(scene, 4, 3, 5)
    import torch
    img = torch.zeros(8 * 8 * 3, device="cuda")
    with pytest.raises(mars.MarsError) as e:
        cache.render_iteration(img, mode=A.MARS_MODE_MARS)   # no pixel estimate yet
    assert "pixel estimate" in str(e.value)
    with pytest.raises(mars.MarsError):
        cache.render_iteration(img, clamp_hi=40.0)
    bad = W.box_scene(4, 4)
    bad.quad_mat = bad.quad_mat.copy()
    bad.quad_mat[0] = 99
    with pytest.raises(mars.MarsError):
        mars.Scene(bad)
    # the cache still works after rejected calls
    cache.render_iteration(img)


@pytest.mark.parametrize("octree", [False, True])
def test_checkpoint_resume_continues_the_run(mars, octree):
    """Checkpoint / resume: the state of a run after a few fixed-point
    iterations, copied into a fresh cache, continues exactly as the original:
    the next iteration's image is bitwise equal (same counts, estimate, guide,
    tree and random numbers); the one after agrees within the pixel bar (the
    statistics of the resumed iteration are summed in another atomic order)."""
    import torch
    cfg = W.config_guided(48, 40)
    scene = mars.Scene(cfg.scene)
    kw = dict(octree=True, max_leaves=4096, split_samples=30.0) if octree else {}
    a = mars.Cache(scene, 8, cfg.techniques, 6, **kw)
    img = torch.zeros(a.n_pixels * 3, dtype=torch.float32, device="cuda")
    for it in range(4):
        a.render_iteration(img, seed=21, iteration=it, mode=0 if it < 2 else 1, update_estimate=True)
        a.update_counts()
    s = a.get_state()
    if octree:
        assert s["oct_n_leaves"] > 512
    b = mars.Cache(scene, 8, cfg.techniques, 6, **kw)
    extra = dict(oct_nodes=s["oct_nodes"], oct_leaf_level=s["oct_leaf_level"]) if octree else {}
    b.set_state(q_rr=s["q_rr"], q_s=s["q_s"], valid=s["valid"], stats=s["stats"], guide_hist=s["guide_hist"],
                guide_cdf=s["guide_cdf"], pixel_estimate=s["pixel_estimate"], run_sum=s["run_sum"],
                n_iterations=s["n_iterations"], has_estimate=s["has_estimate"], VI=s["VI"], CI=s["CI"], **extra)
    outs = []
    for c in (a, b):
        imgs = []
        for it in (4, 5):
            c.render_iteration(img, seed=21, iteration=it, mode=1, update_estimate=True)
            c.update_counts()
            torch.cuda.synchronize()
            imgs.append(img.cpu().numpy().reshape(-1, 3).astype(np.float64))
        outs.append(imgs)
    assert np.array_equal(outs[0][0], outs[1][0])
    assert _pixel_agreement(outs[1][1], outs[0][1]) >= 0.999


@pytest.mark.parametrize("which", ["box", "guided_room"])
def test_relmse_against_a_long_reference_matches_the_oracle(mars, orc, which):
    """Third agreement criterion: the relMSE of the CUDA path's N-iteration
    image and of the oracle's (same random numbers, same teacher-forced counts
    and, for the guided room, guide) against a 65536-samples-per-pixel reference
    agree within 2 % of the oracle's.  The references are the oracle's own
    fixed-count renders at 32 x 32 with other random numbers, stored by
    tests/golden/make_box_reference.py: the box, and the guided room's geometry
    with all three techniques."""
    import os
    name = "box_32x32_fixed_65536spp.txt" if which == "box" else "guided_room_32x32_fixed_65536spp.txt"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    ref = np.loadtxt(path)[:, :3]
    cfg = W.config_box(32, 32) if which == "box" else W.config_guided(32, 32)
    scene, cache = _make(mars, cfg)
    npx = cfg.scene.n_pixels
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=141, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(npx, seed=142, lo=0.05, hi=0.5)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=143) if cfg.techniques & W.TECH_GUIDED else None
    extra = {} if cdf is None else {"guide_cdf": cdf}
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                    **extra)
    g_acc = np.zeros((npx, 3))
    o_acc = np.zeros((npx, 3))
    N = 16
    for k in range(N):
        g, _ = _gpu_iteration(mars, cache, iteration=10 + k, seed=5, mode=1, collect=False)
        o = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                       iteration=10 + k, seed=5, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                       collect=False, guide_cdf=cdf)
        g_acc += g
        o_acc += o.image

    def rel_mse(x):
        t = ((x - ref) ** 2 / (ref ** 2 + 1e-2)).mean(axis=1)
        k = int(np.ceil(1e-4 * t.size))
        return np.sort(t)[:-k].mean() if k else t.mean()

    rg, ro = rel_mse(g_acc / N), rel_mse(o_acc / N)
    assert ro > 0 and abs(rg - ro) <= 0.02 * ro, (rg, ro)


def test_graph_replay_equals_direct_launches(mars):
    """On a capturable stream an iteration that fits one pixel tile is recorded
    once as a CUDA graph and replayed; its per-iteration arguments (seed,
    iteration, mode, running-image count, ...) are read from device memory, so
    a replay renders the next iteration, not the recorded one.  From the same
    state, replayed and directly launched iterations give bitwise equal images
    and counters and statistics equal up to the order of the float64 atomics,
    across modes, seeds, a launch-shape change, a new output buffer, the
    update_estimate flag and a profiled iteration; a graph is recorded again
    only when one of those changes."""
    import torch
    cfg = W.config_guided(48, 40)
    stream = torch.cuda.Stream()   # torch's streams can be captured; the legacy default stream cannot
    scene = mars.Scene(cfg.scene, stream=stream)
    caches = [mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, graphs=g, stream=stream)
              for g in (True, False)]
    bufs = [torch.zeros(caches[0].n_pixels * 3, dtype=torch.float32, device="cuda") for _ in range(2)]
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=701, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=702, lo=0.05, hi=0.5)
    run = W.random_pixel_estimate(cfg.scene.n_pixels, seed=703, lo=0.05, hi=0.5)
    for it in range(8):
        res = []
        for c in caches:
            if it == 3:
                c.set_launch([64, 128, 64, 128], [0, 0, 0, 0], [0, 64, 0, 80])
            c.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, run_sum=run * (it + 1),
                        has_estimate=True, n_iterations=it + 1, stats=np.zeros((cfg.n_cells, 3, 8)),
                        stream=stream)
            img = bufs[1 if it >= 5 else 0]
            st = c.render_iteration(img, seed=31 + it, iteration=it, mode=0 if it < 2 else 1,
                                    update_estimate=(it % 3 != 2), profile=(it == 6), stream=stream)
            g = c.get_state(stream=stream)
            torch.cuda.synchronize()
            res.append((img.cpu().numpy().copy(), st, g))
        (a, sa, ga), (b, sb, gb) = res
        assert np.array_equal(a, b), f"iteration {it}: images differ"
        assert sa["rays"] == sb["rays"] and sa["vertices"] == sb["vertices"], it
        np.testing.assert_allclose(ga["stats"], gb["stats"], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(ga["run_sum"], gb["run_sum"], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(ga["pixel_estimate"], gb["pixel_estimate"], rtol=1e-6, atol=1e-9)
        assert sa["VI"] == pytest.approx(sb["VI"], rel=1e-6) and sa["CI"] == pytest.approx(sb["CI"], rel=1e-9)
    caps = caches[0].info()["graph_captures"]
    # recorded at least for the first iteration, the new launch shape, the new
    # buffer and the update_estimate changes; never for the profiled iteration
    assert 3 <= caps <= 7, caps
    assert caches[1].info()["graph_captures"] == 0


def test_graph_replay_with_arena_overflow(mars):
    """A recorded single-tile iteration whose path trees overflow the arena is
    re-rendered in tiles by direct launches; the image equals that of a cache
    whose arena holds the whole iteration."""
    import torch
    cfg = W.config_box(32, 32)
    stream = torch.cuda.Stream()
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=501, lo=0.5, hi=6.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=502, lo=0.05, hi=0.5)
    res = []
    for cap in (0, 6000):
        scene = mars.Scene(cfg.scene, stream=stream)
        cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, arena_capacity=cap, stream=stream)
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                        stream=stream)
        img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
        st = cache.render_iteration(img, seed=2, iteration=1, mode=1, update_estimate=False, stream=stream)
        stream.synchronize()
        res.append((img.cpu().numpy().copy(), st, cache.info()["graph_captures"]))
    (a, sa, ca), (b, sb, cb) = res
    assert sa["retries"] == 0 and sb["retries"] > 0 and sb["tiles"] > 1
    assert ca == 1 and cb == 1
    assert np.array_equal(a, b)
    assert sa["rays"] == sb["rays"] and sa["vertices"] == sb["vertices"]


@pytest.mark.parametrize("which", ["guided", "heightfield"])
def test_bvh_kind_does_not_change_results(mars, which):
    """The SAH hierarchy (built on the host) and the linear BVH (built on the
    device) hold the same primitives; closest hits break ties in t by the lower
    primitive index, so the image is bitwise equal whichever is traversed and
    only the traversal work differs."""
    import dataclasses
    cfg = W.config_guided(48, 40) if which == "guided" else W.config_heightfield(48, 40)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=801, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=802, lo=0.05, hi=0.5)
    res = []
    for kind in (mars.MARS_BVH_SAH, mars.MARS_BVH_LBVH):
        sc = dataclasses.replace(cfg.scene)
        sc.bvh = kind
        scene = mars.Scene(sc)
        cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
        img, st = _gpu_iteration(mars, cache, iteration=1, seed=9, mode=1)
        res.append((img, st, cache.get_state()["stats"]))
    (a, sa, ta), (b, sb, tb) = res
    assert np.array_equal(a, b)
    assert sa["rays"] == sb["rays"] and sa["vertices"] == sb["vertices"]
    np.testing.assert_allclose(ta, tb, rtol=1e-6, atol=1e-9)
    assert sa["trace_work"][0][0] > 0 and sb["trace_work"][0][0] > 0


@pytest.mark.parametrize("capturable,pinned", [(False, False), (True, False), (False, True), (True, True)])
def test_host_image_equals_device_image(mars, capturable, pinned):
    """An image requested in host memory (page-locked: written by the image pass
    through its device address; pageable: packed on the device and copied back
    once) equals the image written to device memory from the same state, with
    and without the image statistics pass, on the legacy default stream and on a
    stream whose iterations replay a recorded graph."""
    import torch
    cfg = W.config_guided(40, 24)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=901, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=902, lo=0.05, hi=0.5)
    stream = torch.cuda.Stream() if capturable else None
    scene = mars.Scene(cfg.scene, stream=stream)
    cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream)
    dev = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    host = (torch.zeros(cache.n_pixels * 3, dtype=torch.float32, pin_memory=True).numpy() if pinned
            else np.zeros(cache.n_pixels * 3, np.float32))
    for it, upd in ((1, True), (2, False), (3, True)):
        outs = []
        for target in (dev, host):
            cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True,
                            n_iterations=1, stream=stream)
            st = cache.render_iteration(target, seed=5, iteration=it, mode=1, update_estimate=upd, stream=stream)
            torch.cuda.synchronize()
            outs.append((dev.cpu().numpy().copy() if target is dev else host.copy(), st["vertices"]))
        assert np.array_equal(outs[0][0], outs[1][0]), (it, upd)
        assert outs[0][1] == outs[1][1]
        assert np.isfinite(outs[1][0]).all() and outs[1][0].max() > 0


@pytest.mark.parametrize("K", [1, 10, 16])
def test_brightest_pixel_rejection_parity(mars, orc, K):
    """V_I without its K brightest pixels (Sec. 5.1): the GPU's value against the
    oracle's on the GPU's own image of the iteration (same running sum); the K
    pixels are chosen by float32 luminance on both sides, so the choice is the
    same, and the remaining sums agree to float32 rounding."""
    cfg = W.config_guided(48, 40)
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=951, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=952, lo=0.05, hi=0.5)
    rs = W.random_pixel_estimate(cfg.scene.n_pixels, seed=953, lo=0.1, hi=3.0) * 2.0
    res = {}
    for k in (0, K):
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, run_sum=rs, has_estimate=True,
                        n_iterations=2, stats=np.zeros((cfg.n_cells, 3, 8)))
        import torch
        img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
        st = cache.render_iteration(img, seed=7, iteration=2, mode=1, update_estimate=True, vi_drop_brightest=k)
        torch.cuda.synchronize()
        res[k] = (img.cpu().numpy().reshape(-1, 3).astype(np.float64), st)
    a, b = res[0], res[K]
    assert np.array_equal(a[0], b[0])   # the rejection changes V_I only
    vi0, _, _ = orc.image_stats(48, 40, a[0], rs.astype(np.float64), 2, outlier=50.0, drop_k=0)
    viK, _, _ = orc.image_stats(48, 40, a[0], rs.astype(np.float64), 2, outlier=50.0, drop_k=K)
    assert a[1]["VI"] == pytest.approx(vi0, rel=1e-4)
    assert b[1]["VI"] == pytest.approx(viK, rel=1e-4)
    assert b[1]["CI"] == a[1]["CI"]
    with pytest.raises(mars.MarsError):
        cache.render_iteration(None, iteration=3, update_estimate=True, vi_drop_brightest=17)


def test_inverse_variance_combination_parity(mars, orc):
    """Progressive combination (Sec. 5.1): after iterations rendered with
    combine = 2 (restart) and then 1, the library's combined image and weight
    sum equal the oracle's combination of the per-iteration images with weights
    1 / V_I; an iteration with combine = 0 stays out; replayed graphs on a
    capturable stream carry the flag."""
    import torch
    cfg = W.config_guided(40, 32)
    stream = torch.cuda.Stream()
    scene = mars.Scene(cfg.scene, stream=stream)
    cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, stream=stream)
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    imgs, vis = [], []
    for it in range(7):
        comb = 2 if it == 1 else (0 if it in (0, 4) else 1)
        st = cache.render_iteration(img, seed=3, iteration=it, mode=0 if it < 2 else 1, update_estimate=True,
                                    combine=comb, vi_drop_brightest=10 if it >= 3 else 0, stream=stream)
        cache.update_counts(stream=stream)
        stream.synchronize()
        if comb:
            imgs.append(img.cpu().numpy().reshape(-1, 3).astype(np.float64))
            vis.append(st["VI"])
    g_img, g_w = cache.combined_image(stream=stream)
    o_img, o_w = orc.combine(imgs, vis)
    assert g_w == pytest.approx(o_w, rel=1e-6)
    np.testing.assert_allclose(g_img.reshape(-1, 3), o_img, rtol=1e-5, atol=1e-7)
    with pytest.raises(mars.MarsError):
        cache.render_iteration(img, iteration=9, update_estimate=False, combine=1, stream=stream)


@pytest.mark.parametrize("capturable", [False, True])
def test_two_lanes_equal_one_lane(mars, capturable):
    """Pixel tiles dealt to two concurrent lanes (own streams, counters and half
    of the arena each) give the image of one lane bitwise, the same counters and
    the statistics up to the order of the float64 atomics; also when the half
    arenas overflow and tiles are re-rendered."""
    import torch
    cfg = W.config_guided(384, 384)   # two lanes start at 2^17 pixels
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=981, lo=0.3, hi=1.5)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=982, lo=0.05, hi=0.5)
    stream = torch.cuda.Stream() if capturable else None
    scene = mars.Scene(cfg.scene, stream=stream)
    for cap in (0, 400000):
        res = []
        for lanes in (1, 2):
            cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, arena_capacity=cap, lanes=lanes,
                               stream=stream)
            img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
            out = []
            for it in (1, 2):
                cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True,
                                n_iterations=1, stats=np.zeros((cfg.n_cells, 3, 8)), stream=stream)
                st = cache.render_iteration(img, seed=13, iteration=it, mode=1, update_estimate=True, stream=stream)
                g = cache.get_state(stream=stream)
                torch.cuda.synchronize()
                out.append((img.cpu().numpy().copy(), st, g))
            res.append(out)
            cache.close()
        for (a, sa, ga), (b, sb, gb) in zip(res[0], res[1]):
            assert np.array_equal(a, b), cap
            for k in ("rays", "vertices", "estimator_vertices", "wave_entries", "shadow_entries", "shadow_traced"):
                assert sa[k] == sb[k], (cap, k)
            np.testing.assert_allclose(ga["stats"], gb["stats"], rtol=1e-6, atol=1e-9)
            assert sa["VI"] == pytest.approx(sb["VI"], rel=1e-9)
            assert sb["tiles"] >= 2
        if cap:
            assert any(s["retries"] > 0 for _, s, _ in res[1])
        else:
            # the first iteration (no history) of the two-lane cache renders
            # one tile per lane; the one-lane cache one tile
            assert res[0][0][1]["tiles"] == 1 and res[1][0][1]["tiles"] == 2 and res[1][0][1]["retries"] == 0


@pytest.mark.parametrize("techniques,D", [(1, 1), (1, 2), (1, 4), (5, 2), (5, 4), (3, 1), (3, 2), (7, 2)])
def test_technique_sets_and_shallow_depths_parity(mars, orc, techniques, D):
    """Technique subsets (BSDF alone, BSDF + guided without NEE) and the
    shallowest depths (D = 1: camera rays only, no estimator vertex; D = 2: one
    estimator level) against the oracle, on a 32 x 24 crop of the guided room
    with random counts and guide distributions, warm-up and MARS iterations."""
    sc = W.guided_room_scene(seed=2, width=32, height=24, n_spheres=12)
    cfg = W.WorkloadConfig(sc, max_depth=D, grid_n=8, techniques=techniques, iterations=1, warmup=0, name="subset")
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=301 + D, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=302, lo=0.05, hi=2.0)
    cdf = W.random_guide_cdf(cfg.n_cells, seed=303)
    for mode in (0, 1):
        kw = dict(guide_cdf=cdf) if techniques & W.TECH_GUIDED else {}
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=2,
                        stats=np.zeros((cfg.n_cells, 3, 8)), **kw)
        g_img, g_st = _gpu_iteration(mars, cache, iteration=2, seed=11, mode=mode)
        g_state = cache.get_state()
        o = orc.render(sc, grid_n=cfg.grid_n, techniques=techniques, max_depth=D, iteration=2, seed=11, mode=mode,
                       q_rr=q_rr, q_s=q_s, valid=valid, est=est, **kw)
        _check(g_img, o.image, g_state, o, g_st, f"techniques {techniques}, D {D}, mode {mode}")


def _single_quad_scene(width, height):
    """One emitting Lambertian quad facing the camera, partly filling the view:
    a one-primitive hierarchy, rays that miss, and NEE samples that can never
    reach the only light (it lies in the plane of every vertex)."""
    return W.scenes._mk([[0, 0, 1, 0, 1, 0, 1, 0, 0]], [0], [], [],
                        [W.scenes._lambert(0.5, 0.4, 0.3, (2.0, 1.5, 1.0))],
                        [0.5, 0.5, -1.4, 0.5, 0.5, 0.0, 0.0, 1.0, 0.0, 40.0], width, height, "single_quad")


@pytest.mark.parametrize("case", ["one_pixel", "prime_size", "single_quad_sah", "single_quad_lbvh", "all_miss"])
def test_degenerate_inputs_parity(mars, orc, case):
    """Edge cases of the path against the oracle: a 1 x 1 image; a 37 x 29
    image (1073 pixels: every wave ends in a partial warp and block); a scene of
    one primitive under both hierarchy builders; a camera that sees nothing
    (every wave after the first is empty).  A warm-up iteration and a
    teacher-forced MARS iteration each, then the image statistics."""
    import dataclasses
    cfg = W.config_box(37, 29)
    if case == "one_pixel":
        cfg = W.config_box(1, 1)
    elif case.startswith("single_quad"):
        cfg = dataclasses.replace(cfg, scene=_single_quad_scene(37, 29), max_depth=3)
        cfg.scene.bvh = mars.MARS_BVH_SAH if case.endswith("sah") else mars.MARS_BVH_LBVH
    elif case == "all_miss":
        sc = dataclasses.replace(cfg.scene)
        sc.camera = np.array([0.5, 0.5, -1.4, 0.5, 0.5, -3.0, 0.0, 1.0, 0.0, 40.0], np.float32)
        cfg = dataclasses.replace(cfg, scene=sc)
    n = cfg.scene.n_pixels
    kw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth)
    scene, cache = _make(mars, cfg)

    g_img, g_st = _gpu_iteration(mars, cache, iteration=0, seed=2, mode=0)
    o = orc.render(cfg.scene, iteration=0, seed=2, **kw)
    _check(g_img, o.image, cache.get_state(), o, g_st, f"{case} warm-up")

    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=901, lo=0.05, hi=4.0)
    est = W.random_pixel_estimate(n, seed=902, lo=0.05, hi=1.0)
    # statistics accumulate until the count update: start the MARS iteration from none
    zero = np.zeros_like(cache.get_state()["stats"])
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                    stats=zero)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=1, seed=2, mode=1)
    o = orc.render(cfg.scene, iteration=1, seed=2, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est, **kw)
    _check(g_img, o.image, cache.get_state(), o, g_st, f"{case} MARS")
    if case == "all_miss":
        assert not g_img.any() and g_st["rays"] == n and g_st["estimator_vertices"] == 0

    # image statistics of a fresh warm-up iteration from a seeded running sum
    rs = W.random_pixel_estimate(n, seed=903, lo=0.1, hi=3.0) * 2.0
    ones = np.ones((n, 3), np.float32)
    cache.set_state(run_sum=rs, n_iterations=2, has_estimate=True, pixel_estimate=ones)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=2, seed=2, mode=0, update_estimate=True)
    g = cache.get_state()
    o = orc.render(cfg.scene, iteration=2, seed=2, est=ones, **kw)
    vi, o_rs, o_est = orc.image_stats(cfg.scene.width, cfg.scene.height, o.image, rs.astype(np.float64), 2)
    assert _pixel_agreement(g["run_sum"].astype(np.float64), o_rs) >= 0.999
    est_ok = np.abs(g["pixel_estimate"] - o_est) <= 1e-4 * np.abs(o_est) + 1e-7
    assert est_ok.all(axis=1).mean() >= 0.99
    assert g_st["VI"] == pytest.approx(vi, rel=1e-2)
    assert g_st["CI"] == pytest.approx(o.rays / n, rel=1e-3)


NUDGE_ULPS = 4   # float32 evaluation carries errors of a few ulps of its inputs


def _nudge32(v, direction, ulps=NUDGE_ULPS):
    to = np.float32(np.inf) if direction > 0 else np.float32(-np.inf)
    x = np.asarray(v, np.float32)
    for _ in range(ulps):
        x = np.nextafter(x, to)
    return x


def _nudged(scene, direction):
    """The scene with every geometry and camera value moved by NUDGE_ULPS
    float32 ulps (the camera's origin and look-at point move every primary ray,
    and so every hit point, by ulps of the scene's coordinates -- the size of
    the float32 error of a hit point far from the camera)"""
    import dataclasses
    out = dataclasses.replace(scene)
    for f in ("quads", "spheres", "tris", "camera"):
        v = getattr(scene, f)
        if len(v):
            nv = _nudge32(v, direction).astype(np.float64)
            if f == "camera":
                nv[6:] = v[6:]   # up vector and field of view unchanged
            setattr(out, f, nv)
    return out


FULL_RUNS, FULL_RUN_LEN = 64, 64   # 4096 sampled pixels per workload


def _full_size_inputs(which):
    """Seeded inputs of the full-size parity case, built the same way in the
    test process and in the oracle's worker processes: the workload, its
    teacher-forced counts, pixel estimate and guide, and for the heightfields an
    adaptive octree refined by the oracle's own rule from seeded per-leaf sample
    counts (three rounds, split at 100 samples, at most 64k leaves)."""
    import oracle
    if which == "guided_512":
        cfg = W.config_guided(512, 512)
        cells, tree = cfg.n_cells, None
    else:
        cfg = {"heightfield_1024": W.config_heightfield, "large_2048": W.config_large,
               "bdpt_heightfield_1024": W.config_bdpt_heightfield,
               "bdpt_large_2048": W.config_bdpt_large}[which]()
        cells = 65536
        nodes, nn, nl, lvl, lnode = oracle.octree_init(cfg.grid_n, cells)
        rng = np.random.default_rng(1004)
        z = np.zeros((cells, 3, 3), np.float32)
        zv = np.zeros((cells, 3), np.uint8)
        for _ in range(3):
            st = np.zeros((cells, 3, 8))
            st[:nl, 0, 0] = rng.integers(0, 160, size=nl)
            nodes, nn, nl, lvl, lnode, *_ = oracle.octree_refine(cells, 100.0, st, nodes, nn, nl, lvl, lnode,
                                                                 z, z, zv)
        tree = (nodes[:nn].copy(), lvl[:nl].copy(), nl)
    q_rr, q_s, valid = W.random_count_fields(cells, seed=1001, lo=0.1, hi=2.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=1002, lo=0.2, hi=2.0)
    cdf = W.random_guide_cdf(cells, seed=1003) if cfg.techniques & 4 else None
    return cfg, cells, tree, q_rr, q_s, valid, est, cdf


def _full_size_runs(npx):
    stride = npx // FULL_RUNS
    return [r * stride + (r * 7919) % max(1, stride - FULL_RUN_LEN) for r in range(FULL_RUNS)]


def _full_size_oracle(job):
    """Worker (a spawned process): the oracle over some runs of pixels of the
    full-size case, on the scene nudged by `nudge` float32 ulps; returns the
    runs' pixels and statistics and, unnudged, their summed counters."""
    which, nudge, starts = job
    import oracle
    cfg, cells, tree, q_rr, q_s, valid, est, cdf = _full_size_inputs(which)
    sc = cfg.scene if nudge == 0 else _nudged(cfg.scene, nudge)
    if nudge != 0:
        est = _nudge32(est, nudge)
    kw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=7, seed=11,
              mode=oracle.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est, guide_cdf=cdf, collect=True)
    if tree is not None:
        kw["octree"] = (tree[0], cells)
    pix, runs, ctr = {}, {}, np.zeros(8)
    for b in starts:
        r = oracle.render(sc, px_begin=b, px_end=b + FULL_RUN_LEN, **kw)
        pix[b] = (r.image[b:b + FULL_RUN_LEN].copy(), r.px_rays[b:b + FULL_RUN_LEN].copy())
        flat = r.stats.reshape(-1, 8)
        idx = np.flatnonzero(flat[:, 0] > 0)
        runs[b] = (idx, flat[idx].copy())   # the run's populated (cell, technique) entries
        if nudge == 0:
            ctr += r.counters
    return pix, runs, ctr


@pytest.mark.parametrize("which", ["guided_512", "heightfield_1024", "large_2048", "bdpt_heightfield_1024",
                                   "bdpt_large_2048"])
def test_full_size_sampled_parity(mars, orc, which):
    """The workloads at their full sizes, in the launch configuration the
    benchmark times (iteration graphs, two tile lanes, the autotuner's launch
    shape; adaptive octree caches for the heightfield workloads, refined by
    the oracle's rule; the two bidirectional workloads with light
    connections), one teacher-forced MARS iteration of the whole frame
    without a multiplicity cap, compared with the oracle on 4096 pixels in 64
    evenly spread runs: every pixel's random streams are keyed by its index, so
    a run of pixels is rendered identically inside the frame and alone.  The
    statistics of the sampled runs (the CUDA path renders them again as pixel
    ranges into empty statistics) are compared in total within 1e-3 and per
    (cell, technique) entry wherever no disagreeing pixel reaches and 4 ulps of
    input do not move the oracle's entry beyond the bar (a single light
    connection over a short distance carries the float32 error of its end
    points amplified by 1 / d^2, as a glossy pixel does its normal's).

    Pixel bar: these frames hold pixels whose value a float32 evaluation cannot
    pin down -- small GGX spheres (alpha down to 0.05) that reflect a light,
    where a normal's rounding error is amplified by ~1 / alpha^2, and path
    trees whose Alg. 1 decisions sit within rounding of an integer.  The oracle
    finds them itself: moving every geometry and camera value of the float32
    scene and every pixel estimate by NUDGE_ULPS = 4 ulps (both ways; a float32
    evaluation chain of tens of operations carries errors of a few ulps) moves
    those pixels by more than 1e-4 in float64.  Outside
    that set, at least 99.9 % of the sampled pixels agree within 1e-4 (the bar
    of the small parity cases); and the float32 path disagrees on no more
    pixels than NUDGE_ULPS ulps of input move the oracle by."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    import torch
    cfg, cells, tree, q_rr, q_s, valid, est, cdf = _full_size_inputs(which)
    sc = cfg.scene
    npx = sc.n_pixels
    starts = _full_size_runs(npx)
    # the oracle's share starts first, in spawned processes (fork after CUDA hangs)
    procs = max(1, min(32, os.cpu_count() or 1))
    pool = cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"))
    futs = {nudge: [pool.submit(_full_size_oracle, (which, nudge, starts[k::procs])) for k in range(procs)]
            for nudge in (0, 1, -1)}
    kw = {} if tree is None else dict(octree=True, max_leaves=cells, split_samples=1e30,
                                      arena_capacity=2 * npx * cfg.max_depth)
    scene = mars.Scene(sc)
    cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, **kw)
    st = dict(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
    if cdf is not None:
        st["guide_cdf"] = cdf
    if tree is not None:
        st.update(oct_nodes=tree[0], oct_leaf_level=tree[1])
    cache.set_state(**st)
    if tree is not None:
        assert cache.info()["oct_n_leaves"] == tree[2] > cfg.n_cells
    gkw = dict(iteration=7, seed=11, mode=mars.MARS_MODE_MARS)
    launch = cache.autotune(repeats=1, **gkw)
    assert all(t > 0 for t in launch["threads"])
    img = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    g_st = cache.render_iteration(img, update_estimate=False, **gkw)
    torch.cuda.synchronize()
    g = img.cpu().numpy().reshape(-1, 3).astype(np.float64)
    g_rays = cache.get_state()["pixel_rays"].astype(np.float64)
    assert g_st["tiles"] >= 1 and np.isfinite(g).all()
    # the sampled runs again, each as a pixel range into empty statistics
    rays = verts = 0
    g_runs = {}
    zero = np.zeros((cells, 3, 8))
    for b in starts:
        cache.set_state(stats=zero, has_estimate=True, n_iterations=1)
        s_ = cache.render_iteration(img, update_estimate=False, px_range=(b, b + FULL_RUN_LEN), **gkw)
        rays += s_["rays"]
        verts += s_["vertices"]
        g_runs[b] = cache.get_state()["stats"]
    res = {n: [f.result() for f in fl] for n, fl in futs.items()}
    pool.shutdown()
    o_pix = {n: {b: p for r in rl for b, p in r[0].items()} for n, rl in res.items()}
    o_runs_n = {n: {b: v for r in rl for b, v in r[1].items()} for n, rl in res.items()}
    o_runs = o_runs_n[0]
    o_ctr = sum(r[2] for r in res[0])
    g_stats = sum(g_runs.values())
    o_stats_n = {}
    for n, runs_ in o_runs_n.items():
        o_stats_n[n] = np.zeros((cells, 3, 8))
        for idx, vals in runs_.values():
            o_stats_n[n].reshape(-1, 8)[idx] += vals
    o_stats = o_stats_n[0]
    # (cell, technique) entries whose sums NUDGE_ULPS ulps of input move beyond the bar
    tol = _stat_tolerance(o_stats) + 1e-12
    sensitive = np.zeros((cells, 3), bool)
    for n in (1, -1):
        sensitive |= (np.abs(o_stats_n[n] - o_stats) > tol).any(axis=-1)
    del o_stats_n, o_runs_n

    def off(x, y):
        return (np.abs(x - y) > PIX_TOL * np.abs(y) + 1e-7).any(axis=1)

    n_off = n_sens = n_off_well = n_rays = 0
    detail = []
    touched = np.zeros(cells, bool)
    n_flagged = 0
    g_ok = np.zeros((cells, 3, 8))
    o_ok = np.zeros((cells, 3, 8))
    for b in starts:
        o, o_rays = o_pix[0][b]
        f = off(g[b:b + FULL_RUN_LEN], o)
        sens = off(o_pix[1][b][0], o) | off(o_pix[-1][b][0], o)
        rays_off = g_rays[b:b + FULL_RUN_LEN] != o_rays
        n_off += int(f.sum())
        n_sens += int(sens.sum())
        n_off_well += int((f & ~sens).sum())
        n_rays += int(rays_off.sum())
        for k in np.flatnonzero(f & ~sens):
            rel = np.abs(g[b + k] - o[k]) / (np.abs(o[k]) + 1e-30)
            detail.append(f"px {b + k}: rel {rel.max():.1e} rays {int(o_rays[k])}")
        # a run whose pixels, or whose sample count or cost in any (cell,
        # technique) entry, differ took another discrete decision somewhere (an
        # Alg. 1 rounding, a hit, a cell boundary): its cells leave the per-cell
        # bar and its sums the totals
        idx, vals = o_runs[b]
        o_run = np.zeros((cells, 3, 8))
        o_run.reshape(-1, 8)[idx] = vals
        same = np.array_equal(g_runs[b][..., 0], o_run[..., 0]) and np.array_equal(g_runs[b][..., 7], o_run[..., 7])
        if f.any() or rays_off.any() or not same:
            n_flagged += 1
            touched |= (g_runs[b][..., 0].sum(-1) > 0) | (o_run[..., 0].sum(-1) > 0)
        else:
            g_ok += g_runs[b]
            o_ok += o_run
    total = FULL_RUNS * FULL_RUN_LEN
    msg = f"{which}: {n_off} of {total} pixels off by > 1e-4 ({n_off_well} of them well conditioned); " \
          f"{NUDGE_ULPS} ulps of input move {n_sens}; {n_rays} path trees of another size; {n_flagged} of " \
          f"{FULL_RUNS} runs took another branch somewhere; well-conditioned off pixels: {detail[:8]}"
    print(msg)
    assert n_off_well <= 0.001 * total + 1, msg
    assert n_off <= max(n_sens, 0.001 * total + 1), msg
    # statistics of the sampled runs: counters of all runs; sums of the runs
    # that took the same discrete decisions; every entry outside the others' cells
    assert abs(rays - o_ctr[0]) <= 1e-3 * o_ctr[0] + 1 and abs(verts - o_ctr[1]) <= 1e-3 * o_ctr[1] + 1
    assert n_flagged < FULL_RUNS // 2, msg
    assert np.allclose(g_ok.sum(0), o_ok.sum(0), rtol=STAT_TOL, atol=1e-6), which
    pop = (g_stats[..., 0] > 0) | (o_stats[..., 0] > 0)
    e_off = pop & ~(np.abs(g_stats - o_stats) <= tol).all(axis=-1)
    print(f"{which}: {NUDGE_ULPS} ulps of input move {int((sensitive & pop).sum())} of {int(pop.sum())} "
          f"populated entries; {int(e_off.sum())} entries off, {int((e_off & sensitive).sum())} of them sensitive")
    _strict_stats(g_stats, o_stats, touched, which, sensitive=sensitive)


def test_lane_settings_and_autotuned_lanes(mars):
    """Tile lanes as a launch setting: the lane count is checked against the
    cache's, a small image (128 x 128, below the default 2^17-pixel floor) split
    over two lanes once the floor is lowered renders the one-lane image bitwise,
    and the autotuner keeps one or all lanes without touching the learned state."""
    import torch
    cfg = W.config_guided(128, 128)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=991, lo=0.3, hi=1.5)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=992, lo=0.05, hi=0.5)
    stream = torch.cuda.Stream()
    scene = mars.Scene(cfg.scene, stream=stream)
    cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, lanes=2, stream=stream)
    base = cache.get_launch()
    assert base["lanes"] == 2 and base["lane_min_pixels"] == 1 << 17
    with pytest.raises(mars.MarsError):
        cache.set_launch(base["threads"], base["blocks_per_sm"], base["max_registers"], lanes=3)
    with pytest.raises(mars.MarsError):
        cache.set_launch(base["threads"], base["blocks_per_sm"], base["max_registers"], lane_min_pixels=1)
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    out = []
    for lanes, floor in ((1, 1 << 17), (2, 1 << 14)):
        cache.set_launch(base["threads"], base["blocks_per_sm"], base["max_registers"], lanes=lanes,
                         lane_min_pixels=floor)
        got = cache.get_launch()
        assert got["lanes"] == lanes and got["lane_min_pixels"] == floor
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                        stats=np.zeros((cfg.n_cells, 3, 8)), stream=stream)
        st = cache.render_iteration(img, seed=17, iteration=1, mode=1, stream=stream)
        torch.cuda.synchronize()
        out.append((img.cpu().numpy().copy(), st))
    (a, sa), (b, sb) = out
    assert sa["tiles"] == 1 and sb["tiles"] == 2
    assert np.array_equal(a, b) and sa["rays"] == sb["rays"] and sa["vertices"] == sb["vertices"]
    before = cache.get_state(stream=stream)
    chosen = cache.autotune(iteration=2, seed=17, mode=1, repeats=1, stream=stream)
    after = cache.get_state(stream=stream)
    assert chosen["lanes"] in (1, 2) and chosen == cache.get_launch()
    for k in ("q_rr", "q_s", "valid", "stats", "pixel_estimate", "guide_cdf"):
        assert np.array_equal(before[k], after[k]), k
    one = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, lanes=1, stream=stream)
    assert one.get_launch()["lanes"] == 1
    with pytest.raises(mars.MarsError):
        one.set_launch(base["threads"], base["blocks_per_sm"], base["max_registers"], lanes=2)


# ------------------------------------------- bidirectional application (Sec. 5)
TECH_BD = W.TECH_BSDF | W.TECH_NEE | W.TECH_LIGHT


@pytest.mark.parametrize("mode,weights", [(0, 0), (1, 0), (1, 1)])
def test_bidirectional_box_parity(mars, orc, mode, weights):
    """Light connections in the box: warm-up (budgets 1) and a teacher-forced
    MARS iteration with random count fields for all three techniques
    (budget-aware and -unaware whole-path weights): image, per-cell statistics
    (the light connection's value, second moment and cost included) and
    counters against the oracle."""
    cfg = W.WorkloadConfig(W.box_scene(48, 40), max_depth=5, grid_n=8, techniques=TECH_BD, iterations=2, warmup=1,
                           name="box bidirectional")
    scene, cache = _make(mars, cfg)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=601, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=602, lo=0.05, hi=1.0)
    okw = dict(grid_n=cfg.grid_n, techniques=TECH_BD, max_depth=cfg.max_depth, iteration=3, seed=5, weights=weights)
    if mode == 1:
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
        okw.update(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
    g_img, g_st = _gpu_iteration(mars, cache, iteration=3, seed=5, mode=mode, weights=weights)
    g_state = cache.get_state()
    o = orc.render(cfg.scene, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, cfg.scene,
                                      dict(iteration=3, seed=5, mode=mode, weights=weights), okw, px)
    _check(g_img, o.image, g_state, o, g_st, f"box bidirectional mode {mode} weights {weights}", touch)
    assert o.stats[:, 2, 0].sum() > 0 and o.stats[:, 2, 1:4].sum() > 0
    assert g_st["light_samples"] == pytest.approx(o.stats[:, 2, 0].sum(), rel=1e-3)
    assert g_st["light_rays"] == pytest.approx(o.counters[6], rel=1e-3)
    assert g_st["vertices"] == pytest.approx(o.counters[1], rel=1e-3)


def test_bidirectional_heightfield_parity(mars, orc):
    """The bidirectional workload's geometry, small: a heightfield whose emitter
    hides between two spheres (most of the terrain is lit only through light
    paths), triangles and spheres, with an adaptive octree refined by the
    oracle's rule and random counts."""
    sc = W.heightfield_scene(3, n=12, width=40, height=32, n_spheres=20)
    cfg = W.WorkloadConfig(sc, max_depth=6, grid_n=4, techniques=TECH_BD, iterations=2, warmup=1, name="hf bd")
    cells = 1024
    nodes, nn, nl, lvl, lnode = orc.octree_init(4, cells)
    rng = np.random.default_rng(611)
    z = np.zeros((cells, 3, 3), np.float32)
    zv = np.zeros((cells, 3), np.uint8)
    stt = np.zeros((cells, 3, 8))
    stt[:nl, 0, 0] = rng.integers(0, 200, size=nl)
    nodes, nn, nl, lvl, lnode, *_ = orc.octree_refine(cells, 100.0, stt, nodes, nn, nl, lvl, lnode, z, z, zv)
    scene = mars.Scene(sc)
    cache = mars.Cache(scene, 4, TECH_BD, 6, octree=True, max_leaves=cells, split_samples=1e30)
    q_rr, q_s, valid = W.random_count_fields(cells, seed=612, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=613, lo=0.01, hi=0.5)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                    oct_nodes=nodes[:nn], oct_leaf_level=lvl[:nl])
    g_img, g_st = _gpu_iteration(mars, cache, iteration=2, seed=8, mode=1)
    g_state = cache.get_state()
    okw = dict(grid_n=4, techniques=TECH_BD, max_depth=6, iteration=2, seed=8, mode=orc.MODE_MARS, q_rr=q_rr,
               q_s=q_s, valid=valid, est=est, octree=(nodes, cells))
    o = orc.render(sc, **okw)
    touch = lambda px: _touched_cells(mars, orc, cache, sc, dict(iteration=2, seed=8, mode=1), okw, px)
    _check(g_img, o.image, g_state, o, g_st, "heightfield bidirectional", touch)
    assert o.stats[:, 2, 1:4].sum() > 0


@pytest.mark.parametrize("albedo,D", [(0.5, 4), (0.7, 6)])
def test_gpu_bidirectional_furnace_closed_form(mars, albedo, D):
    """The closed furnace through the CUDA path with light connections and
    random counts: the image mean is Le (1 - a^D)/(1 - a) within 3.5 sigma."""
    import torch
    sc = W.furnace_scene(albedo=albedo, radiance=1.5, width=32, height=32)
    scene = mars.Scene(sc)
    cache = mars.Cache(scene, 4, TECH_BD, D)
    q_rr, q_s, valid = W.random_count_fields(64, seed=621, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=622, lo=0.5, hi=4.0)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
    img = torch.zeros(sc.n_pixels * 3, dtype=torch.float32, device="cuda")
    vals = []
    for it in range(40):
        cache.render_iteration(img, iteration=it, mode=1, collect=False, update_estimate=False)
        vals.append(float(img.double().mean()))
    m, se = np.mean(vals), np.std(vals, ddof=1) / math.sqrt(len(vals))
    expected = 1.5 * (1 - albedo ** D) / (1 - albedo)
    assert abs(m - expected) < 3.5 * se + 1e-6, (m, expected, se)


def test_bidirectional_tiles_lanes_and_graphs_do_not_change_the_image(mars):
    """A queue arena too small for the frame (pixel tiles, re-rendered after an
    overflow), two tile lanes and CUDA-graph replay give the image of one
    directly launched tile bit for bit, with light connections."""
    import torch
    cfg = W.WorkloadConfig(W.box_scene(64, 48), max_depth=6, grid_n=8, techniques=TECH_BD, iterations=1, warmup=0,
                           name="box bd")
    scene = mars.Scene(cfg.scene)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=631, lo=0.3, hi=4.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=632, lo=0.05, hi=0.5)
    out = []
    for kw in (dict(graphs=False, lanes=1), dict(arena_capacity=20000, graphs=False, lanes=1),
               dict(graphs=True, lanes=2)):
        cache = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth, **kw)
        cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1)
        if kw.get("lanes") == 2:
            cache.set_launch([128] * 4, [0] * 4, lanes=2, lane_min_pixels=2)
        s = torch.cuda.Stream()
        img = torch.zeros(cfg.scene.n_pixels * 3, dtype=torch.float32, device="cuda")
        for rep in range(2):
            st = cache.render_iteration(img, iteration=4, seed=2, mode=1, update_estimate=False, stream=s)
        torch.cuda.synchronize()
        out.append((img.cpu().numpy().copy(), st))
    assert out[1][1]["tiles"] > 1
    for img, st in out[1:]:
        assert np.array_equal(img, out[0][0])
        assert st["light_samples"] == out[0][1]["light_samples"] and st["rays"] == out[0][1]["rays"]


def test_bidirectional_argument_errors(mars):
    sc = W.box_scene(8, 8)
    scene = mars.Scene(sc)
    with pytest.raises(mars.MarsError) as e:
        mars.Cache(scene, 4, W.TECH_BSDF | W.TECH_GUIDED | W.TECH_LIGHT, 4)
    assert e.value.status == mars.MARS_ERR_INVALID_ARG
    with pytest.raises(mars.MarsError) as e:
        mars.Cache(scene, 4, W.TECH_BSDF | 16, 4)
    assert e.value.status == mars.MARS_ERR_INVALID_ARG
