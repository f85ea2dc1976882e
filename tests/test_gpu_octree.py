"""GPU parity of the adaptive octree cache (MARS_CACHE_OCTREE) against the CPU
oracle: an unrefined octree is the uniform grid; refinement after an update
produces exactly the oracle's tree from the same statistics; rendering with a
refined tree matches the oracle."""
import numpy as np
import pytest

import mars_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mars():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2410_20429_gb300 import build as B
    B.build()
    import paper_2410_20429_gb300 as M
    return M


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _render(M, cache, **kw):
    import torch
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    st = cache.render_iteration(img, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(-1, 3).astype(np.float64), st


def test_unrefined_octree_is_the_grid(mars):
    """An octree that has not split renders the uniform grid's image bit for bit
    and learns the same counts; a MARS iteration from the same learned state
    (the grid's, copied into the octree cache: the float64 and float32
    statistics atomics of the two caches may add in other orders, which moves
    a count or a guide bin by an ulp) renders the same image again."""
    cfg = W.config_guided(40, 32)
    scene = mars.Scene(cfg.scene)
    grid = mars.Cache(scene, 8, cfg.techniques, 6)
    octc = mars.Cache(scene, 8, cfg.techniques, 6, octree=True, max_leaves=4096, split_samples=1e9)
    a, sa = _render(mars, grid, iteration=0, seed=3, update_estimate=True)
    b, sb = _render(mars, octc, iteration=0, seed=3, update_estimate=True)
    assert np.array_equal(a, b) and sa["rays"] == sb["rays"]
    grid.update_counts()
    octc.update_counts()
    ga, gb = grid.get_state(), octc.get_state()
    assert gb["oct_n_leaves"] == 512
    assert np.array_equal(ga["valid"], gb["valid"][:512])
    assert np.allclose(ga["q_rr"], gb["q_rr"][:512], rtol=1e-6, atol=0)
    assert np.allclose(ga["q_s"], gb["q_s"][:512], rtol=1e-3, atol=1e-12)
    st = {}
    for k in ("q_rr", "q_s", "valid", "guide_cdf"):
        v = gb[k].copy()
        v[:512] = ga[k]
        st[k] = v
    octc.set_state(pixel_estimate=ga["pixel_estimate"], run_sum=ga["run_sum"], has_estimate=True,
                   n_iterations=ga["n_iterations"], **st)
    a, _ = _render(mars, grid, iteration=1, seed=3, mode=1)
    b, _ = _render(mars, octc, iteration=1, seed=3, mode=1)
    assert np.array_equal(a, b)


def test_octree_refinement_and_rendering_parity(mars, orc):
    """The guided-room crop of the grid parity test (16 spheres, so that the
    float32-vs-float64 residue under narrow GGX lobes stays below the 0.1 %
    pixel bar; with 64 spheres the grid itself agrees on 99.5 % within 1e-4 and
    100 % within 1e-2)."""
    sc = W.guided_room_scene(seed=0, width=64, height=64, n_spheres=16)
    cfg = W.WorkloadConfig(sc, max_depth=6, grid_n=8, techniques=7, iterations=1, warmup=0, name="octree crop")
    ML = 4096
    scene = mars.Scene(cfg.scene)
    cache = mars.Cache(scene, 8, cfg.techniques, 6, octree=True, max_leaves=ML, split_samples=40.0)
    q_rr, q_s, valid = W.random_count_fields(ML, seed=131, lo=0.2, hi=3.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=132, lo=0.05, hi=0.5)
    cache.set_state(q_rr=q_rr, q_s=q_s, valid=valid, pixel_estimate=est, has_estimate=True, n_iterations=1,
                    VI=0.3, CI=5.0)
    _render(mars, cache, iteration=1, seed=4, mode=1)
    before = cache.get_state()
    cache.set_state(VI=0.3, CI=5.0, n_iterations=1, has_estimate=True)
    cache.update_counts()
    after = cache.get_state()
    # the oracle's update, guide rebuild and refinement from the same statistics
    nodes, nn, nl, lvl, lnode = orc.octree_init(8, ML)
    o_q = orc.update_counts(before["stats"], 0.3, 5.0, cfg.techniques, before["q_rr"], before["q_s"],
                            before["valid"])
    o_cdf = orc.guide_update(before["guide_hist"].astype(np.float64))
    (nodes, nn, nl, lvl, lnode, q_rr2, q_s2, valid2, hist2, cdf2, sp) = orc.octree_refine(
        ML, 40.0, before["stats"], nodes, nn, nl, lvl, lnode, o_q[0], o_q[1], o_q[2],
        before["guide_hist"].astype(np.float64), o_cdf)
    assert sp > 10, "the test should refine"
    assert after["oct_n_nodes"] == nn and after["oct_n_leaves"] == nl
    assert np.array_equal(after["oct_nodes"], nodes[:nn])
    assert np.array_equal(after["oct_leaf_level"], lvl[:nl])
    assert np.array_equal(after["valid"][:nl], valid2[:nl])
    np.testing.assert_allclose(after["q_rr"][:nl], q_rr2[:nl], rtol=1e-6)
    np.testing.assert_allclose(after["guide_cdf"][:nl], cdf2[:nl], atol=2e-7)
    # render with the refined tree on both sides (teacher-forced state)
    img, st = _render(mars, cache, iteration=2, seed=4, mode=1, update_estimate=False)
    g = cache.get_state()
    o = orc.render(cfg.scene, grid_n=8, techniques=cfg.techniques, max_depth=6, iteration=2, seed=4,
                   mode=orc.MODE_MARS, q_rr=after["q_rr"], q_s=after["q_s"], valid=after["valid"],
                   est=after["pixel_estimate"], guide_cdf=after["guide_cdf"], octree=(after["oct_nodes"], ML))
    # the refined leaves add cell boundaries: a vertex within float32 rounding of
    # one (the CUDA path's hit points are float32, the oracle's float64) can take
    # the neighbouring cell's counts and a different subtree, so this bar is
    # 99.5 % (observed 99.8 %) instead of the grid tests' 99.9 %; the image
    # means and the statistics' totals still agree to 1e-3
    ok = (np.abs(img - o.image) <= 1e-4 * np.abs(o.image) + 1e-7).all(axis=1).mean()
    assert ok >= 0.995, ok
    assert abs(img.mean() - o.image.mean()) <= 1e-3 * o.image.mean()
    np.testing.assert_allclose(g["stats"].sum(axis=0), o.stats.sum(axis=0), rtol=1e-3, atol=1e-6)
    used = (g["stats"][..., 0] > 0) | (o.stats[..., 0] > 0)
    assert used[512:].any(), "new leaves receive samples"
    close = (np.abs(g["stats"] - o.stats) <= 1e-3 * np.abs(o.stats) + 1e-9).all(axis=-1)
    assert close[used].mean() >= 0.99
