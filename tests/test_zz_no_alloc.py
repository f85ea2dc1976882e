"""mars_image_stats_static: the image-statistics pass for callers that cannot
allocate device memory (its scratch is a static device array of the library).

Called through the C ABI on caller-owned buffers, twice in a row, and compared
with the statistics that mars_render_iteration computes for the same images
(running sum, pixel estimate, V_I, C_I), within 1e-6 relative; and on images of
other shapes (wider than a block's row loop, taller than its grid, and exactly
as tall as the scratch allows) against the CPU oracle's image statistics of the
same buffers.  This file is
collected last so that a failure here stops a -x run only after every other
test has run; it passes alone and after the other tests.
"""
import ctypes as ct

import numpy as np
import pytest

import mars_workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2410_20429_gb300 import build as B
    B.build()
    import paper_2410_20429_gb300 as M
    from paper_2410_20429_gb300 import _abi as A
    return torch, M, A, A.load()


def test_static_image_stats_match_render_iteration(env):
    torch, M, A, L = env
    w, h = 64, 48
    cfg = W.config_box(w, h)
    scene = M.Scene(cfg.scene)
    cache = M.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    npx = w * h
    rs0 = (W.random_pixel_estimate(npx, seed=901, lo=0.1, hi=3.0) * 2.0).astype(np.float32)
    cache.set_state(run_sum=rs0, n_iterations=2, has_estimate=True, pixel_estimate=np.ones((npx, 3), np.float32))
    run_dev = torch.from_numpy(rs0.reshape(-1).copy()).cuda()        # caller-owned running sum
    est_dev = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    vici = torch.zeros(2, dtype=torch.float64, device="cuda")
    img = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        n_prev = 2 + call
        st = cache.render_iteration(img, iteration=n_prev, seed=4, mode=A.MARS_MODE_WARMUP, update_estimate=True)
        ref = cache.get_state()
        rc = L.mars_image_stats_static(ct.c_void_p(img.data_ptr()), ct.c_void_p(run_dev.data_ptr()),
                                       ct.c_void_p(est_dev.data_ptr()), w, h, n_prev, 50.0, float(st["rays"]),
                                       ct.c_void_p(vici.data_ptr()), ct.c_void_p(stream))
        assert rc == A.MARS_OK, L.mars_last_error_string()
        torch.cuda.synchronize()
        np.testing.assert_allclose(run_dev.cpu().numpy().reshape(-1, 3), ref["run_sum"], rtol=TOL)
        np.testing.assert_allclose(est_dev.cpu().numpy().reshape(-1, 3), ref["pixel_estimate"], rtol=TOL)
        vi, ci = vici.cpu().numpy()
        assert vi == pytest.approx(st["VI"], rel=TOL)
        assert ci == pytest.approx(st["CI"], rel=TOL)


def test_static_image_stats_rejects_images_taller_than_its_scratch(env):
    torch, M, A, L = env
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = ct.c_void_p(buf.data_ptr())
    rc = L.mars_image_stats_static(p, p, p, 1, 8193, 0, 50.0, 1.0, ct.c_void_p(out.data_ptr()), None)
    assert rc == A.MARS_ERR_INVALID_ARG
    assert b"8192" in L.mars_last_error_string()


@pytest.mark.parametrize("w,h", [(300, 1100), (3, 8192)])
def test_static_image_stats_match_the_oracle_on_other_shapes(env, orc, w, h):
    """Rows wider than one block (the per-row loop takes several steps), more
    rows than one grid pass, and the tallest image the scratch holds: the
    running sum, pixel estimate, V_I and C_I of a seeded image agree with the
    oracle's image statistics of the same float32 buffers."""
    torch, M, A, L = env
    npx = w * h
    img = W.random_pixel_estimate(npx, seed=911, lo=0.01, hi=5.0)
    rs0 = W.random_pixel_estimate(npx, seed=912, lo=0.1, hi=3.0) * 3.0
    n_prev, rays = 3, 7.25 * npx
    img_dev = torch.from_numpy(img.reshape(-1).copy()).cuda()
    run_dev = torch.from_numpy(rs0.reshape(-1).copy()).cuda()
    est_dev = torch.zeros(npx * 3, dtype=torch.float32, device="cuda")
    vici = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.mars_image_stats_static(ct.c_void_p(img_dev.data_ptr()), ct.c_void_p(run_dev.data_ptr()),
                                   ct.c_void_p(est_dev.data_ptr()), w, h, n_prev, 50.0, rays,
                                   ct.c_void_p(vici.data_ptr()), ct.c_void_p(stream))
    assert rc == A.MARS_OK, L.mars_last_error_string()
    torch.cuda.synchronize()
    vi, rs, est = orc.image_stats(w, h, img.astype(np.float64), rs0.astype(np.float64), n_prev)
    np.testing.assert_allclose(run_dev.cpu().numpy().reshape(-1, 3), rs, rtol=TOL)
    np.testing.assert_allclose(est_dev.cpu().numpy().reshape(-1, 3), est, rtol=1e-5)
    g_vi, g_ci = vici.cpu().numpy()
    assert g_vi == pytest.approx(vi, rel=1e-5)
    assert g_ci == pytest.approx(rays / npx, rel=1e-12)
