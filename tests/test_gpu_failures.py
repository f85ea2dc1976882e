"""GPU tests of the error paths, driven by the library's host-side failure
injection (mars_debug_inject_failure) and the server's job timeout, so that no
GPU is faulted: an allocation that fails leaves nothing behind and the next
object is created normally; a failed launch poisons only its own cache; a
served job that runs out of memory or time fails alone while the jobs beside
it finish."""
import time

import numpy as np
import pytest

import mars_workloads as W

pytestmark = pytest.mark.gpu

TECH = W.TECH_BSDF | W.TECH_NEE | W.TECH_GUIDED


@pytest.fixture(scope="module")
def mars():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2410_20429_gb300 import build as B
    B.build()
    import paper_2410_20429_gb300 as M
    yield M
    M.inject_failure(M.MARS_INJECT_ALLOC, 0)
    M.inject_failure(M.MARS_INJECT_LAUNCH, 0)


def _render(M, cache, it=0):
    import torch
    img = torch.zeros(cache.n_pixels * 3, dtype=torch.float32, device="cuda")
    st = cache.render_iteration(img, iteration=it, mode=M.MARS_MODE_WARMUP, update_estimate=True)
    torch.cuda.synchronize()
    return img.cpu().numpy(), st


@pytest.mark.parametrize("n", [1, 3, 9])
def test_injected_allocation_failure_in_cache_creation(mars, n):
    """The n-th allocation of a cache's creation fails: creation reports
    MARS_ERR_OOM, and the next cache on the same scene renders the same image as
    a cache created before the failure."""
    cfg = W.config_box(32, 32)
    scene = mars.Scene(cfg.scene)
    ref = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    a, _ = _render(mars, ref)
    mars.inject_failure(mars.MARS_INJECT_ALLOC, n)
    try:
        with pytest.raises(mars.MarsError) as e:
            mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
        assert e.value.status == mars.MARS_ERR_OOM
    finally:
        mars.inject_failure(mars.MARS_INJECT_ALLOC, 0)
    again = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    b, _ = _render(mars, again)
    assert np.array_equal(a, b)


def test_injected_launch_failure_poisons_only_its_cache(mars):
    """A render that fails (injected) returns MARS_ERR_CUDA and poisons its
    cache: every later call on it fails at once, destroying it works, and a
    second cache on the same scene keeps rendering."""
    cfg = W.config_box(32, 32)
    scene = mars.Scene(cfg.scene)
    bad = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    good = mars.Cache(scene, cfg.grid_n, cfg.techniques, cfg.max_depth)
    a, _ = _render(mars, good)
    mars.inject_failure(mars.MARS_INJECT_LAUNCH, 1)
    try:
        with pytest.raises(mars.MarsError) as e:
            _render(mars, bad)
        assert e.value.status == mars.MARS_ERR_CUDA
    finally:
        mars.inject_failure(mars.MARS_INJECT_LAUNCH, 0)
    with pytest.raises(mars.MarsError) as e2:
        bad.update_counts()
    assert "poisoned" in str(e2.value)
    bad.close()
    b, _ = _render(mars, good)
    assert np.array_equal(a, b)
    # an injected update failure poisons too
    mars.inject_failure(mars.MARS_INJECT_LAUNCH, 1)
    try:
        with pytest.raises(mars.MarsError):
            good.update_counts()
    finally:
        mars.inject_failure(mars.MARS_INJECT_LAUNCH, 0)
    with pytest.raises(mars.MarsError):
        _render(mars, good)


def _wait(M, srv, ids, timeout=180.0):
    t0 = time.time()
    out = {}
    while len(out) < len(ids):
        for j in ids:
            if j not in out:
                st, _ = srv.poll(j)
                if st["state"] in (M.MARS_JOB_DONE, M.MARS_JOB_FAILED):
                    out[j] = st
        assert time.time() - t0 < timeout, "jobs did not finish in time"
        time.sleep(0.01)
    return out


def test_served_jobs_failing_by_memory_and_time_leave_the_others(mars):
    """A job whose cache allocation fails (injected while the server is idle)
    ends FAILED with MARS_ERR_OOM; a job with a timeout far below its run time
    ends FAILED with MARS_ERR_TIMEOUT after fewer iterations than asked; a job
    beside it finishes every iteration."""
    srv = mars.Server(8 << 30, 4)
    try:
        sc = W.guided_room_scene(3, 64, 64, n_spheres=16)
        mars.inject_failure(mars.MARS_INJECT_ALLOC, 2)
        try:
            j_oom = srv.submit(sc, grid_n=16, techniques=TECH, max_depth=6, iterations=3, warmup=1, seed=1, key=1)
            r = _wait(mars, srv, [j_oom])
        finally:
            mars.inject_failure(mars.MARS_INJECT_ALLOC, 0)
        assert r[j_oom]["state"] == mars.MARS_JOB_FAILED and r[j_oom]["error"] == mars.MARS_ERR_OOM
        big = W.guided_room_scene(4, 256, 256, n_spheres=64)
        j_slow = srv.submit(big, grid_n=16, techniques=TECH, max_depth=8, iterations=4000, warmup=3, seed=2, key=2,
                            timeout_s=0.05)
        j_ok = srv.submit(sc, grid_n=16, techniques=TECH, max_depth=6, iterations=6, warmup=2, seed=3, key=3)
        r = _wait(mars, srv, [j_slow, j_ok])
        assert r[j_slow]["state"] == mars.MARS_JOB_FAILED and r[j_slow]["error"] == mars.MARS_ERR_TIMEOUT
        assert r[j_slow]["iterations_done"] < 4000
        assert r[j_ok]["state"] == mars.MARS_JOB_DONE and r[j_ok]["iterations_done"] == 6
    finally:
        srv.close()
