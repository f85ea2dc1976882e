"""Float32 versus float64 statistics (the precision study): the same iteration
rendered from the same state on a float64 cache and on a float32-statistics
cache.  The images are identical (statistics never feed back within an
iteration); every statistic of the float32 run is compared with the float64
run and its relative error bounded:

* integer-valued sums (sample count, cost) are exact in float32 below 2^24;
* value sums, moments, mean cost, q^RR, V_I, C_I: the float32 accumulation of
  a few thousand pre-reduced partial sums, within 1e-3 at the worst entry;
* the variance m2 - m1^2 and q^S lose digits to cancellation where the
  variance is small against m2; they are compared where var > 1e-3 m2, within
  5e-2 at the worst entry and 1e-4 at the median.
"""
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


def test_float32_statistics_error_per_statistic(mars):
    from paper_2410_20429_gb300 import precision
    cfg = W.config_guided(160, 128)
    npx = cfg.scene.n_pixels
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=801, lo=0.3, hi=3.0)
    est = W.random_pixel_estimate(npx, seed=802, lo=0.05, hi=0.5)
    rep = precision.compare(cfg.scene, cfg.grid_n, cfg.techniques, cfg.max_depth, q_rr, q_s, valid, est,
                            est * 2.0, 2, iteration=2, seed=9)
    print({k: v for k, v in rep.items()})
    assert rep["images_equal"]
    assert rep["cells_compared"] > 100
    assert rep["n"]["max"] == 0.0 and rep["sum_cost"]["max"] == 0.0
    for k in ("sum_v", "sum_v2", "m1", "m2", "C_t", "q_rr", "V_I", "C_I"):
        assert rep[k]["max"] <= 1e-3, (k, rep[k])
    for k in ("var", "q_s"):
        assert rep[k]["max"] <= 5e-2 and rep[k]["median"] <= 1e-4, (k, rep[k])
