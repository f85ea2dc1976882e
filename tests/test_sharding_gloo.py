"""World-size-2 ranks on the CPU (gloo).

1. The bench's whole-job aggregation over ranks: the time is the slowest
   rank's, the units are summed.
2. The one exchange a pixel-sharded iteration would need: every rank renders
   its half of the pixels, the float64 statistics and counters are summed with
   an all-reduce, and the result equals one unsharded iteration (up to float64
   reassociation); the count update on the reduced statistics equals the update
   on the whole.  Run with the CPU oracle, whose sums are exactly linear in the
   pixel set (the statistics of Sec. 4.1 are sums over samples).
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    import bench
    import mars_workloads as W
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.reduce_over_ranks(10.0 + 5.0 * rank, 100 * (rank + 1), world, "cpu")
        cfg = W.config_box(16, 12)
        npx = cfg.scene.n_pixels
        q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=901, lo=0.3, hi=3.0)
        est = W.random_pixel_estimate(npx, seed=902, lo=0.05, hi=0.5)
        a, b = npx * rank // world, npx * (rank + 1) // world
        r = oracle.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                          mode=oracle.MODE_MARS, iteration=3, seed=5, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                          px_begin=a, px_end=b)
        stats = torch.from_numpy(r.stats.copy())
        ctr = torch.from_numpy(r.counters.copy())
        img = torch.from_numpy(r.image.copy())
        dist.all_reduce(stats)
        dist.all_reduce(ctr)
        dist.all_reduce(img)
        out_q.put((rank, t, u, stats.numpy(), ctr.numpy(), img.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard_by_pixels():
    pytest.importorskip("torch.distributed")
    import mars_workloads as W
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    for _, t, u, *_ in res:
        assert t == 15.0 and u == 300.0
    _, _, _, stats, ctr, img = res[0]
    cfg = W.config_box(16, 12)
    q_rr, q_s, valid = W.random_count_fields(cfg.n_cells, seed=901, lo=0.3, hi=3.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=902, lo=0.05, hi=0.5)
    full = oracle.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                         mode=oracle.MODE_MARS, iteration=3, seed=5, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
    assert np.array_equal(img, full.image)        # every pixel comes from exactly one rank
    np.testing.assert_allclose(stats, full.stats, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ctr[:3], full.counters[:3], rtol=0, atol=0)
    VI, CI = 0.25, full.rays / cfg.scene.n_pixels
    a = oracle.update_counts(stats, VI, CI, cfg.techniques, q_rr, q_s, valid)
    b = oracle.update_counts(full.stats, VI, CI, cfg.techniques, q_rr, q_s, valid)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-6)
