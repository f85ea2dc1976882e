"""Writes the long oracle references used by the relMSE agreement tests
(relative MSE against a 64k-samples-per-pixel reference, the third agreement
criterion of the parity suite).

Each reference is the CPU oracle's own render (``oracle/``, nothing else) at
32 x 32, fixed-count MIS (beta = 1 for every technique), Philox seed 999,
iterations 0 .. 65535, one sample per pixel each:
  box     the Cornell-like box, D = 5, BSDF + NEE;
  guided  the guided room's geometry (64 spheres, 4 ceiling lights), D = 10,
          BSDF + NEE + guided with the uniform guide.
It stores per pixel the mean over the iterations and the variance of that mean
(the sample variance of the iterations divided by their number).

    python tests/golden/make_box_reference.py [--scene box|guided] [--iterations 65536] [--procs N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = {"box": os.path.join(HERE, "box_32x32_fixed_65536spp.txt"),
       "guided": os.path.join(HERE, "guided_room_32x32_fixed_65536spp.txt")}
SEED = 999
WIDTH = HEIGHT = 32


def _config(scene):
    import mars_workloads as W
    return W.config_box(WIDTH, HEIGHT) if scene == "box" else W.config_guided(WIDTH, HEIGHT)


def _chunk(args):
    scene, lo, hi = args
    sys.path.insert(0, ROOT)
    import oracle as orc
    cfg = _config(scene)
    kw = {}
    if scene == "guided":
        kw["guide_cdf"] = np.tile((np.arange(1, orc.GUIDE_BINS + 1) / orc.GUIDE_BINS).astype(np.float32),
                                  (cfg.n_cells, 1))
    s1 = np.zeros((cfg.scene.n_pixels, 3))
    s2 = np.zeros((cfg.scene.n_pixels, 3))
    for it in range(lo, hi):
        r = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                       mode=orc.MODE_FIXED, seed=SEED, iteration=it, collect=False, **kw)
        s1 += r.image
        s2 += r.image ** 2
    return s1, s2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", default="box", choices=sorted(OUT))
    ap.add_argument("--iterations", type=int, default=65536)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle as orc
    orc.build()
    n = a.iterations
    step = (n + 4 * a.procs - 1) // (4 * a.procs)
    chunks = [(a.scene, lo, min(lo + step, n)) for lo in range(0, n, step)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        parts = pool.map(_chunk, chunks)
    s1 = sum(p[0] for p in parts)
    s2 = sum(p[1] for p in parts)
    mean = s1 / n
    var_of_mean = np.maximum(s2 / n - mean ** 2, 0.0) * n / (n - 1) / n
    what = ("box scene, D=5, BSDF+NEE" if a.scene == "box" else
            "guided room geometry (64 spheres, 4 lights), D=10, BSDF+NEE+guided with the uniform guide")
    hdr = (f"{what}, {WIDTH}x{HEIGHT}, fixed-count MIS, Philox seed {SEED}, "
           f"iterations 0..{n - 1}, CPU oracle (oracle/)\n"
           "columns: pixel mean r g b, variance of the mean r g b (pixel index = row)")
    np.savetxt(OUT[a.scene], np.concatenate([mean, var_of_mean], axis=1), fmt="%.10e", header=hdr)
    print(OUT[a.scene])


if __name__ == "__main__":
    main()
