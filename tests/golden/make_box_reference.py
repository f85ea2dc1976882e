"""Writes the long oracle reference of the box scene used by the relMSE
agreement test (relative MSE against a 64k-samples-per-pixel reference, the
third agreement criterion of the parity suite).

The reference is the CPU oracle's own render (``oracle/``, nothing else): the
Cornell-like box at 32 x 32, D = 5, BSDF + NEE, fixed-count MIS (beta = 1 for
every technique), Philox seed 999, iterations 0 .. 65535, one sample per pixel
each.  It stores per pixel the mean over the iterations and the variance of that
mean (the sample variance of the iterations divided by their number).

    python tests/golden/make_box_reference.py [--iterations 65536] [--procs N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "box_32x32_fixed_65536spp.txt")
SEED = 999
WIDTH = HEIGHT = 32


def _chunk(args):
    lo, hi = args
    sys.path.insert(0, ROOT)
    import mars_workloads as W
    import oracle as orc
    cfg = W.config_box(WIDTH, HEIGHT)
    s1 = np.zeros((cfg.scene.n_pixels, 3))
    s2 = np.zeros((cfg.scene.n_pixels, 3))
    for it in range(lo, hi):
        r = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                       mode=orc.MODE_FIXED, seed=SEED, iteration=it, collect=False)
        s1 += r.image
        s2 += r.image ** 2
    return s1, s2


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iterations", type=int, default=65536)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    sys.path.insert(0, ROOT)
    import oracle as orc
    orc.build()
    n = a.iterations
    step = (n + 4 * a.procs - 1) // (4 * a.procs)
    chunks = [(lo, min(lo + step, n)) for lo in range(0, n, step)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        parts = pool.map(_chunk, chunks)
    s1 = sum(p[0] for p in parts)
    s2 = sum(p[1] for p in parts)
    mean = s1 / n
    var_of_mean = np.maximum(s2 / n - mean ** 2, 0.0) * n / (n - 1) / n
    hdr = (f"box scene {WIDTH}x{HEIGHT}, D=5, BSDF+NEE, fixed-count MIS, Philox seed {SEED}, "
           f"iterations 0..{n - 1}, CPU oracle (oracle/)\n"
           "columns: pixel mean r g b, variance of the mean r g b (pixel index = row)")
    np.savetxt(OUT, np.concatenate([mean, var_of_mean], axis=1), fmt="%.10e", header=hdr)
    print(OUT)


if __name__ == "__main__":
    main()
