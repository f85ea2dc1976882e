"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: closed forms
(furnace, polygonal-light irradiance, the budget-unaware optimum of App. A.3),
invariants (sum of MIS weights, unbiasedness under any count field, Alg. 1
marginals), the paper's own derived formulas (rounding variance rho of App. A.2)
and brute force over small grids.
"""
import math
import os

import numpy as np
import pytest

import mars_workloads as W


# --------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors(orc):
    """The oracle's Philox4x32-10 reproduces the published known-answer vectors
    (tests/golden/philox4x32_10_kat.txt, Random123 / Salmon et al. 2011) bit for
    bit; the CUDA path's bits equal the oracle's (every pixel-parity test)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        lhs, rhs = line.split(":")
        words = [int(w, 16) for w in lhs.split()]
        want = [int(w, 16) for w in rhs.split()]
        got = orc.philox(np.array(words[:4], np.uint32), np.array(words[4:], np.uint32))
        assert [int(x) for x in got] == want, line
        n += 1
    assert n == 3


def test_philox_uniform_and_avalanche(orc):
    rng = np.random.default_rng(1)
    key = np.array([12345, 678], np.uint32)
    outs = []
    for i in range(20000):
        outs.append(orc.philox(np.array([i, 7, 3, 0], np.uint32), key))
    o = np.array(outs, dtype=np.uint64)
    u = (o >> np.uint64(8)).astype(np.float64) / 2 ** 24
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    hist = np.histogram(u, bins=64, range=(0, 1))[0]
    exp = u.size / 64
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    bits = np.unpackbits(o.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    # avalanche: one flipped counter bit flips about half of the 128 output bits
    flips = []
    for _ in range(300):
        c = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        b = int(rng.integers(0, 128))
        c2 = c.copy()
        c2[b // 32] ^= np.uint32(1 << (b % 32))
        a1, a2 = orc.philox(c, k), orc.philox(c2, k)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a1, a2)))
    assert abs(np.mean(flips) - 64) < 2.0
    # a bijection of the counter for a fixed key: no collisions
    seen = {tuple(x) for x in o.tolist()}
    assert len(seen) == len(o)


# ---------------------------------------------------------------------- Alg. 1
@pytest.mark.parametrize("betas", [[0.3, 0.45], [1.7, 0.05, 2.25], [0.999, 19.5, 3.0], [4.0, 0.5, 0.5]])
def test_alg1_marginals_and_total(orc, betas):
    """Alg. 1 (App. B.1): with one uniform r, E[gamma_t] = beta_t for every t and
    the total is floor or ceil of sum(beta)."""
    n = 1 << 14
    g = np.array([orc.stochastic_round(betas, (k + 0.5) / n) for k in range(n)])
    b = np.array(betas, np.float32).astype(np.float64)
    assert np.all(np.abs(g.mean(0) - b) <= len(betas) / n + 1e-6)
    tot = g.sum(1)
    assert set(np.unique(tot)) <= {math.floor(b.sum()), math.ceil(b.sum())}
    # every technique's count is floor or ceil of its own budget
    for t in range(len(betas)):
        assert set(np.unique(g[:, t])) <= {math.floor(b[t]), math.ceil(b[t])}


@pytest.mark.parametrize("beta", [0.3, 1.0, 1.4, 2.5, 7.75])
@pytest.mark.parametrize("E,V", [(1.0, 0.5), (2.0, 10.0)])
def test_stochastic_rounding_variance_matches_rho(orc, beta, E, V):
    """App. A.2: V[<I; beta>] = V/beta + rho(beta) E^2 with
    rho = (beta - floor)(ceil - beta) / beta^2, for rounding that divides by the
    real-valued beta.  gamma comes from the oracle's Alg. 1 with one technique;
    E[(sum_{s<=gamma} X)^2 | gamma] = gamma V + gamma^2 E^2."""
    n = 1 << 14
    gam = np.array([orc.stochastic_round([beta], (k + 0.5) / n)[0] for k in range(n)], np.float64)
    b = float(np.float32(beta))
    second = ((gam * V + gam ** 2 * E ** 2) / b ** 2).mean()
    mean = (gam * E / b).mean()
    var = second - mean ** 2
    rho = (b - math.floor(b)) * (math.ceil(b) - b) / b ** 2
    assert mean == pytest.approx(E, rel=1e-3)
    assert var == pytest.approx(V / b + rho * E ** 2, rel=2e-3, abs=1e-6)


# ------------------------------------------------------------------------- MIS
def test_balance_weights_sum_to_one(orc):
    """App. A.1: for every subintegrand the weights of the participating
    techniques sum to one (budget-aware and budget-unaware)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        beta = rng.uniform(0.05, 20, 3)
        pdf = rng.exponential(1.0, 3)
        part = rng.integers(0, 2, 3)
        part[rng.integers(0, 3)] = 1
        for aware in (True, False):
            ws = [orc.balance_weight(beta, pdf, part, t, aware) for t in range(3)]
            assert sum(ws) == pytest.approx(1.0, rel=1e-12)
            for t in range(3):
                if not part[t]:
                    assert ws[t] == 0.0
    # budget-aware weight of a technique grows with its own budget
    w1 = orc.balance_weight([1.0, 1.0, 0], [1.0, 1.0, 0], [1, 1, 0], 0, True)
    w2 = orc.balance_weight([3.0, 1.0, 0], [1.0, 1.0, 0], [1, 1, 0], 0, True)
    assert w1 == pytest.approx(0.5) and w2 == pytest.approx(0.75)


# ----------------------------------------------------------- count rule (Eq. 2)
def test_vertex_count_three_cases_and_clamp(orc):
    """Sec. 3.1 'Optimization': beta = beta_RR if beta_RR < 1, else beta_S if
    beta_S > 1, else 1; clamped to [0.05, 20] (Sec. 4.1).  Grey inputs reduce to
    the scalar formula T / I * q."""
    one = np.ones(3)
    I = np.ones(3, np.float32)
    g = lambda x: np.full(3, x, np.float32)
    # RR regime
    assert orc.vertex_count(g(0.5), g(0.2), one, I) == pytest.approx(0.5, rel=1e-7)
    # splitting regime
    assert orc.vertex_count(g(4.0), g(3.0), one, I) == pytest.approx(3.0, rel=1e-7)
    # disagreement: RR says >= 1, S says <= 1 -> one sample
    assert orc.vertex_count(g(1.5), g(0.5), one, I) == 1.0
    # throughput and pixel estimate scale the factors
    assert orc.vertex_count(g(0.5), g(0.1), 0.5 * one, g(2.0)) == pytest.approx(0.125, rel=1e-7)
    # clamp
    assert orc.vertex_count(g(1e-4), g(0.0), one, I) == pytest.approx(0.05)
    assert orc.vertex_count(g(100.0), g(90.0), one, I) == pytest.approx(20.0)
    # colour: root mean square over channels of the per-channel counts
    q = np.array([0.3, 0.6, 0.9], np.float32)
    rms = math.sqrt((0.3 ** 2 + 0.6 ** 2 + 0.9 ** 2) / 3)
    assert orc.vertex_count(q, q * 0.5, one, I) == pytest.approx(rms, rel=1e-6)


# --------------------------------------------------------- fixed point (App. A)
def _scalar_moments(beta, E, V, C, VD, CD):
    """Proxy model (Sec. 3 'Optimization', EARS simplification): technique
    variance M2/beta - E^2 for beta < 1, V/beta otherwise."""
    var = 0.0
    for b, e, v in zip(beta, E, V):
        m2 = v + e * e
        var += (m2 / b - e * e) if b < 1 else v / b
    return var + VD, float(np.dot(beta, C)) + CD


def _stats_for(E, V, C, n=1e6):
    """Per-cell statistics whose moments are exactly (E, E^2 + V, C)."""
    st = np.zeros((1, 3, 8))
    for t in range(len(E)):
        st[0, t, 0] = n
        st[0, t, 1:4] = n * E[t]
        st[0, t, 4:7] = n * (V[t] + E[t] ** 2)
        st[0, t, 7] = n * C[t]
    return st


def _fixed_point(orc, E, V, C, VD, CD, beta0, steps):
    tech = (1 << len(E)) - 1
    beta = np.array(beta0, float)
    q_rr = np.zeros((1, 3, 3), np.float32)
    q_s = np.zeros((1, 3, 3), np.float32)
    valid = np.zeros((1, 3), np.uint8)
    hist = [beta.copy()]
    for _ in range(steps):
        VI, CI = _scalar_moments(beta, E, V, C, VD, CD)
        q_rr, q_s, valid = orc.update_counts(_stats_for(E, V, C), VI, CI, tech, q_rr, q_s, valid)
        beta = np.array([orc.vertex_count(q_rr[0, t], q_s[0, t], np.ones(3), np.ones(3, np.float32))
                         for t in range(len(E))])
        hist.append(beta.copy())
    return beta, hist


def test_fixed_point_reaches_budget_unaware_optimum(orc):
    """App. A.3: for budget-unaware weights the optimum is
    beta_t* = sqrt(C_D V_t / (V_D C_t)) (the lambda-line argument with
    lambda = sqrt(C_D / V_D)); the update of Eq. 2 converges to it, and is close
    to optimal efficiency within about five steps (Fig. 1DConvergence)."""
    E, V, C = [1.0, 1.0], [40.0, 12.0], [1.0, 30.0]
    VD, CD = 1.0, 4.0
    star = np.sqrt(CD * np.array(V) / (VD * np.array(C)))
    assert np.all(star > 1)  # splitting regime, where the closed form holds
    beta, hist = _fixed_point(orc, E, V, C, VD, CD, [1.0, 1.0], 300)
    assert beta == pytest.approx(star, rel=1e-5)
    ieff = lambda b: np.prod(_scalar_moments(b, E, V, C, VD, CD))
    opt = ieff(star)
    assert ieff(hist[5]) <= opt * 1.05


def test_fixed_point_matches_grid_search_mixed_regime(orc):
    """A case where one technique ends in Russian roulette and one splits:
    an exhaustive grid over [0.05, 20]^2 of the proxy's inverse efficiency has its
    minimum where the fixed point lands (to grid resolution)."""
    E, V, C = [0.05, 2.0], [0.2, 30.0], [6.0, 1.0]
    VD, CD = 0.5, 3.0
    beta, _ = _fixed_point(orc, E, V, C, VD, CD, [1.0, 1.0], 200)
    grid = np.exp(np.linspace(np.log(0.05), np.log(20.0), 400))
    best, arg = np.inf, None
    for b0 in grid:
        for b1 in grid:
            v = np.prod(_scalar_moments([b0, b1], E, V, C, VD, CD))
            if v < best:
                best, arg = v, (b0, b1)
    step = grid[1] / grid[0]
    assert beta[0] < 1 and beta[1] > 1
    assert arg[0] / step <= beta[0] <= arg[0] * step
    assert arg[1] / step <= beta[1] <= arg[1] * step


def test_update_fallbacks(orc):
    """Readings: cells with fewer than two samples or zero cost keep their
    previous factors; V_I <= 1e-12 keeps everything."""
    st = np.zeros((3, 3, 8))
    st[0, 0] = [1, 1, 1, 1, 1, 1, 1, 1]                  # n < 2
    st[1, 0] = [4, 4, 4, 4, 8, 8, 8, 0]                  # cost 0
    st[2, 0] = [4, 4, 4, 4, 8, 8, 8, 8]                  # valid
    q_rr = np.full((3, 3, 3), 7.0, np.float32)
    q_s = np.full((3, 3, 3), 5.0, np.float32)
    valid = np.zeros((3, 3), np.uint8)
    a, b, v = orc.update_counts(st, 0.5, 2.0, 1, q_rr, q_s, valid)
    assert np.all(a[:2] == 7.0) and np.all(v[:2] == 0)
    # cell 2: m1 = 1, m2 = 2, var = 1, C_t = 2 -> q_rr = sqrt(2/2 * 2/0.5) = 2, q_s = sqrt(1/0.5)
    assert a[2, 0] == pytest.approx([2.0] * 3) and b[2, 0] == pytest.approx([math.sqrt(2.0)] * 3)
    assert v[2, 0] == 1 and v[2, 1] == 0
    a, b, v = orc.update_counts(st, 1e-13, 2.0, 1, q_rr, q_s, valid)
    assert np.all(a == 7.0) and np.all(v == 0)


# ----------------------------------------------------------------------- BSDFs
def _sphere_grid(n):
    """Midpoint quadrature over the sphere (z, phi) -> directions, weights."""
    z = -1 + 2 * (np.arange(n) + 0.5) / n
    ph = 2 * np.pi * (np.arange(2 * n) + 0.5) / (2 * n)
    Z, P = np.meshgrid(z, ph, indexing="ij")
    s = np.sqrt(1 - Z ** 2)
    d = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    w = (2.0 / n) * (2 * np.pi / (2 * n))
    return d, w


def _mat_scene(mat_rows):
    sc = W.box_scene(2, 2)
    sc.materials = np.asarray(mat_rows, np.float64).reshape(-1, 8)
    return sc


@pytest.mark.parametrize("mat", [[0, 0.8, 0.5, 0.2, 0, 0, 0, 0],
                                 [1, 0.9, 0.6, 0.3, 0.3, 0, 0, 0],
                                 [1, 1.0, 1.0, 1.0, 0.1, 0, 0, 0]])
def test_bsdf_sampling_density_consistency(orc, mat):
    """The sampling routine and the pdf agree: the probability that a sample is
    valid equals the integral of the pdf over the upper hemisphere, and a
    chi-square test over direction bins accepts the sample histogram.  Lambert
    sampling is cosine-weighted (f cos / p = albedo)."""
    sc = _mat_scene([mat])
    th = 0.6
    wo = np.array([math.sin(th), 0.0, math.cos(th)])
    dirs, w = _sphere_grid(200)
    pdf = np.array([orc.bsdf_eval_local(sc, 0, wo, d)[1] for d in dirs[dirs[:, 2] > 0]])
    integral = pdf.sum() * w
    n = 96
    u = (np.arange(n) + 0.5) / n
    ok = []
    samples = []
    for a in u:
        for b in u:
            good, wi, p = orc.bsdf_sample_local(sc, 0, wo, a, b)
            ok.append(good)
            if good:
                samples.append(wi)
                f, p2 = orc.bsdf_eval_local(sc, 0, wo, wi)
                assert p == pytest.approx(p2, rel=1e-9)
                if mat[0] == 0:
                    assert f / p == pytest.approx(mat[1:4], rel=1e-9)
    assert integral == pytest.approx(np.mean(ok), abs=4e-3)
    # chi-square over 8 x 8 (cos theta, phi) bins of the upper hemisphere
    s = np.array(samples)
    zb = np.minimum((s[:, 2] * 8).astype(int), 7)
    pb = np.minimum(((np.arctan2(s[:, 1], s[:, 0]) % (2 * np.pi)) / (2 * np.pi) * 8).astype(int), 7)
    counts = np.bincount(zb * 8 + pb, minlength=64)
    up = dirs[:, 2] > 0
    du = dirs[up]
    zb2 = np.minimum((du[:, 2] * 8).astype(int), 7)
    pb2 = np.minimum(((np.arctan2(du[:, 1], du[:, 0]) % (2 * np.pi)) / (2 * np.pi) * 8).astype(int), 7)
    exp_p = np.bincount(zb2 * 8 + pb2, weights=pdf * w, minlength=64)
    expected = exp_p * n * n
    m = expected > 5
    chi2 = ((counts[m] - expected[m]) ** 2 / expected[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_ggx_reciprocity_and_energy(orc):
    """f(wo, wi) = f(wi, wo); with F0 = 1 the directional albedo is at most 1
    and approaches 1 for a smooth surface at normal incidence (single
    scattering with height-correlated masking)."""
    sc = _mat_scene([[1, 1.0, 1.0, 1.0, 0.2, 0, 0, 0], [1, 1.0, 1.0, 1.0, 0.02, 0, 0, 0]])
    rng = np.random.default_rng(5)
    for _ in range(50):
        a = rng.normal(size=3); a[2] = abs(a[2]); a /= np.linalg.norm(a)
        b = rng.normal(size=3); b[2] = abs(b[2]); b /= np.linalg.norm(b)
        fa, _ = orc.bsdf_eval_local(sc, 0, a, b)
        fb, _ = orc.bsdf_eval_local(sc, 0, b, a)
        assert fa[0] / b[2] == pytest.approx(fb[0] / a[2], rel=1e-9)
    for mat, lo in ((0, 0.9), (1, 0.995)):
        wo = np.array([0.0, 0.0, 1.0])
        n = 128
        acc = 0.0
        for x in (np.arange(n) + 0.5) / n:
            for y in (np.arange(n) + 0.5) / n:
                good, wi, p = orc.bsdf_sample_local(sc, mat, wo, x, y)
                if good:
                    f, _ = orc.bsdf_eval_local(sc, mat, wo, wi)
                    acc += f[0] / p
        alb = acc / (n * n)
        assert lo <= alb <= 1.0 + 1e-3


def test_guide_pdf_and_sampling(orc):
    """The guide's pdf integrates to one over the sphere and samples land in bin
    b with probability P_b (the CDF difference)."""
    cdf = W.random_guide_cdf(1, seed=9)[0]
    dirs, w = _sphere_grid(256)
    integral = sum(orc.guide_pdf(cdf, d) for d in dirs) * w
    assert integral == pytest.approx(1.0, abs=2e-3)
    P = np.diff(np.concatenate([[0.0], cdf.astype(np.float64)]))
    n = 4096
    counts = np.zeros(256)
    for k in range(n):
        wv, p = orc.guide_sample(cdf, (k + 0.5) / n, 0.37, 0.61)
        z = wv[2]
        ph = math.atan2(wv[1], wv[0]) % (2 * math.pi)
        b = min(int((z + 1) * 8), 15) * 16 + min(int(ph / (2 * math.pi) * 16), 15)
        counts[b] += 1
        assert p == pytest.approx(P[b] * 256 / (4 * math.pi), rel=1e-6)
    assert np.abs(counts / n - P).max() < 2.0 / n + 1e-6


def test_guide_update(orc):
    h = np.zeros((2, 256))
    h[1, 17] = 5.0
    cdf = orc.guide_update(h)
    P = np.diff(np.concatenate([np.zeros((2, 1)), cdf.astype(np.float64)], axis=1), axis=1)
    assert P[0] == pytest.approx(np.full(256, 1 / 256), abs=1e-6)
    assert P[1, 17] == pytest.approx(0.9 + 0.1 / 256, abs=1e-6)
    assert P[1, 3] == pytest.approx(0.1 / 256, abs=1e-6)
    assert cdf[:, -1].tolist() == [1.0, 1.0]


# ----------------------------------------------------------------- image stats
def test_image_stats_small_case(orc):
    """3 x 2 image worked by hand: box filter over in-image neighbours, V_I as the
    mean squared relative deviation with the sample clamped at 50 x estimate."""
    img = np.array([[1, 1, 1], [2, 2, 2], [3, 3, 3], [4, 4, 4], [5, 5, 5], [600, 600, 600]], float)
    vi, rs, est = orc.image_stats(3, 2, img, np.zeros_like(img), 0)
    # pixel (0,0): neighbours (0,0),(1,0),(0,1),(1,1) -> (1 + 2 + 4 + 5) / 4 = 3
    assert est[0, 0] == pytest.approx(3.0)
    # pixel (1,0): all six pixels -> 615 / 6
    assert est[1, 0] == pytest.approx(615 / 6)
    # pixel (2,1): (2,3,5,600)/4
    assert est[5, 0] == pytest.approx(610 / 4)
    manual = 0.0
    for p in range(6):
        e = est[p, 0]
        i = min(img[p, 0], 50 * e)
        manual += ((i - e) / e) ** 2
    assert vi == pytest.approx(manual / 6)
    # a constant image is its own estimate: zero variance
    c = np.full((12, 3), 0.7)
    vi2, _, est2 = orc.image_stats(4, 3, c, np.zeros_like(c), 0)
    assert vi2 == pytest.approx(0.0, abs=1e-20) and est2 == pytest.approx(0.7)
    # running mean over iterations and the floor at 1e-3 x channel mean
    z = np.zeros((4, 3)); z[0] = 8.0
    vi3, rs3, est3 = orc.image_stats(4, 1, z, np.full((4, 3), 8.0), 1)
    assert rs3[0, 0] == 16.0 and rs3[3, 0] == 8.0
    assert est3[3, 0] == pytest.approx(4.0)   # mean of (4, 4) from pixels 2 and 3


# --------------------------------------------------------- whole-render pins
def _mean_and_sem(vals):
    v = np.asarray(vals)
    return v.mean(), v.std(ddof=1) / math.sqrt(len(v))


@pytest.mark.parametrize("albedo,D", [(0.5, 3), (0.8, 4)])
@pytest.mark.parametrize("counts", ["beta1", "random"])
def test_furnace_closed_form(orc, albedo, D, counts):
    """Closed furnace: every pixel's expectation is Le (1 - a^D) / (1 - a),
    independent of the count field (Sec. 3 'Continuous sample counts': dividing
    by the real-valued beta keeps the estimator unbiased)."""
    sc = W.furnace_scene(albedo=albedo, radiance=1.5, width=12, height=12)
    cells = 4 ** 3
    q_rr, q_s, valid = W.random_count_fields(cells, seed=11, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=12, lo=0.5, hi=4.0)
    vals = []
    for it in range(60):
        kw = dict(grid_n=4, techniques=W.TECH_BSDF | W.TECH_NEE, max_depth=D, iteration=it)
        if counts == "random":
            kw.update(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
        vals.append(orc.render(sc, **kw).image.mean())
    m, se = _mean_and_sem(vals)
    expected = 1.5 * (1 - albedo ** D) / (1 - albedo)
    assert abs(m - expected) < 3.5 * se + 1e-9


@pytest.mark.parametrize("M", [1.5, 4.0])
def test_multiplicity_cap_keeps_the_furnace_and_bounds_the_tree(orc, M):
    """Path multiplicity cap: budgets limited to max(clamp_lo, M / P).  The
    furnace expectation is unchanged (it is one more count field), and the
    traced vertices per pixel and depth stay near M even where the uncapped
    field splits at every bounce."""
    albedo, D = 0.8, 5
    sc = W.furnace_scene(albedo=albedo, radiance=1.5, width=8, height=8)
    cells = 4 ** 3
    q_rr = np.full((cells, 3, 3), 40.0, np.float32)   # beta = 20 (the clamp) everywhere
    q_s = np.full((cells, 3, 3), 40.0, np.float32)
    valid = np.ones((cells, 3), np.uint8)
    est = np.full((sc.n_pixels, 3), 0.1, np.float32)
    kw = dict(grid_n=4, techniques=W.TECH_BSDF | W.TECH_NEE, max_depth=D, mode=orc.MODE_MARS, q_rr=q_rr,
              q_s=q_s, valid=valid, est=est, max_mult=M)
    vals, verts = [], []
    for it in range(40):
        r = orc.render(sc, iteration=it, **kw)
        vals.append(r.image.mean())
        verts.append(r.vertices / sc.n_pixels)
    m, se = _mean_and_sem(vals)
    expected = 1.5 * (1 - albedo ** D) / (1 - albedo)
    assert abs(m - expected) < 3.5 * se + 1e-9
    # expected traced vertices per pixel: at most 1 + M per later depth (and
    # at least the camera ray)
    assert np.mean(verts) <= 1 + (D - 1) * M * 1.1
    uncapped = orc.render(sc, iteration=0, **dict(kw, max_mult=0.0))
    assert uncapped.vertices / sc.n_pixels > 20 * np.mean(verts)


@pytest.mark.parametrize("weights", [0, 1])
@pytest.mark.parametrize("counts", ["beta1", "random"])
def test_polygon_light_irradiance_closed_form(orc, weights, counts):
    """Floor under a square Lambertian emitter, two segments: the pixel value
    is albedo / pi x irradiance, and the irradiance of a rectangle seen from a
    point on its axis is the classical corner form factor sum (Lambert).  This
    pins the NEE density (light pmf, area and cosine Jacobian), the BSDF density
    and their multi-sample MIS combination."""
    sc = W.area_light_plane_scene(width=6, height=6, albedo=0.5, radiance=2.0)
    eps = 1e-4 * 2.0        # ray offset = 1e-4 x largest scene extent (the floor is 2 wide)
    c = 1.0 - eps
    X = 0.5 / c

    def corner(x, y):
        return (x / math.sqrt(1 + x * x) * math.atan(y / math.sqrt(1 + x * x))
                + y / math.sqrt(1 + y * y) * math.atan(x / math.sqrt(1 + y * y))) / (2 * math.pi)

    expected = 0.5 / math.pi * (math.pi * 2.0 * 4 * corner(X, X))
    q_rr, q_s, valid = W.random_count_fields(8, seed=21, lo=0.2, hi=6.0, p_valid=1.0)
    est = np.full((sc.n_pixels, 3), 0.25, np.float32)
    vals = []
    for it in range(150):
        kw = dict(grid_n=2, techniques=W.TECH_BSDF | W.TECH_NEE, max_depth=2, iteration=it, weights=weights)
        if counts == "random":
            kw.update(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
        vals.append(orc.render(sc, **kw).image.mean())
    m, se = _mean_and_sem(vals)
    assert abs(m - expected) < 3.5 * se


def test_unbiased_under_random_counts_box(orc):
    """Box scene: the image mean under a random count field equals the image
    mean with beta = 1 within the combined 3.5 sigma (App. A.1 'Unbiasedness')."""
    cfg = W.config_box(16, 16)
    cells = cfg.n_cells
    q_rr, q_s, valid = W.random_count_fields(cells, seed=31, lo=0.05, hi=3.0)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=32, lo=0.05, hi=1.0)
    a, b = [], []
    for it in range(150):
        kw = dict(grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth, iteration=it)
        a.append(orc.render(cfg.scene, **kw).image.mean(0))
        b.append(orc.render(cfg.scene, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                            seed=7, **kw).image.mean(0))
    a, b = np.array(a), np.array(b)
    for ch in range(3):
        ma, sa = _mean_and_sem(a[:, ch])
        mb, sb = _mean_and_sem(b[:, ch])
        assert abs(ma - mb) < 3.5 * math.hypot(sa, sb)


def test_guided_technique_unbiased(orc):
    """Three techniques (BSDF, NEE, guided) on a small crop of the guided room:
    with a random guide distribution and random counts the image mean matches
    BSDF+NEE alone (the guided technique only redistributes samples)."""
    sc = W.guided_room_scene(seed=0, width=8, height=8, n_spheres=16)
    cells = 4 ** 3
    cdf = W.random_guide_cdf(cells, seed=41, sparsity=0.5)
    q_rr, q_s, valid = W.random_count_fields(cells, seed=42, lo=0.1, hi=2.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=43, lo=0.2, hi=2.0)
    a, b = [], []
    for it in range(120):
        kw = dict(grid_n=4, max_depth=4, iteration=it)
        a.append(orc.render(sc, techniques=3, **kw).image.mean())
        b.append(orc.render(sc, techniques=7, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                            guide_cdf=cdf, seed=5, **kw).image.mean())
    ma, sa = _mean_and_sem(a)
    mb, sb = _mean_and_sem(b)
    assert abs(ma - mb) < 3.5 * math.hypot(sa, sb)


def test_statistics_bookkeeping(orc):
    """With beta = 1 every estimator vertex draws one sample per technique, so
    n per technique equals the number of estimator vertices; rays (the cost
    unit) are the camera rays plus every drawn sample; a technique's summed
    cost is at least its sample count."""
    cfg = W.config_box(16, 16)
    r = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth)
    nv = r.counters[2]
    n = r.stats[:, :, 0].sum(0)
    assert n[0] == nv and n[1] == nv and n[2] == 0
    assert r.rays == cfg.scene.n_pixels + n.sum()
    assert np.all(r.stats[:, 1, 7] == r.stats[:, 1, 0])      # NEE: one ray per sample
    assert np.all(r.stats[:, 0, 7] >= r.stats[:, 0, 0])
    # estimator vertices never exceed the traced vertices
    assert r.counters[2] <= r.counters[1]


# --------------------------------------------------------- adaptive octree
def _leaf_boxes(nodes, lmax=10):
    """brute force: every leaf's integer box at the finest level, by walking the tree"""
    boxes = {}
    stack = [(0, 0, 0, 0, 0)]
    while stack:
        k, lvl, x, y, z = stack.pop()
        v = int(nodes[k])
        size = 1 << (lmax - lvl)
        if v < 0:
            boxes[~v] = (x, y, z, size)
            continue
        half = size // 2
        for o in range(8):
            stack.append((v + o, lvl + 1, x + (o & 1) * half, y + ((o >> 1) & 1) * half, z + ((o >> 2) & 1) * half))
    return boxes


def _random_refinement(orc, grid_n, max_leaves, rounds, seed):
    rng = np.random.default_rng(seed)
    nodes, nn, nl, lvl, lnode = orc.octree_init(grid_n, max_leaves)
    q_rr = rng.uniform(0.1, 3, (max_leaves, 3, 3)).astype(np.float32)
    q_s = (q_rr * 0.5).astype(np.float32)
    valid = (rng.uniform(size=(max_leaves, 3)) < 0.7).astype(np.uint8)
    hist = rng.exponential(size=(max_leaves, 256))
    cdf = np.cumsum(hist, 1) / hist.sum(1, keepdims=True)
    cdf = cdf.astype(np.float32)
    for r in range(rounds):
        stats = np.zeros((max_leaves, 3, 8))
        stats[:nl, :, 0] = rng.integers(0, 60, size=(nl, 3))
        (nodes, nn2, nl2, lvl, lnode, q_rr2, q_s2, valid2, hist2, cdf2, sp) = orc.octree_refine(
            max_leaves, 100.0, stats, nodes, nn, nl, lvl, lnode, q_rr, q_s, valid, hist, cdf)
        # the rule: leaves in id order with >= 100 samples split while the cap allows
        want = [L for L in range(nl) if stats[L, :, 0].sum() >= 100 and lvl[L] < 10]
        assert sp == min(len(want), (max_leaves - nl) // 7)
        assert nl2 == nl + 7 * sp and nn2 == nn + 8 * sp
        for s_, L in enumerate(want[:sp]):
            for o in range(1, 8):
                c = nl + 7 * s_ + o - 1
                assert np.array_equal(q_rr2[c], q_rr2[L]) and np.array_equal(valid2[c], valid2[L])
                assert np.array_equal(cdf2[c], cdf2[L])
        nn, nl, q_rr, q_s, valid, hist, cdf = nn2, nl2, q_rr2, q_s2, valid2, hist2, cdf2
    return nodes, nn, nl, lvl, q_rr, q_s, valid, cdf


def test_octree_refinement_rule_and_partition(orc):
    """Refinement follows the stated rule (leaves in id order with enough
    samples, cap on the leaf count, children inherit counts and guide), and the
    leaves always partition the scene box: the descent finds, for random
    points, the unique leaf whose box contains them."""
    nodes, nn, nl, lvl, *_ = _random_refinement(orc, 4, 640, 3, seed=7)
    assert nl > 64
    boxes = _leaf_boxes(nodes)
    assert sorted(boxes) == list(range(nl))
    vol = sum(b[3] ** 3 for b in boxes.values())
    assert vol == 1024 ** 3                      # the leaves tile the box exactly
    rng = np.random.default_rng(8)
    lo, ext = np.array([-1.0, 0.5, 2.0]), np.array([3.0, 2.0, 5.0])
    for _ in range(400):
        p = lo + ext * rng.uniform(0, 1, 3)
        leaf = orc.octree_cell(lo, ext, nodes, p)
        x, y, z, size = boxes[leaf]
        idx = np.clip(np.floor(((p - lo) / ext).astype(np.float32) * np.float32(1024)), 0, 1023)
        assert x <= idx[0] < x + size and y <= idx[1] < y + size and z <= idx[2] < z + size
        assert lvl[leaf] == 10 - int(np.log2(size))


def test_octree_without_splits_is_the_grid_and_refined_tree_is_unbiased(orc):
    """The initial octree numbers its leaves like the uniform grid, so an
    unrefined octree renders exactly the grid's image and statistics; under a
    refined tree with random counts the box's image mean is that of beta = 1
    (any count field keeps the estimator unbiased)."""
    cfg = W.config_box(24, 20)
    kw = dict(grid_n=8, techniques=cfg.techniques, max_depth=cfg.max_depth, seed=1)
    nodes, nn, nl, lvl, lnode = orc.octree_init(8, 2048)
    a = orc.render(cfg.scene, iteration=0, **kw)
    b = orc.render(cfg.scene, iteration=0, octree=(nodes, 2048), **kw)
    assert np.array_equal(a.image, b.image) and np.array_equal(a.stats, b.stats[:512])
    nodes, nn, nl, lvl, q_rr, q_s, valid, cdf = _random_refinement(orc, 8, 2048, 2, seed=9)
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=10, lo=0.05, hi=0.5)
    ref, mars = [], []
    for it in range(30):
        ref.append(orc.render(cfg.scene, iteration=it, **kw).image.mean())
        mars.append(orc.render(cfg.scene, iteration=it, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid,
                               est=est, octree=(nodes, 2048), **kw).image.mean())
    m1, s1 = _mean_and_sem(ref)
    m2, s2 = _mean_and_sem(mars)
    assert abs(m1 - m2) < 3.5 * math.sqrt(s1 ** 2 + s2 ** 2)


def _flat_mean_case(W, H, n_prev, m, bright):
    """An image equal to the colour m everywhere except the pixels of `bright`
    (index -> colour), with a running sum chosen so that the new running mean is
    m at every pixel: the pixel estimate is then m exactly (a box filter of a
    constant, above the 1e-3 floor), and a pixel's V_I term is
    sum_ch ((I_ch - m_ch) / m_ch)^2."""
    n = W * H
    img = np.tile(np.asarray(m, np.float64), (n, 1))
    for p, c in bright.items():
        img[p] = c
    run_sum = (n_prev + 1) * np.tile(np.asarray(m, np.float64), (n, 1)) - img
    return img, run_sum


def test_brightest_pixel_rejection_closed_form(orc):
    """Sec. 5.1 "Implementation": the K brightest pixels of a pass leave its V_I.
    On a flat image with K bright outliers V_I is 0 when all K are dropped; with
    K - 1 dropped exactly the dimmest outlier remains, unclamped; brightness is
    luminance, so a strongly blue pixel of low luminance stays in the mean while a
    brighter green one is dropped; and K = 0 keeps the clamped estimate."""
    W, H, n_prev = 8, 6, 3
    n = W * H
    m = np.array([0.5, 0.3, 0.2])
    alphas = {5: 100.0, 17: 60.0, 30: 80.0}   # I = alpha * m
    img, rs = _flat_mean_case(W, H, n_prev, m, {p: a * m for p, a in alphas.items()})
    vi3, _, est = orc.image_stats(W, H, img, rs, n_prev, outlier=50.0, drop_k=3)
    assert np.allclose(est, np.tile(m, (n, 1)), rtol=1e-12)
    assert vi3 == pytest.approx(0.0, abs=1e-24)
    vi2, _, _ = orc.image_stats(W, H, img, rs, n_prev, outlier=50.0, drop_k=2)
    assert vi2 == pytest.approx(3 * (60.0 - 1) ** 2 / (3 * (n - 2)), rel=1e-12)
    vi1, _, _ = orc.image_stats(W, H, img, rs, n_prev, outlier=50.0, drop_k=1)
    assert vi1 == pytest.approx(3 * ((60.0 - 1) ** 2 + (80.0 - 1) ** 2) / (3 * (n - 1)), rel=1e-12)
    # K = 0: the clamp at 50 x estimate bounds every outlier term at 3 * 49^2
    vi0, _, _ = orc.image_stats(W, H, img, rs, n_prev, outlier=50.0, drop_k=0)
    assert vi0 == pytest.approx(3 * (3 * 49.0 ** 2) / (3 * n), rel=1e-12)
    # luminance decides: pixel 9 is blue (B = 40 m_B, luminance ~ 0.6), pixel 21
    # green (G = 5 m_G, luminance ~ 1.3); K = 1 drops the green one
    img2, rs2 = _flat_mean_case(W, H, n_prev, m, {9: m * np.array([1.0, 1.0, 40.0]),
                                                  21: m * np.array([1.0, 5.0, 1.0])})
    v, _, _ = orc.image_stats(W, H, img2, rs2, n_prev, drop_k=1)
    assert v == pytest.approx(39.0 ** 2 / (3 * (n - 1)), rel=1e-12)


def test_inverse_variance_combination_closed_form(orc):
    """Sec. 5.1: iterations combine with weights 1 / V_I.  Constant images a_i
    with variances V_i give sum(a_i / V_i) / sum(1 / V_i); equal variances give
    the plain mean; an iteration with 100x the variance barely counts."""
    imgs = [np.full((4, 3), a) for a in (1.0, 2.0, 4.0)]
    out, w = orc.combine(imgs, [0.5, 0.25, 1.0])
    assert w == pytest.approx(2 + 4 + 1)
    assert np.allclose(out, (1 / 0.5 + 2 / 0.25 + 4 / 1.0) / 7.0)
    out, _ = orc.combine(imgs, [0.3, 0.3, 0.3])
    assert np.allclose(out, np.mean([1.0, 2.0, 4.0]))
    out, _ = orc.combine([np.full(3, 1.0), np.full(3, 10.0)], [1.0, 100.0])
    assert np.allclose(out, (1.0 + 0.1) / 1.01)


# ------------------------------------------- local statistics (Sec. 4.1)
def _furnace_bsdf_only(orc, albedo, radiance, D, **kw):
    sc = W.furnace_scene(albedo=albedo, radiance=radiance, width=10, height=10)
    return sc, orc.render(sc, grid_n=2, techniques=W.TECH_BSDF, max_depth=D, **kw)


@pytest.mark.parametrize("counts", ["beta1", "random"])
def test_local_moments_closed_form_furnace_depth2(orc, counts):
    """Sec. 4.1 "Local estimates": every recorded sample is the technique's
    primary estimate <L_r,t> itself (not divided by its budget).  In the closed
    furnace with BSDF sampling alone and D = 2, a sample drawn at the first
    vertex hits a wall whose emission ends the path, so its value is
    f cos / p * Le = a Le exactly (cosine sampling of a Lambertian surface), under
    any count field: m1 = a Le, m2 = (a Le)^2, var = 0, and its cost is the one
    ray it traced, C_t = 1.  The number of samples is the sum of the rounded
    budgets, one per pixel without learned counts."""
    a, Le = 0.625, 1.5                          # exact in float32, as the scene stores them
    kw = {}
    if counts == "random":
        q_rr, q_s, valid = W.random_count_fields(8, seed=61, lo=0.1, hi=6.0, p_valid=1.0)
        est = W.random_pixel_estimate(100, seed=62, lo=0.5, hi=3.0)  # clamp limit 50 est >> a Le
        kw = dict(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
    sc, r = _furnace_bsdf_only(orc, a, Le, 2, **kw)
    st = r.stats[:, 0, :].sum(0)
    n = st[0]
    if counts == "beta1":
        assert n == sc.n_pixels
    else:
        assert n != sc.n_pixels and n == r.rays - sc.n_pixels
    assert r.stats[:, 1:, 0].sum() == 0.0
    m1 = st[1:4] / n
    m2 = st[4:7] / n
    assert m1 == pytest.approx([a * Le] * 3, rel=1e-12)
    assert m2 == pytest.approx([(a * Le) ** 2] * 3, rel=1e-12)
    assert np.all(np.abs(m2 - m1 * m1) <= 1e-12 * (a * Le) ** 2)
    assert st[7] == n


def test_local_moments_closed_form_furnace_depth3(orc):
    """D = 3 in one cell without learned counts: a first-vertex sample is worth
    a (Le + a Le) (its child vertex's one sample a Le, divided by beta = 1) and
    costs 2 rays (its own and its child's sample); a second-vertex sample is
    worth a Le and costs 1.  So n = 2P, m1 = a Le (2 + a) / 2,
    m2 = (a Le)^2 ((1 + a)^2 + 1) / 2 and C_t = 3/2."""
    a, Le = 0.625, 1.25
    sc = W.furnace_scene(albedo=a, radiance=Le, width=8, height=8)
    r = orc.render(sc, grid_n=1, techniques=W.TECH_BSDF, max_depth=3)
    s = r.stats[0, 0]
    P = sc.n_pixels
    assert s[0] == 2 * P
    assert s[1:4] / s[0] == pytest.approx([a * Le * (2 + a) / 2] * 3, rel=1e-12)
    assert s[4:7] / s[0] == pytest.approx([(a * Le) ** 2 * ((1 + a) ** 2 + 1) / 2] * 3, rel=1e-12)
    assert s[7] / s[0] == 1.5


def test_outlier_clamp_binds_at_the_throughput_scaled_limit(orc):
    """Sec. 4.1 "Outlier clamping" (reading: a sample's image contribution
    T v stays below 50 times the pixel estimate, so v <= 50 I / T per channel).
    Furnace, D = 3, budgets 1 (no valid counts), pixel estimate c small enough
    that every sample is clamped: first-vertex samples (T = 1) record exactly
    50 c, second-vertex samples (T = a, the first bounce's f cos / p) record
    50 c / a.  Swapping T and I, or taking T from the parent, fails this."""
    a, Le = 0.5, 1.5
    c = np.float32(0.004)                      # 50 c / a = 0.4 < a Le = 0.75
    sc = W.furnace_scene(albedo=a, radiance=Le, width=8, height=8)
    P = sc.n_pixels
    cells = 2 ** 3
    est = np.full((P, 3), c, np.float32)
    r = orc.render(sc, grid_n=2, techniques=W.TECH_BSDF, max_depth=3, mode=orc.MODE_MARS,
                   q_rr=np.zeros((cells, 3, 3), np.float32), q_s=np.zeros((cells, 3, 3), np.float32),
                   valid=np.zeros((cells, 3), np.uint8), est=est)
    st = r.stats[:, 0, :].sum(0)
    lim1, lim2 = 50.0 * float(c), 50.0 * float(c) / a
    assert st[0] == 2 * P
    assert st[1:4] == pytest.approx([P * (lim1 + lim2)] * 3, rel=1e-9)
    assert st[4:7] == pytest.approx([P * (lim1 ** 2 + lim2 ** 2)] * 3, rel=1e-9)
    # the image itself is not clamped: each pixel is Le (1 + a + a^2)
    assert r.image == pytest.approx(np.full((P, 3), Le * (1 + a + a * a)), rel=1e-12)
    # the same render without a pixel estimate records the unclamped values
    r0 = orc.render(sc, grid_n=2, techniques=W.TECH_BSDF, max_depth=3)
    s0 = r0.stats[:, 0, :].sum(0)
    assert s0[1:4] == pytest.approx([P * (a * Le * (1 + a) + a * Le)] * 3, rel=1e-12)


def test_cost_counts_the_rays_of_a_sample_subtree(orc):
    """Sec. 4.1 (C_t, "path length generated"; reading: a sample costs its own
    ray plus every ray of its subtree).  Furnace with BSDF sampling alone,
    D = 3, random budgets: a first-vertex sample costs 1 plus its child vertex's
    sample count, a second-vertex sample 1, so the summed cost is
    n_total + n_2 with n_1 = (estimator vertices - pixels) and n_2 = n_total - n_1."""
    a, Le = 0.75, 1.0
    cells = 2 ** 3
    q_rr, q_s, valid = W.random_count_fields(cells, seed=71, lo=0.2, hi=5.0, p_valid=1.0)
    for it in range(3):
        est = W.random_pixel_estimate(100, seed=72 + it, lo=0.3, hi=2.0)
        sc, r = _furnace_bsdf_only(orc, a, Le, 3, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                                   iteration=it)
        st = r.stats[:, 0, :].sum(0)
        n_tot = st[0]
        n1 = r.counters[2] - sc.n_pixels
        n2 = n_tot - n1
        assert n1 > 0 and n2 > 0 and n1 != n2
        assert st[7] == n_tot + n2
        assert r.rays == sc.n_pixels + n_tot


def test_recorded_values_add_up_to_the_image(orc):
    """With budgets 1 the secondary estimate at the first vertex is the plain
    sum of one BSDF and one NEE sample value, so in the furnace (D = 2, every
    camera ray sees a wall emitting Le) the image summed over pixels equals
    P Le plus the recorded value sums of both techniques."""
    sc = W.furnace_scene(albedo=0.375, radiance=2.0, width=12, height=9)
    r = orc.render(sc, grid_n=2, techniques=W.TECH_BSDF | W.TECH_NEE, max_depth=2)
    s = r.stats.sum(0)
    assert s[0, 0] == sc.n_pixels and s[1, 0] == sc.n_pixels
    lhs = r.image.sum(0)
    rhs = sc.n_pixels * 2.0 + s[0, 1:4] + s[1, 1:4]
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ------------------------------------- fixed point in a render (App. A.3)
def _relvar_cost(vals, counters):
    v = vals[:, 0]
    m = v.mean()
    return float(np.mean(((v - m) / m) ** 2)), float(counters[0] / len(v)), float(m)


@pytest.mark.parametrize("weights", [0, 1])
def test_fixed_point_in_a_render_reaches_the_grid_search_optimum(orc, weights):
    """Sec. 3 "Fixed point" and App. A.3 on a rendered case small enough for
    brute force: one pixel, one cell, D = 2 (the only estimator vertex is the
    first, where T = 1 and the pixel estimate is constant, so one (beta_BSDF,
    beta_NEE) pair describes the whole count field).  The fixed-point iteration
    runs as in a render: each step renders the pixel, records the local
    statistics, takes V_I and C_I from the step's samples and updates the
    counts.  Its efficiency 1 / (relative variance x rays) is then measured
    beside a brute-force grid of constant budget pairs (common random numbers)
    and must reach 95 % of the grid maximum.  The light is partly occluded so
    that both techniques are noisy; a nearly deterministic technique instead
    lands on fractional splitting whose rounding noise the proxy drops (the
    paper's simplification for beta > 1)."""
    sc = W.occluded_light_plane_scene(width=1, height=1)
    kw = dict(grid_n=1, techniques=W.TECH_BSDF | W.TECH_NEE, max_depth=2, weights=weights, outlier=1e30)
    vals, stats, ctr = orc.render_samples(sc, 8192, seed=11, **kw)
    rv, ci, m = _relvar_cost(vals, ctr)
    run_sum, n_run = vals[:, 0].sum(), len(vals)
    q_rr = np.zeros((1, 3, 3), np.float32)
    q_s = np.zeros((1, 3, 3), np.float32)
    valid = np.zeros((1, 3), np.uint8)
    for step in range(28):
        I = np.float32(run_sum / n_run)
        q_rr, q_s, valid = orc.update_counts(stats, rv, ci, 3, q_rr, q_s, valid)
        vals, stats, ctr = orc.render_samples(sc, 8192, seed=100 + step, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s,
                                              valid=valid, est=np.full((1, 3), I, np.float32), **kw)
        run_sum += vals[:, 0].sum()
        n_run += len(vals)
        v = vals[:, 0]
        rv = float(np.mean(((v - I) / I) ** 2))
        ci = float(ctr[0] / len(v))
    I = np.float32(run_sum / n_run)
    beta = [orc.vertex_count(q_rr[0, t], q_s[0, t], np.ones(3), np.full(3, I, np.float32)) for t in range(2)]
    N = 16384
    est = np.full((1, 3), I, np.float32)

    def efficiency(qr, qs, vd):
        vals, _, ctr = orc.render_samples(sc, N, seed=7, mode=orc.MODE_MARS, q_rr=qr, q_s=qs, valid=vd, est=est,
                                          collect=False, **kw)
        rv, c, _ = _relvar_cost(vals, ctr)
        return 1.0 / (rv * c)

    e_fp = efficiency(q_rr, q_s, valid)
    grid = 0.25 * 2.0 ** (0.75 * np.arange(9))
    best, arg = 0.0, None
    for bB in grid:
        for bN in grid:
            q = np.zeros((1, 3, 3), np.float32)
            q[0, 0, :] = bB * I
            q[0, 1, :] = bN * I
            e = efficiency(q, q, np.ones((1, 3), np.uint8))
            if e > best:
                best, arg = e, (bB, bN)
    assert e_fp >= 0.95 * best, (beta, arg, e_fp / best)


# ------------------------------------------------- the long oracle reference
def _box_reference():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "box_32x32_fixed_65536spp.txt")
    a = np.loadtxt(path)
    return a[:, :3], a[:, 3:]


def test_long_box_reference_agrees_with_a_fresh_oracle_render(orc):
    """The stored 65536-iteration reference (tests/golden/make_box_reference.py,
    written by the oracle alone) agrees with a fresh 256-iteration oracle render
    under other random numbers: with the per-iteration variance the reference
    stores (its variance of the mean x 65536), the squared differences divided
    by the variance of the difference average 1, and the image means agree
    within 4 sigma per channel."""
    ref, ref_var = _box_reference()
    cfg = W.config_box(32, 32)
    n, n_ref = 256, 65536
    s1 = np.zeros_like(ref)
    for it in range(n):
        r = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                       mode=orc.MODE_FIXED, seed=4321, iteration=it, collect=False)
        s1 += r.image
    m = s1 / n
    var_d = ref_var * n_ref / n + ref_var
    ok = var_d > 0
    assert np.all(m[~ok] == ref[~ok])          # pixels that never vary (always black)
    z2 = (m[ok] - ref[ok]) ** 2 / var_d[ok]
    assert 0.85 < z2.mean() < 1.2, z2.mean()
    assert np.all(np.abs(m.sum(0) - ref.sum(0)) < 4 * np.sqrt(var_d.sum(0)))


def test_long_guided_room_reference_agrees_with_a_fresh_oracle_render(orc):
    """The stored 65536-iteration reference of the guided room's geometry at 32 x
    32 (tests/golden/make_box_reference.py --scene guided, written by the oracle
    alone) agrees with a fresh 512-iteration oracle render under other random
    numbers: the image mean within 4 sigma per channel, and most pixels within 2
    sigma (their values are heavy-tailed -- small glossy lobes and lights -- so
    the squared deviations do not average to one at this sample count)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "guided_room_32x32_fixed_65536spp.txt")
    a = np.loadtxt(path)
    ref, ref_var = a[:, :3], a[:, 3:]
    cfg = W.config_guided(32, 32)
    cdf = np.tile((np.arange(1, orc.GUIDE_BINS + 1) / orc.GUIDE_BINS).astype(np.float32), (cfg.n_cells, 1))
    n, n_ref = 512, 65536
    s1 = np.zeros_like(ref)
    for it in range(n):
        r = orc.render(cfg.scene, grid_n=cfg.grid_n, techniques=cfg.techniques, max_depth=cfg.max_depth,
                       mode=orc.MODE_FIXED, seed=4321, iteration=it, collect=False, guide_cdf=cdf)
        s1 += r.image
    m = s1 / n
    var_d = ref_var * n_ref / n + ref_var
    assert (var_d > 0).all()
    assert np.all(np.abs(m.sum(0) - ref.sum(0)) < 4 * np.sqrt(var_d.sum(0)))
    z = (m - ref) / np.sqrt(var_d)
    assert (np.abs(z) < 2).mean() > 0.9


# ----------------------------------------- bidirectional application (Sec. 5)
TECH_BDPT = W.TECH_BSDF | W.TECH_NEE | 8   # BSDF, NEE, light connection


@pytest.mark.parametrize("weights", [0, 1])
@pytest.mark.parametrize("counts", ["beta1", "random"])
def test_bidirectional_furnace_closed_form(orc, weights, counts):
    """Sec. 5: path tracing, NEE and connections to light subpaths combined
    with budget-aware (or -unaware) balance weights over every strategy of a
    full path.  The closed furnace keeps its closed form Le (1 - a^D)/(1 - a)
    under any count field: the weights of the strategies that sample a path
    sum to one and every technique divides by its real-valued budget."""
    albedo, D = 0.6, 5
    sc = W.furnace_scene(albedo=albedo, radiance=1.5, width=10, height=10)
    cells = 4 ** 3
    q_rr, q_s, valid = W.random_count_fields(cells, seed=111, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=112, lo=0.5, hi=4.0)
    vals = []
    for it in range(60):
        kw = dict(grid_n=4, techniques=TECH_BDPT, max_depth=D, iteration=it, weights=weights)
        if counts == "random":
            kw.update(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
        r = orc.render(sc, **kw)
        vals.append(r.image.mean())
    assert r.stats[:, 2, 0].sum() > 0     # light connection samples were drawn
    m, se = _mean_and_sem(vals)
    expected = 1.5 * (1 - albedo ** D) / (1 - albedo)
    assert abs(m - expected) < 3.5 * se + 1e-9


def test_bidirectional_unbiased_where_light_paths_matter(orc):
    """A heightfield lit by one small emitter hidden between two spheres (the
    bidirectional workload's geometry, small): with random count fields for
    all three techniques the image mean equals BSDF + NEE with budgets 1
    within 3.5 sigma (App. A.1's unbiasedness, now over whole-path weights),
    and the light connections carry a share of it."""
    sc = W.heightfield_scene(3, n=6, width=32, height=24, n_spheres=6)
    cells = 4 ** 3
    q_rr, q_s, valid = W.random_count_fields(cells, seed=121, lo=0.1, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=122, lo=0.05, hi=2.0)
    a, b, lc = [], [], []
    for it in range(100):
        kw = dict(grid_n=4, max_depth=5, iteration=it)
        a.append(orc.render(sc, techniques=3, **kw).image.mean())
        r = orc.render(sc, techniques=TECH_BDPT, mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est,
                       seed=9, **kw)
        b.append(r.image.mean())
        lc.append(r.stats[:, 2, 1:4].sum())
    ma, sa = _mean_and_sem(a)
    mb, sb = _mean_and_sem(b)
    assert abs(ma - mb) < 3.5 * math.hypot(sa, sb)
    assert np.mean(lc) > 0


def test_light_connection_cost_and_roulette(orc):
    """A light connection sample costs the rays its light subpath traced plus
    one per connection.  In the closed furnace every light ray finds a wall, so
    each light vertex costs one ray and one connection (cost = 2 x light rays);
    with D = 3 only first vertices draw the technique (a connection from x_2
    would exceed D segments) and each subpath holds one vertex (cost 2 per
    sample); with D = 4 the subpath of a first-vertex sample continues past
    y_1 with the throughput-based survival probability, which for a grey
    Lambertian surface is its albedo a."""
    a = 0.625
    sc = W.furnace_scene(albedo=a, radiance=1.0, width=12, height=12)
    P = sc.n_pixels
    r = orc.render(sc, grid_n=2, techniques=TECH_BDPT, max_depth=3)
    s = r.stats[:, 2, :].sum(0)
    assert s[0] == P and s[7] == 2 * P and r.counters[6] == P
    n_light, rays = 0.0, []
    for it in range(40):
        r = orc.render(sc, grid_n=2, techniques=TECH_BDPT, max_depth=4, iteration=it)
        s = r.stats[:, 2, :].sum(0)
        assert s[0] == 2 * P and s[7] == 2 * r.counters[6]
        rays.append(r.counters[6] / P)
    # per pixel: the depth-1 sample traces 1 + Bernoulli(a) rays, the depth-2 one 1
    m, se = _mean_and_sem(rays)
    assert abs(m - (2 + a)) < 4 * se + 1e-9


def test_whole_path_weights_reduce_to_the_vertex_weights_without_light_connections(orc):
    """With the light connection's budget 0 everywhere (clamp_lo = 0 and q = 0:
    no sample is drawn and, budget-aware, the strategy's count is 0), the
    whole-path balance weights of the bidirectional renderer reduce to the
    per-vertex balance heuristic of BSDF sampling and NEE (App. A.1): camera
    path and NEE are the only strategies, and the whole-path density ratio of
    the two is the ratio of their solid-angle densities at the last vertex.
    The images agree to rounding at every depth.  (Budget-unaware weights
    count every technique once whatever its budget, so they need budgets
    above 0 -- the paper's clamp [0.05, 20] -- to stay unbiased.)"""
    weights = 0
    cfg = W.config_box(20, 16)
    cells = cfg.n_cells
    q_rr, q_s, valid = W.random_count_fields(cells, seed=131, lo=0.1, hi=3.0, p_valid=1.0)
    q_rr[:, 2] = 0.0
    q_s[:, 2] = 0.0
    est = W.random_pixel_estimate(cfg.scene.n_pixels, seed=132, lo=0.05, hi=1.0)
    kw = dict(grid_n=cfg.grid_n, max_depth=cfg.max_depth, iteration=4, seed=3, mode=orc.MODE_MARS, q_rr=q_rr,
              q_s=q_s, valid=valid, est=est, clamp_lo=0.0, weights=weights, outlier=1e30)
    a = orc.render(cfg.scene, techniques=3, **kw)
    b = orc.render(cfg.scene, techniques=TECH_BDPT, **kw)
    assert b.stats[:, 2, 0].sum() == 0 and a.rays == b.rays
    np.testing.assert_allclose(b.image, a.image, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b.stats[:, :2], a.stats[:, :2], rtol=1e-12, atol=1e-15)


def _patch_counts_and_expectation(hits, prims, prim, axes, lo, hi, density, n, grid=8):
    """Landings of n drawn steps on primitive `prim` inside the rectangle
    [lo, hi] of the coordinates `axes`, and their expected number: n times the
    integral of `density` (a function of a point) over the rectangle, by the
    midpoint rule on a grid x grid lattice."""
    sel = prims == prim
    for a, l0, h0 in zip(axes, lo, hi):
        sel &= (hits[:, a] >= l0) & (hits[:, a] < h0)
    count = int(sel.sum())
    plane = hits[prims == prim][0].copy()
    total = 0.0
    for i in range(grid):
        for j in range(grid):
            x = plane.copy()
            x[axes[0]] = lo[0] + (i + 0.5) * (hi[0] - lo[0]) / grid
            x[axes[1]] = lo[1] + (j + 0.5) * (hi[1] - lo[1]) / grid
            total += density(x)
    area = (hi[0] - lo[0]) * (hi[1] - lo[1])
    return count, n * total / grid ** 2 * area


def _assert_frequency_matches(count, expected):
    # Poisson scatter of the count, plus 2 % for the midpoint rule
    assert expected > 400
    assert abs(count - expected) < 5.0 * math.sqrt(expected) + 0.02 * expected, (count, expected)


def test_light_side_densities_match_the_drawn_light_steps(orc):
    """Brute force on the light-side densities P<- of the whole-path weights:
    light subpath steps drawn by the renderer's own routines land on a patch as
    often as the density the weights give those steps says.  Emission: cosine
    directions from a point of the light, landings on a floor patch and on a
    wall patch (the cosines at the light and at the landing point differ, and
    no 1/pi or 1/d^2 may be missing).  Bounce: BSDF sampling with the light
    arriving from the light point, then the roulette, at a floor vertex, landings
    on two wall patches: the density is that of the sampled direction towards
    the landing point given the direction the light came from, times the
    survival probability, converted by the cosine at the landing point --
    Lambertian floor (survival 0.5) and a GGX floor whose lobe the landings
    follow."""
    n = 400_000
    rng = np.random.default_rng(2024)
    scene = W.light_step_scene()
    y0 = np.array([0.0, 1.0, 0.0])
    org = y0 + np.array([0.0, -1.0, 0.0]) * 1e-4   # the emission origin is offset along the light normal
    hits, prims = orc.light_emit(scene, 0, y0, rng.uniform(size=(n, 2)))

    def emit_density(x):
        return orc.light_density(scene, 0, y0, x - org, x)[0]

    for prim, axes, lo, hi in ((0, (0, 2), (0.3, -0.5), (0.5, -0.3)), (1, (1, 2), (0.3, 0.0), (0.5, 0.2))):
        _assert_frequency_matches(*_patch_counts_and_expectation(hits, prims, prim, axes, lo, hi, emit_density, n))

    for alpha, y0, y1, patches in (
            (0.0, np.array([0.0, 1.0, 0.0]), np.array([-0.3, 0.0, 0.2]),
             (((1, 2), (0.2, -0.2), (0.5, 0.1)), ((1, 2), (0.6, 0.3), (0.9, 0.6)))),
            (0.3, np.array([-0.2, 1.0, 0.0]), np.array([0.5, 0.0, 0.0]),
             (((1, 2), (0.66, -0.05), (0.76, 0.05)), ((1, 2), (0.4, 0.1), (0.5, 0.2))))):
        scene = W.light_step_scene(alpha)
        d1 = y1 - (y0 + np.array([0.0, -1.0, 0.0]) * 1e-4)
        hits, prims = orc.light_bounce(scene, 0, y0, d1, rng.uniform(size=(n, 3)))

        def bounce_density(x, scene=scene, y0=y0, d1=d1):
            return orc.light_density(scene, 0, y0, d1, x)[1]

        for axes, lo, hi in patches:
            _assert_frequency_matches(*_patch_counts_and_expectation(hits, prims, 1, axes, lo, hi, bounce_density,
                                                                     n))


@pytest.mark.parametrize("D,counts", [(2, "beta1"), (2, "random"), (3, "beta1")])
def test_guide_deposits_closed_form_in_the_furnace(orc, D, counts):
    """Guide learning records, per continuation sample, the incident radiance
    over the multi-sample density of the indirect techniques (real budgets):
    sum_t beta_t E_t[L_i / (beta_B p_B + beta_G p_G)] = the integral of L_i over
    the hemisphere, whatever the budgets.  In the closed furnace (radiance Le,
    albedo a, uniform guide, no NEE) every camera vertex therefore deposits
    2 pi Le in expectation when D = 2; when D = 3 it deposits 2 pi (1 + a) Le (the
    incident radiance includes the next vertex's reflected estimate) and each
    of its 0.75 children on average (the BSDF child, and the guided child when it
    lands above the surface: half of the uniform guide) deposits 2 pi Le."""
    a, le = 0.5, 1.5
    sc = W.furnace_scene(albedo=a, radiance=le, width=16, height=16)
    cells = 2 ** 3
    cdf = np.tile((np.arange(1, orc.GUIDE_BINS + 1) / orc.GUIDE_BINS).astype(np.float32), (cells, 1))
    q_rr, q_s, valid = W.random_count_fields(cells, seed=21, lo=0.2, hi=3.0)
    est = W.random_pixel_estimate(sc.n_pixels, seed=22, lo=0.5, hi=4.0)
    tot = []
    for it in range(30):
        kw = dict(grid_n=2, techniques=W.TECH_BSDF | W.TECH_GUIDED, max_depth=D, iteration=it, guide_cdf=cdf)
        if counts == "random":
            kw.update(mode=orc.MODE_MARS, q_rr=q_rr, q_s=q_s, valid=valid, est=est)
        tot.append(orc.render(sc, **kw).hist.sum() / sc.n_pixels)
    m, se = _mean_and_sem(tot)
    expected = 2 * math.pi * le * (1.0 if D == 2 else (1 + a) + 0.75)
    assert abs(m - expected) < 3.5 * se, (m, se, expected)
