"""CPU checks of the benchmark's measurement helpers: the clock-sample summary
(window filtering, throttle reasons), relMSE and the single-rank aggregation."""
import datetime
import time

import numpy as np
import pytest

import bench


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, rows, t0):
    path = tmp_path / "clocks.csv"
    path.write_text("".join(rows))
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc, s.path, s.t0 = _DoneProc(), str(path), t0
    s.f = open(tmp_path / "sink", "w")
    return s


def _row(ts, clk, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return f"{stamp}, 0, {clk}, 2070, 500.0, 0x0, " + ", ".join(reasons) + "\n"


def test_clock_summary_keeps_only_samples_under_load(tmp_path):
    now = time.time()
    rows = [_row(now - 5.0, 1000),                      # before begin(): idle, dropped
            _row(now - 0.50, 2070), _row(now - 0.48, 2060), _row(now - 0.46, 2070),
            _row(now + 30.0, 900)]                      # after stop(): dropped
    st = _sampler(tmp_path, rows, t0=now - 0.6).stop("test window")
    assert st["samples"] == 3 and st["sm_mhz"] == 2070.0 and st["sm_min_mhz"] == 2060.0
    assert st["sm_max_mhz"] == 2070.0 and st["reasons"] == [] and st["window"] == "test window"


def test_clock_summary_reports_throttle_reasons(tmp_path):
    now = time.time()
    rows = [_row(now - 0.3, 1800, ("Not Active", "Not Active", "Not Active", "Active")),
            _row(now - 0.2, 1500, ("Active", "Not Active", "Not Active", "Not Active")),
            "garbage line\n"]
    st = _sampler(tmp_path, rows, t0=now - 0.4).stop()
    assert st["samples"] == 2 and st["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples(tmp_path):
    st = _sampler(tmp_path, [], t0=time.time()).stop()
    assert st["sm_mhz"] is None and st["reasons"] == ["no samples under load"]


def test_rel_mse_basics():
    rng = np.random.default_rng(0)
    ref = rng.uniform(0.1, 2.0, size=(64, 64, 3))
    assert bench.rel_mse(ref, ref) == 0.0
    # a uniform 10 % error on every pixel: (0.1 R)^2 / (R^2 + 0.01), no outliers to drop
    v = bench.rel_mse(1.1 * ref, ref)
    expect = ((0.1 * ref) ** 2 / (ref ** 2 + 1e-2)).reshape(-1, 3).mean(axis=1)
    k = int(np.ceil(1e-4 * expect.size))
    assert v == pytest.approx(np.sort(expect)[:-k].mean(), rel=1e-12)
    # one wild pixel is dropped with the 0.01 % largest terms
    bad = ref.copy()
    bad[3, 5] = 1e6
    assert bench.rel_mse(bad, ref) < 1e-12


def test_single_rank_aggregation_is_identity():
    assert bench.reduce_over_ranks(12.5, 3e6, 1, "cpu") == (12.5, 3e6)


def test_rel_mse_subtracts_the_reference_variance():
    """A noise-free image against a noisy reference of known variance: the raw
    relMSE charges the reference's noise to the image, the corrected one does
    not (E[(I - R)^2] = Var(I) + bias^2 + Var(R))."""
    rng = np.random.default_rng(1)
    truth = rng.uniform(0.2, 2.0, size=(256 * 256, 3))
    var = (0.05 * truth) ** 2
    ref = truth + rng.normal(size=truth.shape) * np.sqrt(var)
    raw = bench.rel_mse(truth, ref)
    fixed = bench.rel_mse(truth, ref, var)
    assert raw > 1e-3
    assert abs(fixed) < 0.05 * raw
    # an image with its own error keeps it: Var(I) survives the correction
    img = truth + rng.normal(size=truth.shape) * 0.1 * truth
    own = ((0.1 * truth) ** 2 / (truth ** 2 + 1e-2)).mean()
    assert bench.rel_mse(img, ref, var) == pytest.approx(own, rel=0.05)


def test_every_called_name_is_defined():
    """Every plain function name bench.py calls is defined in it, imported or a
    builtin (the GPU-only code paths cannot run here)."""
    import ast
    import builtins
    import os
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")).read()
    tree = ast.parse(src)
    defined = set(dir(builtins))
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            defined.add(node.name)
            defined.update(a.arg for a in node.args.args + node.args.kwonlyargs) if isinstance(node, ast.FunctionDef) \
                else None
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            defined.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, ast.Store):
            defined.add(node.id)
        elif isinstance(node, ast.arg):
            defined.add(node.arg)
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    assert not called - defined, sorted(called - defined)


def test_rel_mse_at_the_images_scale_is_scale_free():
    """relMSE with eps = 1e-2 x the reference's squared mean does not change
    when the image and the reference are scaled together (what the bench's
    `ratio_scaled` relies on), while the fixed eps = 1e-2 does."""
    rng = np.random.default_rng(2)
    ref = rng.uniform(0.0, 0.05, size=(128 * 128, 3))
    img = ref * (1.0 + 0.2 * rng.normal(size=ref.shape))
    for k in (1.0, 37.0):
        eps = 1e-2 * float((k * ref).mean()) ** 2
        r = bench.rel_mse(k * img, k * ref, eps=eps)
        if k == 1.0:
            r1 = r
    assert r == pytest.approx(r1, rel=1e-9)
    assert bench.rel_mse(37.0 * img, 37.0 * ref) > 5 * bench.rel_mse(img, ref)


def test_measured_traffic_is_per_unit_and_keyed_by_the_sources(tmp_path, monkeypatch):
    """The committed traffic summary gives bytes per unit for every wave kernel,
    and is ignored once the kernel sources or build flags hash differently."""
    import os
    sha = next(line.split()[1] for line in open(os.path.join(os.path.dirname(bench.__file__), bench.TRAFFIC_FILE))
               if line.startswith("sources_sha256"))
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)
    vals = bench.measured_traffic()
    assert set(vals) == {"k_trace", "k_shade", "k_shadow", "k_reverse"}
    assert all(10.0 < v < 1000.0 for v in vals.values())
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: "0" * 64)
    assert bench.measured_traffic() == {}
