"""The seeded input generators against the recipes they state: grid sizes,
floes per cell, radius and thickness laws, cover, placement without overlap
under the cell's periodic metric (and the domain's where stated), floes at
rest, the ensemble stacking, and determinism.  CPU only; the full-size
power-law and batched workloads are checked on smaller grids with the same
laws (their generators take nx)."""
import math

import numpy as np

from paper_2303_07819_gb300 import inputs as I


def cells(f, p):
    Lcx, Lcy = p["Lx"] / p["nx"], p["Ly"] / p["ny"]
    return np.floor(f["y"] / Lcy).astype(int) * p["nx"] + np.floor(f["x"] / Lcx).astype(int)


def min_gap(x, y, r, Lx, Ly):
    """smallest d - (r_l + r_j) over distinct pairs, periodic minimum image"""
    dx = np.subtract.outer(x, x)
    dy = np.subtract.outer(y, y)
    dx -= Lx * np.round(dx / Lx)
    dy -= Ly * np.round(dy / Ly)
    g = np.hypot(dx, dy) - np.add.outer(r, r)
    np.fill_diagonal(g, np.inf)
    return g.min() if len(x) > 1 else np.inf


def cell_gaps(f, p):
    Lcx, Lcy = p["Lx"] / p["nx"], p["Ly"] / p["ny"]
    c = cells(f, p)
    return min(min_gap(f["x"][c == k], f["y"][c == k], f["r"][c == k], Lcx, Lcy) for k in np.unique(c))


def test_square_4x4():
    s = I.square_4x4()
    p, f = s["params"], s["floes"]
    assert (p["nx"], p["ny"], p["Lx"], p["Ly"], s["dt"]) == (4, 4, 100e3, 100e3, 10.0)
    assert np.array_equal(np.bincount(cells(f, p), minlength=16), np.full(16, 16))
    assert np.array_equal(cells(f, p), s["meta"]["cell"])
    assert f["r"].max() <= 2500.0 and f["r"].min() > 0.0 and np.all(f["h"] == 1.0)
    # overlap-free under the cell metric and under the domain metric
    assert cell_gaps(f, p) > 0.0
    assert min_gap(f["x"], f["y"], f["r"], p["Lx"], p["Ly"]) > 0.0
    for k in ("u", "v", "omega", "theta"):
        assert np.all(f[k] == 0.0)
    assert p["wind_x"] == 0.0 and p["wind_y"] == 0.0 and p["Ca"] == 0.0


def test_powerlaw_laws_on_8x8():
    s = I.powerlaw_32x32(nx=8)
    p, f = s["params"], s["floes"]
    assert p["Lx"] == 8 * 12.5e3 and s["dt"] == 5.0
    counts = np.bincount(cells(f, p), minlength=64)
    assert counts.min() >= 1 and abs(counts.mean() - 64.0) < 4.0   # Poisson(64) over 64 cells: sd of the mean 1
    # radii: p(r) ~ r^-2 on [0.2, 3] km, then a per-cell scale <= 1 (cover at most 55 %)
    sc = s["meta"]["radius_scale"]
    assert np.all(sc <= 1.0) and np.all(sc > 0.0)
    c = cells(f, p)
    assert np.all(f["r"] <= 3000.0 * sc[c] * (1 + 1e-12))
    Ac = (p["Lx"] / p["nx"]) ** 2
    cover = np.bincount(c, weights=np.pi * f["r"] ** 2, minlength=64) / Ac
    assert cover.max() <= 0.55 + 1e-9
    assert cell_gaps(f, p) > 0.0
    assert min_gap(f["x"], f["y"], f["r"], p["Lx"], p["Ly"]) > 0.0
    # thickness lognormal with mean 1.5 m and sd 0.5 m
    assert abs(f["h"].mean() - 1.5) < 0.05 and abs(f["h"].std() - 0.5) < 0.05
    assert p["modes"].shape == (8, 4) and p["wind_x"] == 10.0 and p["Ca"] == 1.2e-3


def test_power_law_radii_distribution():
    """Inverse-CDF sampling of p(r) ~ r^-2 on [a, b]: the sample CDF matches
    F(r) = (1/a - 1/r) / (1/a - 1/b) (Kolmogorov-Smirnov distance)."""
    rng = np.random.default_rng(3)
    a, b = 200.0, 3000.0
    r = np.sort(I.power_law_radii(rng, 20000, a, b))
    F = (1 / a - 1 / r) / (1 / a - 1 / b)
    emp = np.arange(1, r.size + 1) / r.size
    assert r.min() >= a and r.max() <= b
    assert np.abs(F - emp).max() < 1.63 / math.sqrt(r.size)      # KS at the 1 % level


def test_batched_laws_on_32x32():
    s = I.batched_128x128(nx=32)
    p, f = s["params"], s["floes"]
    assert p["Lx"] == 32 * 25e3 and s["dt"] == 5.0 and p["wind_period"] == 6 * 3600.0
    counts = np.bincount(cells(f, p), minlength=32 * 32)
    assert counts.min() >= 8 and counts.max() <= 1024
    # lognormal(median 96, sigma 0.69) before clipping: median and log-spread
    assert abs(np.median(counts) - 96) <= 6
    assert abs(np.log(counts).std() - 0.69) < 0.05
    assert np.array_equal(cells(f, p), s["meta"]["cell"])
    assert cell_gaps(f, p) > 0.0
    for k in ("u", "v", "omega"):
        assert np.all(f[k] == 0.0)


def test_full_batched_floe_count():
    """The timed workload's size is fixed by its seed: 128 x 128 cells,
    1,982,044 floes, a mean of 121 per cell and E[n^2]/E[n] = 192 (the pair
    work's weighting); the lognormal counts alone, without placing the floes."""
    rng = np.random.default_rng(I.BASE_SEED + 2)
    counts = I.lognormal_counts(rng, 128 * 128, 96.0, 0.69, 8, 1024).astype(np.float64)
    assert counts.sum() == 1_982_044
    assert round(counts.mean()) == 121 and round((counts ** 2).sum() / counts.sum()) == 192


def test_ensemble_stacking():
    e = I.ensemble_16x256x256(nreal=3, nx=8)
    p, f = e["params"], e["floes"]
    assert p["nens"] == 3
    Ly = p["Ly"]
    real = np.floor(f["y"] / Ly).astype(int)
    assert set(np.unique(real)) <= {0, 1, 2}
    # one ocean for all realizations, their own floes
    one = I.ensemble_16x256x256(nreal=1, nx=8)
    assert np.array_equal(p["modes"], one["params"]["modes"])
    k0 = real == 0
    for k in f:
        assert np.array_equal(f[k][k0], one["floes"][k]), k
    counts = np.bincount(np.floor(f["y"] / (Ly / p["ny"])).astype(int) * p["nx"]
                         + np.floor(f["x"] / (p["Lx"] / p["nx"])).astype(int), minlength=3 * 64)
    assert counts.min() >= 1 and counts.max() <= 64


def test_generators_are_deterministic():
    for make in (I.square_4x4, lambda: I.powerlaw_32x32(nx=4), lambda: I.batched_128x128(nx=8)):
        a, b = make(), make()
        for k in a["floes"]:
            assert np.array_equal(a["floes"][k], b["floes"][k]), k
        assert np.array_equal(a["params"]["modes"], b["params"]["modes"])
    assert not np.array_equal(I.square_4x4(seed=1)["floes"]["x"], I.square_4x4()["floes"]["x"])
