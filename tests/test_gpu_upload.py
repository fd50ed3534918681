"""Uploads: the caller's FP64 floes are checked and converted into the cell
layout on the device (ms_init and ms_set_floes).  The stored state must be
what the plain IEEE arithmetic of the assignment gives: cell = floor of the
wrapped position over the cell side, FP32 positions the offset in the cell
as 32-bit fixed point rounded to nearest even, the other FP32 fields the
FP64 values rounded once; FP64 positions the offset itself.  numpy computes
the same operations here, so the comparison is bit for bit."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def expected(p, f, precision):
    """floes() of a model holding f, from the assignment's arithmetic"""
    nens = int(p.get("nens", 1))
    nx, ny = int(p["nx"]), int(p["ny"]) * nens
    Lx, Ly = float(p["Lx"]), float(p["Ly"]) * nens
    Lcx, Lcy = float(p["Lx"]) / p["nx"], float(p["Ly"]) / p["ny"]
    Xw = f["x"] - Lx * np.floor(f["x"] / Lx)
    Yw = f["y"] - Ly * np.floor(f["y"] / Ly)
    ix = np.clip(np.floor(Xw / Lcx), 0, nx - 1)
    iy = np.clip(np.floor(Yw / Lcy), 0, ny - 1)
    out = {}
    if precision == 0:
        fix = lambda fr: (np.rint(fr * 4294967296.0).astype(np.int64) & 0xFFFFFFFF).astype(np.float64)
        out["x"] = (ix + fix((Xw - ix * Lcx) / Lcx) / 4294967296.0) * Lcx
        out["y"] = (iy + fix((Yw - iy * Lcy) / Lcy) / 4294967296.0) * Lcy
        for k in ("theta", "u", "v", "omega", "r", "h"):
            out[k] = f[k].astype(np.float32).astype(np.float64)
    else:
        out["x"] = ix * Lcx + (Xw - ix * Lcx)
        out["y"] = iy * Lcy + (Yw - iy * Lcy)
        for k in ("theta", "u", "v", "omega", "r", "h"):
            out[k] = f[k].copy()
    return out


def scenarios():
    ens = I.stack_ensemble([I.powerlaw_32x32(seed=200 + e, nx=4) for e in range(3)])
    # non-dimensional domain, cell sides 4/48 and 2/24 not representable
    return [I.batched_128x128(seed=5, nx=16), I.scenario41(96, 48, 48, 24), ens]


@pytest.mark.parametrize("precision", [0, 1])
def test_init_and_set_floes_round_as_the_host(ms, precision):
    for s in scenarios():
        p, f = s["params"], s["floes"]
        g = ms.Model(p, f, precision)
        got, want = g.floes(), expected(p, f, precision)
        for k in want:
            assert np.array_equal(got[k], want[k]), k
        # moved within their cells (and a wrapped copy of the x positions:
        # one period further, the same floe) through ms_set_floes
        rng = np.random.default_rng(7)
        m = {k: v.copy() for k, v in got.items()}
        Lcx = float(p["Lx"]) / p["nx"]
        cx = (np.floor(m["x"] / Lcx) + 0.5) * Lcx
        m["x"] = m["x"] + rng.uniform(0.1, 0.5, m["x"].shape) * (cx - m["x"]) + float(p["Lx"])
        m["u"] = m["u"] + rng.normal(0.0, 0.01, m["u"].shape)
        m["r"] = m["r"] * 0.99
        g.set_floes(m)
        got, want = g.floes(), expected(p, m, precision)
        for k in want:
            assert np.array_equal(got[k], want[k]), k
        g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_set_floes_rejects_and_keeps_state(ms, precision):
    """A non-finite value, r <= 0, h <= 0 or a floe outside its cell is
    reported with the smallest offending index, and the model keeps its
    floes and moments."""
    s = I.powerlaw_32x32(nx=4)
    g = ms.Model(s["params"], s["floes"], precision)
    g.step(s["dt"], 3)
    f0, m0 = g.floes(), g.moments()
    n = f0["x"].shape[0]
    cases = [("omega", n - 1, np.inf, "non-finite"), ("y", 5, np.nan, "non-finite"), ("r", 17, 0.0, "r <= 0"),
             ("h", 3, -1.0, "r <= 0"), ("x", 9, None, "left its cell")]
    for key, idx, val, msg in cases:
        bad = {k: v.copy() for k, v in f0.items()}
        if val is None:
            bad["x"][idx] += float(s["params"]["Lx"]) / s["params"]["nx"]
            bad["x"][idx + 40] += float(s["params"]["Lx"]) / s["params"]["nx"]
        else:
            bad[key][idx] = val
            if idx + 50 < n:
                bad["r"][idx + 50] = -1.0      # a later index: the smaller one is reported
        with pytest.raises(ms.MsError) as e:
            g.set_floes(bad)
        assert e.value.code == -1 and msg in str(e.value) and f"floe {idx} " in str(e.value), str(e.value)
        f1 = g.floes()
        for k in f0:
            assert np.array_equal(f0[k], f1[k]), (key, k)
        assert np.array_equal(m0, g.moments())
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_uploading_the_held_state_continues_the_run(ms, precision):
    """Uploading, at an interval boundary, the floes the model holds (what the
    bench's end-to-end loop does every step) changes nothing in FP32: the
    fixed-point round trip is exact, the moments pass of ms_set_floes leaves
    the coupling window alone, and an interval's first step searches again
    either way, so the run goes on bit for bit as the uninterrupted one,
    coupling included.  FP64 keeps positions as offsets from the cell origin
    while the API speaks global coordinates, so there the round trip can move
    a floe by an ulp of its global coordinate (get, set, get is still exact)
    and the run goes on within 1e-10."""
    from tests.parity import rel_errors, report
    s = I.batched_128x128(seed=12, nx=8)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    a = ms.Model(p, s["floes"], precision)
    b = ms.Model(p, s["floes"], precision)
    a.step(dt, 3 * N0)
    b.step(dt, N0)
    for _ in range(2):
        b.set_floes(b.floes())
        b.step(dt, N0)
    fa, fb = a.floes(), b.floes()
    qa, qb = a.coupling()["q"], b.coupling()["q"]
    if precision == 0:
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        assert np.array_equal(a.moments(), b.moments())
        assert np.array_equal(qa, qb)
    else:
        for k in fa:
            assert np.allclose(fa[k], fb[k], rtol=1e-10, atol=1e-6 if k in "xy" else 1e-12), k
        err = rel_errors(b.moments(), a.moments(), p, 1e-12)
        assert err.max() <= 1e-10, report(err)
        assert np.linalg.norm(qa - qb) <= 1e-10 * np.linalg.norm(qa)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_half_open_cells_match_the_oracle(ms, orc, precision):
    """Floes on a cell's left edge, at X = Lx and at negative coordinates
    are assigned as the oracle assigns them (half-open cells, floor wrap):
    by ms_init's counting sort on the device, by ms_floe_cells, and by the
    device-side check of ms_set_floes, which accepts the same floes again."""
    L = 4.0e4
    dX = L / 4
    xs = [dX, 2 * dX, L, -dX, 0.5 * dX]
    ys = [0.5 * dX, dX, 3 * dX, 0.5 * dX, -0.5 * dX]
    n = len(xs)
    fl = {"x": np.array(xs), "y": np.array(ys), "theta": np.zeros(n), "u": np.zeros(n), "v": np.zeros(n),
          "omega": np.zeros(n), "r": np.full(n, 100.0), "h": np.ones(n)}
    p = I._phys(dt=5.0)
    p.update({"nx": 4, "ny": 4, "Lx": L, "Ly": L, "modes": np.zeros((0, 4))})
    g = ms.Model(p, fl, precision)
    o = orc.Model(p, fl)
    assert np.array_equal(g.moments()[:, 0], o.moments()[:, 0])
    assert g.moments()[:, 0].tolist() == [0, 1, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 2, 0, 0, 0]
    assert ms.floe_cells(p, fl).tolist() == [1, 6, 12, 3, 12]
    for a, b in zip(g.layout(), o.layout()):
        assert np.array_equal(a, b)
    g.set_floes(fl)
    assert np.array_equal(g.moments()[:, 0], o.moments()[:, 0])
    g.close()


def _oracle_layout(orc, p, fl):
    o = orc.Model(p, fl)
    off, orig = o.layout()
    o.close()
    return off, orig


@pytest.mark.parametrize("name", ["powerlaw_32x32", "batched_128x128"])
def test_layout_is_the_oracles(ms, orc, name):
    """The cell layout ms_init builds on the device (cell of each floe,
    offsets, the floes of each cell in the caller's order) equals the
    oracle's, index for index, on the full-size workloads (65k and 2M
    floes), and ms_floe_cells gives the cells it used."""
    s = I.WORKLOADS[name]()
    p, fl = s["params"], s["floes"]
    g = ms.Model(p, fl, 0)
    off, orig = g.layout()
    o_off, o_orig = _oracle_layout(orc, p, fl)
    assert np.array_equal(off, o_off)
    assert np.array_equal(orig, o_orig)
    cell = np.repeat(np.arange(off.size - 1), np.diff(off))
    cells_of = ms.floe_cells(p, fl)
    assert np.array_equal(cells_of[orig], cell)
    g.close()


def test_layout_of_a_full_cell_in_shuffled_order(ms, orc):
    """4096 floes in one cell (the FP32 limit) and a few in others, given in
    a random order: each cell's floes come out in ascending caller order,
    as the oracle stores them; an empty model has an all-zero layout."""
    rng = np.random.default_rng(7)
    L = 8.0e5
    n0 = 4096
    x = np.concatenate([rng.uniform(0.0, L / 2, n0), rng.uniform(L / 2, L, 37)])
    y = np.concatenate([rng.uniform(0.0, L / 2, n0), rng.uniform(0.0, L, 37)])
    perm = rng.permutation(x.size)
    n = x.size
    fl = {"x": x[perm], "y": y[perm], "theta": np.zeros(n), "u": np.zeros(n), "v": np.zeros(n),
          "omega": np.zeros(n), "r": np.full(n, 10.0), "h": np.ones(n)}
    p = I._phys(dt=5.0)
    p.update({"nx": 2, "ny": 2, "Lx": L, "Ly": L, "modes": np.zeros((0, 4)), "couple": 0})
    g = ms.Model(p, fl, 0)
    off, orig = g.layout()
    o_off, o_orig = _oracle_layout(orc, p, fl)
    assert np.array_equal(off, o_off) and np.array_equal(orig, o_orig)
    assert off[1] - off[0] == n0
    for c in range(4):
        assert (np.diff(orig[off[c]:off[c + 1]]) > 0).all()
    g.close()
    empty = {k: np.zeros(0) for k in fl}
    g = ms.Model(p, empty, 0)
    off, orig = g.layout()
    assert not off.any() and orig.size == 0
    g.close()
