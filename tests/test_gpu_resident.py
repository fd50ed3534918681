"""Launch variant 5: every cell of up to 1024 floes resident for a whole run
of fine steps, a floe per thread (2 or 4 for cells above 256 floes),
contacts from candidate lists summed in ascending partner order.

Parity with the FP64 oracle within the FP32 tolerance on cells of every size
class (including a cell above 1024 floes, which runs the per-step block
kernel), contacts dense enough to overflow a list, and bitwise equality of a
run however it is split into launches (graph intervals, single steps, odd
runs), through coarse steps and gradual updates."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from tests.parity import rel_errors, report
from tests.test_gpu_parity import TOL32, ragged_scenario

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def _same(a, b):
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.moments(), b.moments())
    ca, cb = a.coupling(), b.coupling()
    for k in ("q", "targets", "window"):
        assert np.array_equal(ca[k], cb[k]), k


def test_every_class_matches_oracle(orc, ms):
    """Cells of 0 to 1100 floes (empty cells, packed groups of small cells,
    2 and 4 floes per thread, and a cell above 1024 floes on the per-step
    block kernel), 250 steps: two coarse steps with their gradual updates;
    moments and the coarse solution within the FP32 tolerance."""
    s = ragged_scenario([0, 1, 3, 9, 17, 31, 33, 64, 100, 129, 200, 256, 257, 300, 511, 513, 700, 1024, 1100],
                        L_c=25e3, seed=41)
    p = s["params"]
    o = orc.Model(p, s["floes"])
    g = ms.Model(p, s["floes"], ms.MS_FP32)
    g.set_launch(5, 128, 0, 1.3)
    o.step(s["dt"], 250)
    g.step(s["dt"], 250)
    mo, mg = o.moments(), g.moments()
    assert np.array_equal(mo[:, 0], mg[:, 0])
    e = rel_errors(mg, mo, p, 1e-6)
    assert e.max() <= TOL32, report(e)
    qo, qg = o.coupling()["q"], g.coupling()["q"]
    for f in range(4):
        assert np.linalg.norm(qg[f] - qo[f]) <= TOL32 * np.linalg.norm(qo[f]), f
    assert g.info()["variant"] == 5


def test_runs_split_anywhere_are_bitwise_equal(ms):
    """An interval from the graph (one launch per class), the same steps one
    launch each, and runs of odd lengths that end inside gradual-update
    periods (the floes' running window sums carried between launches): the
    same floes, moments, window and coarse solution bit for bit, across two
    coarse steps."""
    s = I.batched_128x128(seed=7, nx=16)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    models = [ms.Model(p, s["floes"], ms.MS_FP32) for _ in range(3)]
    for m in models:
        m.set_launch(5, 128, 0, 1.3)
    a, b, c = models
    total = 2 * N0 + 17
    a.step(dt, total)
    for _ in range(total):
        b.step(dt, 1)
    done = 0
    for k in (37, 1, 62, 9, 3, 88, 17):
        c.step(dt, k)
        done += k
    assert done == total
    assert a.info()["graph_replays"] == 2 and b.info()["graph_replays"] == 0
    _same(a, b)
    _same(a, c)


def test_repeat_runs_are_bitwise_equal(ms):
    """Builds happen at times that depend on a floating-point speed sum (a
    shared-memory atomic, whose order varies), and floes switch between their
    candidate list and the all-cell walk when a list overflows; neither may
    change a result.  Two models of a crowded workload, three coarse
    intervals from the graph, and the same steps in runs of 7: the same floes
    and coarse solution bit for bit."""
    s = I.batched_128x128(seed=23, nx=8)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    f = {k: v.copy() for k, v in s["floes"].items()}
    f["x"] = f["x"] + 0.15 * (np.floor(f["x"] / 25e3) * 25e3 + 12.5e3 - f["x"])
    ms_ = [ms.Model(p, f, ms.MS_FP32) for _ in range(3)]
    for m in ms_:
        m.set_launch(5, 128, 0, 1.3)
    ms_[0].step(dt, 3 * N0)
    ms_[1].step(dt, 3 * N0)
    for _ in range(3 * N0 // 7):
        ms_[2].step(dt, 7)
    ms_[2].step(dt, 3 * N0 - 7 * (3 * N0 // 7))
    _same(ms_[0], ms_[1])
    _same(ms_[0], ms_[2])


def test_packing_does_not_change_results(ms):
    """Which cells share a block (block_floes), the skin horizon, and a
    cell's place among the other cells of its block do not change a result:
    its floes run the code of its own size class and its per-cell sums are
    exact integer sums.  Three coarse intervals of the batched workload's
    laws on 24 x 24 cells (cells of 8 to 1024 floes) under four launch
    choices: the same floes, moments and coarse solution bit for bit."""
    s = I.batched_128x128(seed=29, nx=24)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    runs = []
    for skin, cap in ((32.0, 256), (32.0, 96), (16.0, 160), (48.0, 208)):
        m = ms.Model(p, s["floes"], ms.MS_FP32)
        m.set_resident(skin, cap)
        m.step(dt, 3 * N0 + 17)
        runs.append(m)
    for m in runs[1:]:
        _same(runs[0], m)
    for m in runs:
        m.close()


def test_contacts_and_list_overflow(orc, ms):
    """A 3 km floe ringed by 60 floes of 150 m that touch it (its list of at
    most 16 candidates overflows and it tests every floe of its cell), plus
    loose floes: within the FP32 tolerance of the oracle over 60 steps, and
    the same result as the neighbour-list kernel of variant 4."""
    rng = np.random.default_rng(31)
    L_c, nx = 25e3, 2
    ang = 2 * np.pi * (np.arange(60) + 0.5) / 60
    x = np.concatenate([[12.5e3], 12.5e3 + 3140.0 * np.cos(ang)])
    y = np.concatenate([[12.5e3], 12.5e3 + 3140.0 * np.sin(ang)])
    r = np.concatenate([[3000.0], np.full(60, 150.0)])
    for cx, cy in ((1, 0), (0, 1), (1, 1)):
        x = np.concatenate([x, cx * L_c + rng.uniform(2e3, 23e3, 5)])
        y = np.concatenate([y, cy * L_c + rng.uniform(2e3, 23e3, 5)])
        r = np.concatenate([r, np.full(5, 400.0)])
    n = x.shape[0]
    p = I._phys(dt=5.0)
    p.update({"nx": nx, "ny": nx, "Lx": nx * L_c, "Ly": nx * L_c,
              "modes": I.random_modes(rng, 4, nx * L_c, nx * L_c, 0.1)})
    fl = I._floes(x, y, r, np.ones(n), u=rng.normal(0, 0.05, n), v=rng.normal(0, 0.05, n))
    o = orc.Model(p, fl)
    g = ms.Model(p, fl, ms.MS_FP32)
    d = ms.Model(p, fl, ms.MS_FP32)
    g.set_launch(5, 128, 0, 1.3)
    d.set_launch(4, 128, 0, 1.3)
    for m in (o, g, d):
        m.step(5.0, 60)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)
    e = rel_errors(g.moments(), d.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)


def test_crowded_cells_match_oracle(orc, ms):
    """Floes squeezed towards each cell's centre line (many overlaps, so
    many contacts and list rebuilds by displacement), 40 steps: within the
    FP32 tolerance of the oracle."""
    s = I.batched_128x128(seed=13, nx=4)
    p, dt = s["params"], s["dt"]
    f = {k: v.copy() for k, v in s["floes"].items()}
    f["x"] = f["x"] + 0.2 * (np.floor(f["x"] / 25e3) * 25e3 + 12.5e3 - f["x"])
    o = orc.Model(p, f)
    g = ms.Model(p, f, ms.MS_FP32)
    g.set_launch(5, 128, 0, 1.3)
    o.step(dt, 40)
    g.step(dt, 40)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)
    assert g.info()["deep_contacts"] >= 0


def test_upload_inside_an_interval(ms):
    """ms_set_floes inside a coarse interval folds the floes' running window
    sums into the window first: the coarse solution after the interval agrees
    with variant 4 (which adds every step to the window) within the FP32
    tolerance (P_omega differs by about 2e-5 between two FP32 launch
    variants, the same as between two reduction orders of one)."""
    s = I.batched_128x128(seed=17, nx=8)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    res = []
    for variant in (4, 5):
        g = ms.Model(p, s["floes"], ms.MS_FP32)
        g.set_launch(variant, 128, 0, 1.3)
        g.step(dt, N0 + 43)
        g.set_floes(g.floes())
        g.step(dt, N0 - 43 + 5)
        res.append((g.coupling()["q"], g.moments()))
    for f in range(4):
        a, b = res[0][0][f], res[1][0][f]
        assert np.linalg.norm(a - b) <= TOL32 * np.linalg.norm(a), f
    e = rel_errors(res[1][1], res[0][1], p, 1e-6)
    assert e.max() <= 1e-4, report(e)


def test_checkpoint_inside_an_interval(ms, tmp_path):
    """A checkpoint written inside a gradual-update period carries the running
    window sums: the resumed run equals the uninterrupted one bit for bit."""
    s = I.batched_128x128(seed=11, nx=16)
    p, dt = s["params"], s["dt"]
    path = str(tmp_path / "v5.ck")
    a = ms.Model(p, s["floes"], ms.MS_FP32)
    b = ms.Model(p, s["floes"], ms.MS_FP32)
    c = ms.Model(p, s["floes"], ms.MS_FP32)
    for m in (a, b, c):
        m.set_launch(5, 128, 0, 1.3)
    a.step(dt, 235)
    b.step(dt, 137)
    b.save(path)
    c.load_checkpoint(path)
    assert c.info()["variant"] == 5
    c.step(dt, 98)
    _same(a, c)


def test_diverged_state_is_reported(ms):
    """Every floe given 1e12 m/s (finite, so the upload accepts it): the
    skins and reaches grow beyond the cells (every floe becomes a large one,
    lists overflow to the all-cell walk) and then turn inf and NaN; every
    class finishes its run, the step reports MS_ERR_UNSTABLE and the context
    stays usable."""
    s = ragged_scenario([0, 20, 100, 300, 700, 1000], seed=31)
    g = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    g.set_launch(5, 128, 0, 1.3)
    g.step(s["dt"], 3)
    f = g.floes()
    f["u"][:] = 1.0e12
    g.set_floes(f)
    with pytest.raises(ms.MsError) as e:
        g.step(s["dt"], 30)
    assert e.value.code == -3, str(e.value)
    assert np.all(np.isfinite(ms.Model(s["params"], s["floes"], ms.MS_FP32).moments()))


@pytest.mark.parametrize("scen", ["square", "powerlaw"])
def test_ocean_expansion_is_exact_to_fp32(orc, ms, scen):
    """The resident kernels evaluate the current from each floe's first-order
    expansion about a nearby centre, within a radius that keeps the dropped
    term below FP32 rounding.  Over the first 50 steps (before contacts and
    coupling amplify rounding) the moments stay as close to the oracle as the
    kernels that sum the modes every step (variant 4) do: within 2e-5 in
    every column, where a missing or wrong gradient term leaves 1e-4."""
    s = I.square_4x4() if scen == "square" else I.powerlaw_32x32(nx=4)
    p = s["params"]
    o = orc.Model(p, s["floes"])
    o.step(s["dt"], 50)
    for v in (4, 5):
        g = ms.Model(p, s["floes"], ms.MS_FP32)
        g.set_launch(v, 128, 0, 1.3)
        g.step(s["dt"], 50)
        e = rel_errors(g.moments(), o.moments(), p, 1e-6)
        assert e.max() <= 2e-5, (v, report(e))
