"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (relative, per moment field, 2-norm over cells):
  FP64 path  <= 1e-10 over 100 steps (and through the first coarse steps);
  FP32 path  <= 1e-4  over 100 steps.
"""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from tests.parity import rel_errors, report

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def run_pair(orc, ms, scen, precision, nsteps, params=None):
    p = dict(scen["params"], **(params or {}))
    o = orc.Model(p, scen["floes"])
    g = ms.Model(p, scen["floes"], precision)
    o.step(scen["dt"], nsteps)
    g.step(scen["dt"], nsteps)
    return o, g, p


@pytest.mark.parametrize("nsteps", [1, 100, 250])
def test_fp64_msdem_square(orc, ms, nsteps):
    s = I.square_4x4()
    o, g, p = run_pair(orc, ms, s, ms.MS_FP64, nsteps)
    e = rel_errors(g.moments(), o.moments(), p, 1e-12)
    assert e.max() <= TOL64, report(e)
    if nsteps >= 100:
        co, cg = o.coupling(), g.coupling()
        assert cg["have_q"] == co["have_q"] and cg["have_targets"] == co["have_targets"]
        for key in ("q", "targets"):
            a, b = cg[key], co[key]
            assert np.linalg.norm(a - b) <= TOL64 * max(np.linalg.norm(b), 1e-300), key


def test_fp64_msdem_floes_square(orc, ms):
    s = I.square_4x4()
    o, g, p = run_pair(orc, ms, s, ms.MS_FP64, 100)
    fo, fg = o.floes(), g.floes()
    assert np.max(np.abs(fo["x"] - fg["x"])) < 1e-6 and np.max(np.abs(fo["y"] - fg["y"])) < 1e-6
    for k in ("u", "v", "omega", "r"):
        assert np.linalg.norm(fo[k] - fg[k]) <= TOL64 * np.linalg.norm(fo[k]) + 1e-20, k


def test_fp32_msdem_square(orc, ms):
    s = I.square_4x4()
    o, g, p = run_pair(orc, ms, s, ms.MS_FP32, 100)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)


@pytest.mark.parametrize("precision", [0, 1])
def test_msdem_powerlaw_small(orc, ms, precision):
    """The power-law workload's laws (power-law radii, lognormal thickness, 8 Fourier modes,
    wind) on 4 x 4 cells of 12.5 km, ~1000 floes, cells up to ~90 floes."""
    s = I.powerlaw_32x32(nx=4)
    o, g, p = run_pair(orc, ms, s, precision, 100)
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    e = rel_errors(g.moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)


@pytest.mark.parametrize("precision", [0, 1])
def test_truth_square(orc, ms, precision):
    s = I.square_4x4()
    p = s["params"]
    o = orc.Truth(p, s["floes"])
    g = ms.Model(p, s["floes"], precision)
    o.step(s["dt"], 100)
    g.truth_step(s["dt"], 100)
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    e = rel_errors(g.truth_moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)


def test_truth_powerlaw_small_fp64(orc, ms):
    s = I.powerlaw_32x32(nx=4)
    p = s["params"]
    o = orc.Truth(p, s["floes"])
    g = ms.Model(p, s["floes"], ms.MS_FP64)
    o.step(s["dt"], 50)
    g.truth_step(s["dt"], 50)
    e = rel_errors(g.truth_moments(), o.moments(), p, 1e-12)
    assert e.max() <= TOL64, report(e)


@pytest.mark.parametrize("precision", [0, 1])
def test_velocity_modes_msdem_and_truth(orc, ms, precision):
    """Compressible velocity-mode currents against the oracle: the Sec. 4.3
    current (real wave numbers, not periodic over the domain) on 96 x 48
    floes and 12 x 6 cells (64 per cell), msDEM over two coarse steps and the
    truth DEM; then stream-function and velocity modes together on the power-law workload's
    cells."""
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    s = I.scenario4x(3, 96, 48, 12, 6)
    p = s["params"]
    o, g, _ = run_pair(orc, ms, s, precision, 250)
    e = rel_errors(g.moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)
    ot = orc.Truth(dict(p, couple=0), s["floes"])
    gt = ms.Model(dict(p, couple=0), s["floes"], precision)
    ot.step(s["dt"], 200)
    gt.truth_step(s["dt"], 200)
    e = rel_errors(gt.truth_moments(), ot.moments(), p, eps)
    assert e.max() <= tol, report(e)
    # stream-function modes and velocity modes together (the power-law workload's laws)
    c = I.powerlaw_32x32(nx=4)
    L = c["params"]["Lx"]
    vm = np.array([[0.03, -0.02, 2 * np.pi * 1.3 / L, 2 * np.pi * 0.4 / L, 0.3],
                   [-0.01, 0.04, 2 * np.pi * -0.7 / L, 2 * np.pi * 2.1 / L, 1.1]])
    o, g, p = run_pair(orc, ms, c, precision, 100, params={"vmodes": vm})
    e = rel_errors(g.moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)


def ragged_scenario(counts, L_c=12.5e3, seed=5):
    """Cells with the given floe counts (0 allowed) on a small periodic grid,
    power-law radii rescaled to 45% cover, the power-law workload's forcing."""
    rng = np.random.default_rng(seed)
    nx = ny = int(np.ceil(np.sqrt(len(counts))))
    counts = list(counts) + [0] * (nx * ny - len(counts))
    L = L_c * nx
    radii = [I.power_law_radii(rng, int(c), 100.0, 1500.0) for c in counts]
    radii, _ = I._rescale_cells(radii, L_c * L_c, 0.45)
    x, y, r, cell = I.place_floes(rng, nx, ny, L, L, radii, domain_check=False)
    h = I.lognormal_mean_sd(rng, x.shape[0], 1.5, 0.5)
    p = I._phys(dt=5.0)
    p.update({"nx": nx, "ny": ny, "Lx": L, "Ly": L, "modes": I.random_modes(rng, 8, L, L, 0.1),
              "Ca": 1.2e-3, "wind_x": 10.0, "wind_y": 0.0})
    fl = I._floes(x, y, r, h)
    fl["u"] = rng.normal(0, 0.1, x.shape[0])
    fl["v"] = rng.normal(0, 0.1, x.shape[0])
    return {"params": p, "floes": fl, "dt": 5.0}


@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_and_empty_cells(orc, ms, precision):
    """Cells of 0, 1, 2, 31, 33, 64, 127, 129, 300 floes: empty cells, a lone
    floe, and counts on both sides of the warp and block tiles."""
    s = ragged_scenario([0, 1, 2, 31, 33, 64, 127, 129, 300])
    o, g, p = run_pair(orc, ms, s, precision, 30)
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    mo, mg = o.moments(), g.moments()
    assert np.array_equal(mo[:, 0], mg[:, 0])
    e = rel_errors(mg, mo, p, eps)
    assert e.max() <= tol, report(e)


def test_no_floes(ms):
    p = dict(I.square_4x4()["params"])
    fl = {k: np.zeros(0) for k in ("x", "y", "theta", "u", "v", "omega", "r", "h")}
    g = ms.Model(p, fl, ms.MS_FP32)
    g.step(10.0, 150)
    assert np.all(g.moments() == 0.0)
    g.truth_step(10.0, 3)
    assert np.all(g.truth_moments() == 0.0)


def test_diverged_state_is_reported(ms):
    """Every floe given 1e12 m/s (finite, so the upload accepts it): drag and
    forward Euler drive the state through huge finite values to inf and NaN
    within a few steps.  The list rebuilds meanwhile see a skin of 4 |v|max
    dt n_t far beyond the cell; the large-floe bin search caps its reach at
    the cell side, so packed, warp-list and block-list cells all finish their
    steps, the step reports MS_ERR_UNSTABLE, and the context stays usable."""
    s = ragged_scenario([0, 20, 100, 300, 700], seed=31)
    g = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    g.set_launch(4, 128, 0, 1.3)
    g.step(s["dt"], 3)
    f = g.floes()
    f["u"][:] = 1.0e12
    g.set_floes(f)
    with pytest.raises(ms.MsError) as e:
        g.step(s["dt"], 30)
    assert e.value.code == -3, str(e.value)
    assert g.moments().shape[0] == 9
    assert np.all(np.isfinite(ms.Model(s["params"], s["floes"], ms.MS_FP32).moments()))


def test_largest_cell_fp32(orc, ms):
    """A cell at the 4096-floe limit (several shared-memory tiles), one step."""
    s = ragged_scenario([4096], L_c=100e3, seed=9)
    p = dict(s["params"], couple=0)
    o, g, _ = run_pair(orc, ms, s, ms.MS_FP32, 1, params=p)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= 1e-5, report(e)


def test_graph_replay_equals_single_steps(ms):
    s = I.square_4x4()
    a = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    b = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    a.step(s["dt"], 230)
    for _ in range(230):
        b.step(s["dt"], 1)
    assert a.info()["graph_replays"] >= 2 and b.info()["graph_replays"] == 0
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_resident_run_equals_single_steps(ms):
    """Variant 3 keeps each warp cell in shared memory for a whole coarse
    interval (one launch per interval on the graph path) and runs one step
    per launch otherwise: the two give the same floes and moments bitwise,
    across coarse steps and gradual updates."""
    s = I.batched_128x128(seed=7, nx=16)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    a = ms.Model(p, s["floes"], ms.MS_FP32)
    b = ms.Model(p, s["floes"], ms.MS_FP32)
    a.set_launch(3, 128, 0, 1.3)
    b.set_launch(3, 128, 0, 1.3)
    a.step(dt, 2 * N0 + 17)
    for _ in range(2 * N0 + 17):
        b.step(dt, 1)
    assert a.info()["graph_replays"] == 2 and b.info()["graph_replays"] == 0
    li = a.info()["launches_per_interval"]
    assert 1 <= li % N0 <= 5           # one launch per warp or packed class, N0 per block class
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.moments(), b.moments())
    assert np.array_equal(a.coupling()["q"], b.coupling()["q"])


def test_neighbour_lists_graph_equals_single_steps(ms):
    """Variant 4 keeps candidate lists in device memory across steps; an
    interval replayed from the graph and the same steps launched one by one
    give the same floes bitwise, across list rebuilds, coarse steps and
    gradual updates; after set_floes the lists are rebuilt (a moved floe must
    not keep stale partners)."""
    s = I.batched_128x128(seed=9, nx=16)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    a = ms.Model(p, s["floes"], ms.MS_FP32)
    b = ms.Model(p, s["floes"], ms.MS_FP32)
    a.set_launch(4, 128, 0, 1.3)
    b.set_launch(4, 128, 0, 1.3)
    a.step(dt, 2 * N0 + 23)
    for _ in range(2 * N0 + 23):
        b.step(dt, 1)
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.moments(), b.moments())
    # squeeze every cell's floes a quarter of the way towards its centre line
    # through the public API (many new overlaps): variant 4 must search again
    # and agree with variant 2 given the same floes
    d = ms.Model(p, s["floes"], ms.MS_FP32)
    d.set_launch(2, 128, 0, 1.3)
    d.step(dt, 2 * N0 + 23)
    f = a.floes()
    f["x"] = f["x"] + 0.25 * (np.floor(f["x"] / 25e3) * 25e3 + 12.5e3 - f["x"])
    a.set_floes(f)
    d.set_floes(f)
    a.step(dt, 7)
    d.step(dt, 7)
    ea = rel_errors(a.moments(), d.moments(), p, 1e-6)
    assert ea.max() < 1e-4, report(ea)


def test_launch_variants_agree(ms):
    """Threads per block and the persistent work queue change only the order
    of the moment reduction, never a floe's arithmetic: floes agree bitwise
    until the first coarse step, which feeds the reduced moments back."""
    s = I.powerlaw_32x32(nx=4)
    ref = refm = None
    for threads in (64, 128, 256):
        for persistent in (0, 1):
            g = ms.Model(s["params"], s["floes"], ms.MS_FP32)
            g.set_launch(0, threads, persistent)
            g.step(s["dt"], 99)
            f = g.floes()
            g.step(s["dt"], 31)
            mo = g.moments()
            if ref is None:
                ref, refm = f, mo
            for k in f:
                assert np.array_equal(f[k], ref[k]), (threads, persistent, k)
            e = rel_errors(mo, refm, s["params"], 1e-6)
            assert e.max() < 1e-5, report(e)


def test_autotune_keeps_results(ms):
    s = I.powerlaw_32x32(nx=8)
    a = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    b = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    best = b.autotune(s["dt"], reps=3)
    assert best > 0
    ib = b.info()
    a.set_launch(ib["variant"], ib["threads"], ib["persistent"], ib["bin_beta_milli"] / 1000.0)
    a.set_resident(ib["skin_steps_milli"] / 1000.0, ib["block_floes"])
    assert a.info()["block_floes"] == ib["block_floes"]
    a.step(s["dt"], 120)
    b.step(s["dt"], 120)
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    ea = rel_errors(b.moments(), a.moments(), s["params"], 1e-6)
    assert ea.max() < 1e-6, report(ea)


def test_time_kernel_leaves_state(ms):
    s = I.square_4x4()
    a = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    a.step(s["dt"], 5)
    before = a.floes()
    t0 = a.time_kernel(0, s["dt"], 5)
    t1 = a.time_kernel(1, s["dt"], 5)
    t2 = a.time_kernel(2, s["dt"], 2)
    assert t0 > 0 and t1 > 0 and t2 > t0
    after = a.floes()
    for k in before:
        assert np.array_equal(before[k], after[k])


def test_argument_errors(ms):
    s = I.square_4x4()
    g = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    g.step(10.0, 1)
    with pytest.raises(ms.MsError) as e:
        g.step(5.0, 1)
    assert e.value.code == -1
    bad = {k: v.copy() for k, v in s["floes"].items()}
    bad["u"][3] = np.nan
    with pytest.raises(ms.MsError):
        ms.Model(s["params"], bad, ms.MS_FP32)
    big = {k: v.copy() for k, v in s["floes"].items()}
    big["r"][0] = 7000.0           # 2 r >= L_c / 2 = 12.5 km
    with pytest.raises(ms.MsError):
        ms.Model(s["params"], big, ms.MS_FP32)
    moved = g.floes()
    moved["x"][0] += 30e3          # into another cell
    with pytest.raises(ms.MsError):
        g.set_floes(moved)


def test_set_floes_roundtrip(ms):
    s = I.square_4x4()
    g = ms.Model(s["params"], s["floes"], ms.MS_FP64)
    g.step(10.0, 7)
    f = g.floes()
    g.set_floes(f)
    f2 = g.floes()
    for k in f:
        assert np.array_equal(f[k], f2[k]), k


def test_set_floes_from_page_locked_memory(ms):
    """ms_set_floes sends page-locked arrays without a host copy and others
    through its staging buffer: the same state either way, then the same
    steps; a bad value in page-locked memory is still refused."""
    torch = pytest.importorskip("torch")
    s = I.powerlaw_32x32(nx=8)
    a = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    b = ms.Model(s["params"], s["floes"], ms.MS_FP32)
    for m in (a, b):                 # the same coupling state in both
        m.step(s["dt"], 30)
    f = a.floes()
    pinned = torch.empty((8, a.n), dtype=torch.float64).pin_memory().numpy()
    fp = {k: pinned[i] for i, k in enumerate(ms.FLOE_KEYS)}
    for k in f:
        fp[k][:] = f[k]
    a.set_floes(fp)
    b.set_floes(f)
    for m in (a, b):
        m.step(s["dt"], 120)
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert np.array_equal(a.moments(), b.moments())
    fp["h"][17] = -1.0
    with pytest.raises(ms.MsError, match="floe 17"):
        a.set_floes(fp)
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_fp32_variants_match_oracle(orc, ms, variant):
    """Brute-force, block-binned, warp-binned, resident warp-binned and
    neighbour-list pair search: each within the FP32 tolerance of the oracle
    over 100 steps on a ragged mix of cells (0 to 300 floes, so every size
    class and every launch kind runs)."""
    s = ragged_scenario([0, 1, 5, 17, 31, 33, 64, 65, 100, 127, 129, 200, 256, 257, 300], seed=21)
    p = s["params"]
    o = orc.Model(p, s["floes"])
    g = ms.Model(p, s["floes"], ms.MS_FP32)
    g.set_launch(variant, 128, 0, 1.0)
    o.step(s["dt"], 100)
    g.step(s["dt"], 100)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)


def test_neighbour_lists_every_class_match_oracle(orc, ms):
    """Variant 4 over 100 steps (ten list rebuilds, list steps between them,
    a coarse step) on cells in every size class: the four block classes (300,
    400, 520 and 700 floes), the warp classes and the packed one; within the
    FP32 tolerance of the oracle."""
    s = ragged_scenario([0, 1, 20, 35, 70, 130, 200, 300, 400, 520, 700], seed=23)
    p = s["params"]
    o = orc.Model(p, s["floes"])
    g = ms.Model(p, s["floes"], ms.MS_FP32)
    g.set_launch(4, 128, 0, 1.3)
    o.step(s["dt"], 100)
    g.step(s["dt"], 100)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)


def test_neighbour_list_overflow(orc, ms):
    """A 3 km floe ringed by 60 floes of 150 m that touch it: its candidate
    list (at most 31 entries) overflows, so its cell searches again every
    step; the result stays within the FP32 tolerance of the oracle and of
    the warp-binned kernel (variant 2) over 30 steps."""
    rng = np.random.default_rng(31)
    L_c, nx = 25e3, 2
    ang = 2 * np.pi * (np.arange(60) + 0.5) / 60
    x = np.concatenate([[12.5e3], 12.5e3 + 3140.0 * np.cos(ang)])
    y = np.concatenate([[12.5e3], 12.5e3 + 3140.0 * np.sin(ang)])
    r = np.concatenate([[3000.0], np.full(60, 150.0)])
    # a few loose floes in the other cells
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
    g.set_launch(4, 128, 0, 1.3)
    d.set_launch(2, 128, 0, 1.3)
    for m in (o, g, d):
        m.step(5.0, 30)
    e = rel_errors(g.moments(), o.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)
    e = rel_errors(g.moments(), d.moments(), p, 1e-6)
    assert e.max() <= TOL32, report(e)


def test_fp32_variants_agree_one_step(ms):
    """One step of the power-law workload's laws on 16 x 16 cells: the pair searches
    find the same contacts, so moments agree to FP32 summation order."""
    s = I.powerlaw_32x32(nx=16)
    res = []
    for variant in (0, 1, 2, 3, 4, 5):
        g = ms.Model(s["params"], s["floes"], ms.MS_FP32)
        g.set_launch(variant, 128, 0, 1.0)
        g.step(s["dt"], 1)
        res.append(g.moments())
    for r in res[1:]:
        e = rel_errors(r, res[0], s["params"], 1e-6)
        assert e.max() < 1e-6, report(e)


def test_fp32_probe(ms):
    """The FMA probe (the FP32-pipe roofline's denominator) reports a rate
    between 30 and 100 TFLOP/s on a GB300 (nominal 152 SMs x 128 lanes x 2
    flops x 2.07 GHz = 80.6); reps < 1 is an argument error."""
    t = ms.probe_fp32(3)
    assert 30.0 < t < 100.0, t
    with pytest.raises(ms.MsError) as e:
        ms.probe_fp32(0)
    assert e.value.code == -1
