"""Sec. 4.4, floes driven into a wall: the uniform current (0.3, 0) pushes
the Sec. 4.1 floes against rigid walls at x = 0 and x = 4 (periodic in y).

Readings (the paper gives the boundary condition in one sentence):
  * the truth DEM's wall is the contact law of Eq. (2.2) with the wall as a
    floe at rest, without spin, of unbounded radius and at least the floe's
    thickness; a centre that would pass a wall stays on it;
  * the coarse Lax-Friedrichs step has ghost cells beyond the walls: zero
    (walls = 1, the zero Dirichlet condition as stated) or mirroring the
    boundary cell (walls = 2, an impermeable wall that keeps the coarse mass);
  * each cell's own DEM stays doubly periodic (Sec. 3.1).

CPU tests pin the oracle: the wall law is the limit of the pinned pair law
for an ever larger partner; a single floe comes to rest against the wall
with the wall holding exactly the drag at rest; the walled LF step equals the
periodic one on a grid padded with the ghost columns; the mirrored walls keep
the mass.  GPU tests compare the CUDA path with the oracle and run the
paper-size scenario."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from tests.parity import rel_errors, report

LX = 4.0
P = {"nx": 4, "ny": 4, "Lx": LX, "Ly": 2.0, "E": 1.0e3, "G": 0.7, "eta": 0.2, "mu": 0.3, "h_ref": 1.0,
     "rho_o": 1.0, "Cd": 613.0, "rho_ice": 1.0}


def test_wall_is_the_limit_of_an_unbounded_floe(orc):
    """The wall against floe l equals the pair law against a resting,
    non-spinning floe of radius R = 1e5 r_l (thicker than l) whose edge lies
    on the wall line, placed with no periodic image: forces and torque agree
    to the O(r/R) of the limit, contact or not, on both walls (a larger R
    would lose the overlap to the rounding of the partner's position)."""
    rng = np.random.default_rng(44)
    hits = 0
    for k in range(400):
        side = k % 2
        r = rng.uniform(0.005, 0.05)
        d = rng.uniform(-0.9, 1.2) * r
        x = d if side == 0 else LX - d
        u, v, w, h = rng.normal(0, 0.3), rng.normal(0, 0.3), rng.normal(0, 5.0), rng.uniform(0.5, 2.0)
        nw, o = orc.wall(P, LX, (x, u, v, w, r, h))
        R = 1.0e5 * r
        xj = -R if side == 0 else LX + R
        hit, op = orc.pair(P, 0.0, 0.0, (x, 1.0, u, v, w, r, h), (xj, 1.0, 0.0, 0.0, 0.0, R, 10.0 * h))
        assert nw == int(hit) == int(d < r), (k, d, r)
        if hit:
            hits += 1
            scale = np.abs(op[:3]).max()
            assert np.allclose(o[:3], op[:3], rtol=1e-4, atol=1e-9 * scale), (k, o[:3], op[:3])
            assert np.isclose(o[6], op[6], rtol=1e-6) and np.isclose(o[7], op[7], rtol=1e-4)
    assert hits > 250


def test_wall_mirror_symmetry(orc):
    """A floe at the left wall is the mirror image of one at the right wall:
    x -> Lx - x, u -> -u, omega -> -omega gives Fx -> -Fx, Fy -> Fy, T -> -T."""
    rng = np.random.default_rng(7)
    for _ in range(100):
        r = rng.uniform(0.01, 0.05)
        d = rng.uniform(-0.5, 0.99) * r
        u, v, w, h = rng.normal(0, 0.3), rng.normal(0, 0.3), rng.normal(0, 5.0), rng.uniform(0.5, 2.0)
        _, a = orc.wall(P, LX, (LX - d, u, v, w, r, h))
        _, b = orc.wall(P, LX, (d, -u, v, -w, r, h))
        assert np.allclose([b[0], b[1], b[2]], [-a[0], a[1], -a[2]], rtol=1e-12, atol=1e-15)


def test_floe_comes_to_rest_against_the_wall(orc):
    """One floe driven by the current u_o = (0.3, 0) into the right wall (the
    truth DEM, walls = 1): it stops with its centre inside the domain, and
    the wall then holds exactly the ocean drag at rest, Eq. (2.1c):
    Fx_wall = -Cd rho_o pi r^2 0.3^2."""
    r, h = 0.05, 1.0
    p = dict(P, nx=4, ny=2, uo_x=0.3, uo_y=0.0, walls=1, couple=0)
    fl = {"x": np.array([LX - 2.5 * r]), "y": np.array([1.0]), "theta": np.zeros(1), "u": np.array([0.3]),
          "v": np.zeros(1), "omega": np.zeros(1), "r": np.array([r]), "h": np.array([h])}
    t = orc.Truth(p, fl)
    t.step(1e-4, 30000)
    f = t.floes()
    assert 0.0 < f["x"][0] < LX and abs(f["u"][0]) < 1e-9 and abs(f["v"][0]) < 1e-12
    _, o = orc.wall(p, LX, (f["x"][0], f["u"][0], f["v"][0], f["omega"][0], r, h))
    at_rest = p["Cd"] * p["rho_o"] * np.pi * r * r * 0.3 ** 2
    assert abs(o[0] + at_rest) <= 1e-8 * at_rest, (o[0], at_rest)


def _random_lf(seed, nx, ny):
    rng = np.random.default_rng(seed)
    nc = nx * ny
    q = rng.uniform(0.2, 1.0, (4, nc))
    q[1:3] *= rng.choice([-1.0, 1.0], (2, nc))
    V = rng.normal(0.0, 0.3, (2, nc))
    S = rng.normal(0.0, 0.1, (4, nc))
    return q, V, S


def _pad(a, nx, ny):
    """[k][ny*nx] -> [k][ny*(nx+2)], interior columns 1..nx"""
    k = a.shape[0]
    out = np.zeros((k, ny, nx + 2))
    out[:, :, 1:nx + 1] = a.reshape(k, ny, nx)
    return out


def test_lf_zero_walls_is_the_zero_padded_periodic_step(orc):
    """walls = 1 equals the periodic LF step on the grid with a zero column
    on each side (reset to zero before every substep): bit for bit."""
    nx, ny, dx, dy, dtau = 7, 5, 0.3, 0.2, 0.05
    q, V, S = _random_lf(1, nx, ny)
    got = orc.lf_bc(nx, ny, dx, dy, q.ravel(), V.ravel(), S.ravel(), dtau, 3, 1).reshape(4, -1)
    qp, Vp, Sp = _pad(q, nx, ny), _pad(V, nx, ny), _pad(S, nx, ny)
    for _ in range(3):
        qp[:, :, 0] = 0.0
        qp[:, :, nx + 1] = 0.0
        qp = orc.lf(nx + 2, ny, dx, dy, qp.ravel(), Vp.ravel(), Sp.ravel(), dtau, 1).reshape(4, ny, nx + 2)
    assert np.array_equal(got, qp[:, :, 1:nx + 1].reshape(4, -1))
    # and it is not the periodic step
    per = orc.lf(nx, ny, dx, dy, q.ravel(), V.ravel(), S.ravel(), dtau, 3).reshape(4, -1)
    assert not np.allclose(per, got)


def test_lf_mirror_walls_is_the_mirror_padded_periodic_step(orc):
    """walls = 2 equals the periodic LF step on the padded grid whose ghost
    columns mirror the boundary columns before every substep (rho, rho v_y,
    P_omega copied, rho v_x and <v_x> negated): bit for bit."""
    nx, ny, dx, dy, dtau = 6, 4, 0.25, 0.3, 0.04
    q, V, S = _random_lf(2, nx, ny)
    got = orc.lf_bc(nx, ny, dx, dy, q.ravel(), V.ravel(), S.ravel(), dtau, 4, 2).reshape(4, -1)
    qp, Vp, Sp = _pad(q, nx, ny), _pad(V, nx, ny), _pad(S, nx, ny)
    Vp[0, :, 0], Vp[0, :, nx + 1] = -Vp[0, :, 1], -Vp[0, :, nx]
    sign = np.array([1.0, -1.0, 1.0, 1.0])[:, None]
    for _ in range(4):
        qp[:, :, 0] = sign * qp[:, :, 1]
        qp[:, :, nx + 1] = sign * qp[:, :, nx]
        qp = orc.lf(nx + 2, ny, dx, dy, qp.ravel(), Vp.ravel(), Sp.ravel(), dtau, 1).reshape(4, ny, nx + 2)
    assert np.array_equal(got, qp[:, :, 1:nx + 1].reshape(4, -1))


def test_lf_mirror_walls_keep_the_mass(orc):
    """Without sources the impermeable walls keep sum(rho) and sum(P_omega)
    over 50 substeps to rounding; the zero walls lose mass."""
    nx, ny, dx, dy, dtau = 9, 6, 0.2, 0.2, 0.05
    q, V, S = _random_lf(3, nx, ny)
    S[0] = 0.0
    S[3] = 0.0
    m2 = orc.lf_bc(nx, ny, dx, dy, q.ravel(), V.ravel(), S.ravel(), dtau, 50, 2).reshape(4, -1)
    m1 = orc.lf_bc(nx, ny, dx, dy, q.ravel(), V.ravel(), S.ravel(), dtau, 50, 1).reshape(4, -1)
    for f in (0, 3):
        assert abs(m2[f].sum() - q[f].sum()) <= 1e-13 * np.abs(q[f]).sum(), f
    assert m1[0].sum() < 0.9 * q[0].sum()


def test_truth_walls_binned_search_equals_all_pairs(orc):
    """With walls, the binned truth search (no image across x) gives the
    all-pairs loop's floes bit for bit as the floes pile up at the wall."""
    s = I.scenario44(48, 24, 6, 3)
    p = dict(s["params"], couple=0)
    fl = dict(s["floes"])
    fl["x"] = fl["x"] + 0.04   # the last column touches the right wall from the start
    a, b = orc.Truth(p, fl), orc.Truth(p, fl)
    a.set_brute(True)
    a.step(s["dt"], 300)
    b.step(s["dt"], 300)
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert fa["x"].max() <= LX and fa["x"].min() >= 0.0


def sweep44(make_truth, make_model, walls, nfx, nfy, grids, times):
    from tests.test_convergence4x import concentration, l2
    s = I.scenario44(nfx, nfy, 48, 24)
    dt = s["dt"]
    truth, done = {}, 0
    t = make_truth(dict(s["params"], couple=0, walls=walls), s["floes"])
    for T in times:
        n = int(round(T / dt))
        t.step(dt, n - done)
        done = n
        truth[T] = t.floes()
    errs = {T: [] for T in times}
    cols = {}
    for nx, ny in grids:
        s = I.scenario44(nfx, nfy, nx, ny)
        m, done = make_model(dict(s["params"], walls=walls), s["floes"]), 0
        for T in times:
            n = int(round(T / dt))
            m.step(dt, n - done)
            done = n
            c_ms = m.moments()[:, 6] / ((LX / nx) * (2.0 / ny))
            c_tr = concentration(truth[T], nx, ny)
            errs[T].append(l2(c_ms, c_tr, nx, ny))
            cols[(nx, T)] = (c_ms.reshape(ny, nx).mean(0), c_tr.reshape(ny, nx).mean(0))
    return errs, cols, truth


@pytest.mark.parametrize("walls", [1, 2])
def test_oracle_sec44(orc, walls):
    """Oracle on a quarter of the paper's floes per direction (96 x 48),
    grids 6 x 3 to 24 x 12, T = 0.2 and 1: the truth floes pile up at the
    right wall (its column's concentration above that of the column before
    it, every centre inside the walls); the msDEM error falls as the grid is
    refined at T = 0.2, and converges more slowly at T = 1 (Sec. 4.4: larger
    errors, lower rates than Secs. 4.1-4.3)."""
    import os
    from tests.test_convergence4x import order
    orc.set_threads(os.cpu_count() or 1)
    grids = ((6, 3), (12, 6), (24, 12))
    errs, cols, truth = sweep44(lambda p, f: orc.Truth(p, f), lambda p, f: orc.Model(p, f), walls, 96, 48,
                                grids, (0.2, 1.0))
    x = truth[1.0]["x"]
    assert x.min() >= 0.0 and x.max() <= LX
    ctr = cols[(24, 1.0)][1]
    assert ctr[-1] > ctr[-2] > 0.0, ctr
    e2 = errs[0.2]
    assert all(a > b for a, b in zip(e2, e2[1:])), e2
    assert order(grids, errs[1.0]) < order(grids, e2) and order(grids, e2) > 0.5, errs
    cms = cols[(24, 1.0)][0]
    if walls == 2:
        assert cms[-1] > cols[(24, 0.2)][0][-1], cms     # the coarse field piles up at the wall too


# ------------------------------------------------------------------ GPU
TOL64, TOL32 = 1e-10, 1e-4


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_walls_truth(orc, ms, precision):
    """The truth DEM between walls against the oracle: the Sec. 4.4 floes
    (96 x 48) shifted so that the last column presses on the right wall,
    300 steps; every centre stays inside the walls."""
    s = I.scenario44(96, 48, 12, 6)
    p = dict(s["params"], couple=0)
    fl = dict(s["floes"])
    fl["x"] = fl["x"] + 0.02
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    o = orc.Truth(p, fl)
    g = ms.Model(p, fl, precision)
    o.step(s["dt"], 300)
    g.truth_step(s["dt"], 300)
    e = rel_errors(g.truth_moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)
    f = g.truth_floes()
    assert f["x"].min() >= 0.0 and f["x"].max() <= LX
    if precision == 1:
        fo = o.floes()
        assert np.max(np.abs(f["x"] - fo["x"])) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("walls", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_walls_msdem(orc, ms, walls, precision):
    """msDEM with walls against the oracle: Sec. 4.4 on 96 x 48 floes and
    12 x 6 cells, 250 steps (two coarse steps with the walled LF step and
    the gradual updates they drive): moments and coarse state."""
    s = I.scenario44(96, 48, 12, 6)
    p = dict(s["params"], walls=walls)
    tol, eps = (TOL64, 1e-12) if precision == 1 else (TOL32, 1e-6)
    o = orc.Model(p, s["floes"])
    g = ms.Model(p, s["floes"], precision)
    o.step(s["dt"], 250)
    g.step(s["dt"], 250)
    e = rel_errors(g.moments(), o.moments(), p, eps)
    assert e.max() <= tol, report(e)
    qo, qg = o.coupling()["q"], g.coupling()["q"]
    assert np.linalg.norm(qg - qo) <= tol * np.linalg.norm(qo)


@pytest.mark.gpu
def test_gpu_sec44_paper_size(ms):
    """The paper's size, 480 x 240 = 115,200 floes, grids 12 x 6 to 48 x 24,
    FP32 path, T = 0.2, 0.6, 1, both wall readings: the truth floes pile up
    at the right wall and stay inside the walls; the msDEM error falls with
    dX at T = 0.2 and converges more slowly at T = 1 (Sec. 4.4); the mirrored
    walls keep the coarse mass and pile it up at the right wall, the zero
    walls lose mass through the walls."""
    from tests.test_convergence4x import order
    grids = ((12, 6), (24, 12), (48, 24))
    times = (0.2, 0.6, 1.0)

    def truth(p, f):
        m = ms.Model(p, f, ms.MS_FP32)

        class T:
            step = m.truth_step
            floes = m.truth_floes
        return T

    models = {}

    def model(p, f):
        m = ms.Model(p, f, ms.MS_FP32)
        models[(p["nx"], p["walls"])] = m
        return m

    for walls in (1, 2):
        errs, cols, tr = sweep44(truth, model, walls, 480, 240, grids, times)
        x = tr[1.0]["x"]
        assert x.min() >= 0.0 and x.max() <= LX
        ctr = cols[(48, 1.0)][1]
        assert ctr[-1] > ctr[-2], ctr
        e2 = errs[0.2]
        assert all(a > b for a, b in zip(e2, e2[1:])), errs
        assert order(grids, errs[1.0]) < order(grids, e2), errs
        # coarse mass at T = 1 against the floes' mass (rho_ice = h = 1), which
        # the first coarse step takes over from the cells' DEMs
        mass = models[(48, walls)].coupling()["q"][0].sum() * (LX / 48) * (2.0 / 24)
        m0 = float(np.sum(np.pi * I.scenario44(480, 240)["floes"]["r"] ** 2))
        if walls == 2:
            assert abs(mass - m0) <= 1e-6 * m0, (mass, m0)   # FP32 radii
            cms = cols[(48, 1.0)][0]
            assert cms[-1] > cols[(48, 0.2)][0][-1], cms
        else:
            assert mass < 0.99 * m0, (mass, m0)
        print(walls, {T: [round(v, 4) for v in errs[T]] for T in times},
              {T: round(order(grids, errs[T]), 3) for T in times}, "coarse mass / initial", mass / m0)
