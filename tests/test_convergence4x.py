"""The paper's Sec. 4.2 and 4.3 scenarios as convergence tests of the whole
coupled method against the truth DEM.

Both keep the floes, domain, time step and initial state of Sec. 4.1 and
change the ocean current: u_o = (0.3 - 0.1 cos(pi x), 0) gathers and
scatters the floes (Sec. 4.2, with collisions); u_o = (0.3 - 0.1 sin(0.1 pi
x) cos(pi y), 0.05 cos(0.1 pi x) sin(pi y)) is a mild compressible current
(Sec. 4.3).  The error is the L2 difference of the msDEM floe concentration
from the truth DEM's on the coarse grid (Sec. 4.1's norm).  The paper reports
orders close to one for short times in Sec. 4.2 and about 0.75 in Sec. 4.3,
smaller at later times.  The drag constant of these non-dimensional runs is
a reading (the paper gives none): see inputs.SEC4_DRAG."""
import os

import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I


def concentration(fl, nx, ny):
    dx, dy = 4.0 / nx, 2.0 / ny
    x, y = fl["x"] % 4.0, fl["y"] % 2.0
    cell = np.floor(y / dy).astype(int) * nx + np.floor(x / dx).astype(int)
    return np.bincount(cell, weights=np.pi * fl["r"] ** 2, minlength=nx * ny) / (dx * dy)


def l2(c_ms, c_tr, nx, ny):
    return float(np.sqrt(np.sum((c_ms - c_tr) ** 2) * (4.0 / nx) * (2.0 / ny)))


def order(grids, errs):
    d = np.log([4.0 / g[0] for g in grids])
    return float(np.polyfit(d, np.log(errs), 1)[0])


def sweep(make_truth, make_model, which, nfx, nfy, grids, times):
    """errors[T] over the grids; msDEM and truth advanced through the times."""
    s = I.scenario4x(which, nfx, nfy, 48, 24)
    dt = s["dt"]
    truth, done = {}, 0
    t = make_truth(dict(s["params"], couple=0), s["floes"])
    for T in times:
        n = int(round(T / dt))
        t.step(dt, n - done)
        done = n
        truth[T] = t.floes()
    errs = {T: [] for T in times}
    for nx, ny in grids:
        s = I.scenario4x(which, nfx, nfy, nx, ny)
        m, done = make_model(s["params"], s["floes"]), 0
        for T in times:
            n = int(round(T / dt))
            m.step(dt, n - done)
            done = n
            errs[T].append(l2(m.moments()[:, 6] / ((4.0 / nx) * (2.0 / ny)), concentration(truth[T], nx, ny),
                              nx, ny))
    return errs


@pytest.mark.parametrize("which", [2, 3])
def test_oracle_sec4x_converges(orc, which):
    """Oracle on a quarter of the paper's floes per direction (96 x 48),
    grids with 256 to 16 floes per cell, T = 0.2: the error falls as the
    coarse grid is refined, at an order of about one."""
    orc.set_threads(os.cpu_count() or 1)
    grids = ((6, 3), (12, 6), (24, 12))
    errs = sweep(lambda p, f: orc.Truth(p, f), lambda p, f: orc.Model(p, f), which, 96, 48, grids, (0.2,))[0.2]
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert 0.5 <= order(grids, errs) <= 1.5, errs


@pytest.mark.gpu
def test_gpu_sec4x_paper_size():
    """The paper's size, 480 x 240 = 115,200 floes, grids 12 x 6 to 48 x 24
    (1,600 to 100 floes per cell, the paper's finest), FP32 path, T = 0.2,
    0.6, 1: errors fall with dX at every time; Sec. 4.2 converges at an order
    close to one at T = 0.2; Sec. 4.3 at about 0.75 at T = 1, below its
    order at T = 0.2."""
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    grids = ((12, 6), (24, 12), (48, 24))
    times = (0.2, 0.6, 1.0)

    def truth(p, f):
        m = msdem.Model(p, f, msdem.MS_FP32)

        class T:
            step = m.truth_step
            floes = m.truth_floes
        return T

    model = lambda p, f: msdem.Model(p, f, msdem.MS_FP32)
    e2 = sweep(truth, model, 2, 480, 240, grids, times)
    e3 = sweep(truth, model, 3, 480, 240, grids, times)
    for e in (e2, e3):
        for T in times:
            assert all(a > b for a, b in zip(e[T], e[T][1:])), (T, e[T])
    assert 0.8 <= order(grids, e2[0.2]) <= 1.6, e2
    o3 = {T: order(grids, e3[T]) for T in times}
    assert 0.5 <= o3[1.0] <= 1.0 and o3[1.0] < o3[0.2], o3
