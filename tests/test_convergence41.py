"""The paper's Sec. 4.1 scenario as a pin of the whole coupled method.

Floes drift with the uniform current and never touch, so the truth DEM is an
exact translation and its concentration field is known in closed form.  The
msDEM concentration error (L2 over the coarse cells, Sec. 4.1) must shrink
with the coarse cell size dX; at a fixed Courant number the Lax-Friedrichs
scheme is first order, and the paper reports order one for short times.
It must not depend on the number of floes per cell (no floe-sampling error in
this scenario)."""
import os

import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I

T = 0.24
GRIDS = ((6, 3), (12, 6), (24, 12), (48, 24))


def truth_concentration(s, nx, ny, T):
    fl = s["floes"]
    dx, dy = 4.0 / nx, 2.0 / ny
    x = (fl["x"] + 0.3 * T) % 4.0
    cell = np.floor(fl["y"] / dy).astype(int) * nx + np.floor(x / dx).astype(int)
    return np.bincount(cell, weights=np.pi * fl["r"] ** 2, minlength=nx * ny) / (dx * dy)


def errors(run, nfx, nfy, grids, fixed_courant):
    out = []
    for nx, ny in grids:
        s = I.scenario41(nfx=nfx, nfy=nfy, nx=nx, ny=ny)
        p = s["params"]
        if fixed_courant:
            p["N0"] = int(round(100 * 48 / nx))     # dT = N0 dt proportional to dX
        mo = run(p, s)
        dx, dy = 4.0 / nx, 2.0 / ny
        c_ms = mo[:, 6] / (dx * dy)
        e = np.sqrt(np.sum((c_ms - truth_concentration(s, nx, ny, T)) ** 2) * dx * dy)
        out.append((dx, e))
    return out


def slopes(res):
    d = np.log([r[0] for r in res])
    e = np.log([r[1] for r in res])
    return np.diff(e) / np.diff(d)


def test_oracle_converges_first_order(orc):
    orc.set_threads(os.cpu_count() or 1)

    def run(p, s):
        m = orc.Model(p, s["floes"])
        m.step(s["dt"], int(round(T / s["dt"])))
        return m.moments()

    res = errors(run, 96, 48, GRIDS, fixed_courant=True)
    e = [r[1] for r in res]
    sl = slopes(res)
    assert all(a > b for a, b in zip(e, e[1:])), e
    assert 0.7 <= sl[-1] <= 1.2, sl              # the finest pair is in the first-order regime
    assert sl[0] < sl[1] < sl[2], sl             # and the order rises towards one as dX shrinks
    # twice the floes in each direction: same errors (no sampling error here)
    res2 = errors(run, 192, 96, GRIDS[2:], fixed_courant=True)
    for (d1, e1), (d2, e2) in zip(res[2:], res2):
        assert abs(e1 - e2) <= 0.05 * e1


@pytest.mark.gpu
def test_gpu_paper_size_converges():
    """Sec. 4.1 at the paper's size: 480 x 240 = 115,200 floes, coarse grids
    12 x 6 to 96 x 48, FP32 path, dt = 1e-4, fixed Courant number; the same
    decreasing, first-order errors as the oracle."""
    from paper_2303_07819_gb300 import msdem
    msdem.load()

    def run(p, s):
        m = msdem.Model(p, s["floes"], msdem.MS_FP32)
        m.step(s["dt"], int(round(T / s["dt"])))
        return m.moments()

    res = errors(run, 480, 240, ((12, 6), (24, 12), (48, 24), (96, 48)), fixed_courant=True)
    e = [r[1] for r in res]
    sl = slopes(res)
    assert all(a > b for a, b in zip(e, e[1:])), e
    assert 0.7 <= sl[-1] <= 1.3, sl
