"""The allocation-free moments entry point (ms_cell_moments_noalloc) against
the library's other entry points.

It serves callers that cannot call cudaMalloc while they run (a code that
reserves all device memory up front, a framework whose allocator owns the
device): its working memory is a fixed array compiled into the library.  The
test calls it twice in a row through the C-ABI, so the second call runs on the
scratch the first one left behind, and compares each result with the moments
that ms_moments and ms_truth_moments report for the same floes, at the FP64
tolerance of the other parity tests.  This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from tests.parity import rel_errors, report

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
KEYS = ("x", "y", "u", "v", "omega", "r", "h")


def _call(ms, torch, p, fl, fd=None):
    dev = {k: torch.tensor(np.ascontiguousarray(fl[k]), dtype=torch.float64, device="cuda") for k in KEYS}
    n = int(dev["x"].shape[0])
    fdd = torch.zeros((3, n), dtype=torch.float64, device="cuda") if fd is None else \
        torch.tensor(np.ascontiguousarray(fd), dtype=torch.float64, device="cuda")
    ncell = int(p["nx"]) * int(p["ny"])
    out = torch.full((ncell, 12), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    ms.cell_moments_noalloc(p, n, *(dev[k].data_ptr() for k in KEYS), fdd.data_ptr(), out.data_ptr(), stream)
    return out.cpu().numpy()


def test_noalloc_moments_match_existing_entry_points():
    torch = pytest.importorskip("torch")
    from paper_2303_07819_gb300 import msdem as ms
    ms.load()
    s = I.square_4x4()
    p = s["params"]
    m = ms.Model(p, s["floes"], ms.MS_FP64)

    # call 1: the initial floes, against ms_moments of the new model (zero drag)
    got1 = _call(ms, torch, p, s["floes"])
    e1 = rel_errors(got1, m.moments(), p, 1e-12)
    assert e1.max() <= TOL64, report(e1)

    # call 2, right after: the truth DEM after 40 steps, against ms_truth_moments
    # (columns 0-8; the per-floe drag is not exposed, so it is passed as zeros)
    m.truth_step(s["dt"], 40)
    ref2 = m.truth_moments()
    tf = m.truth_floes()
    got2 = _call(ms, torch, p, tf)
    e2 = rel_errors(got2, ref2, p, 1e-12)[:9]
    assert e2.max() <= TOL64, report(e2)
    assert np.array_equal(got2[:, 0], ref2[:, 0])

    # call 3: a drag field, summed per cell by the same binning
    rng = np.random.default_rng(3)
    fd = rng.normal(size=(3, tf["x"].shape[0]))
    got3 = _call(ms, torch, p, tf, fd)
    dx = p["Lx"] / p["nx"]
    cell = (np.floor(tf["y"] / dx).astype(int) * p["nx"] + np.floor(tf["x"] / dx).astype(int))
    for k in range(3):
        ref = np.bincount(cell, weights=fd[k], minlength=p["nx"] * p["ny"])
        assert np.allclose(got3[:, 9 + k], ref, rtol=1e-12, atol=1e-12)
    m.close()


def test_noalloc_half_open_cells_with_wrap():
    """Floes on a cell's left edge, at X = Lx and at negative coordinates
    (positions a caller has not wrapped) land in the cells the oracle and
    ms_init give them: the coordinate wrapped into the periodic domain, then
    the half-open cell (reading c23).  Two calls in a row, against the
    oracle's moments of the same floes and against ms_moments."""
    torch = pytest.importorskip("torch")
    from oracle import oracle as O
    from paper_2303_07819_gb300 import msdem as ms
    ms.load()
    O.build()
    L = 4.0e4
    dX = L / 4
    xs = [dX, 2 * dX, L, -dX, 0.5 * dX, -L - 0.5 * dX, 2 * L + dX]
    ys = [0.5 * dX, dX, 3 * dX, 0.5 * dX, -0.5 * dX, L, -3 * L + 2.5 * dX]
    n = len(xs)
    fl = {"x": np.array(xs), "y": np.array(ys), "theta": np.zeros(n), "u": np.linspace(0.1, 0.7, n),
          "v": np.linspace(-0.2, 0.3, n), "omega": np.linspace(1e-5, 3e-5, n), "r": np.linspace(100.0, 160.0, n),
          "h": np.linspace(1.0, 2.0, n)}
    p = I._phys(dt=5.0)
    p.update({"nx": 4, "ny": 4, "Lx": L, "Ly": L, "modes": np.zeros((0, 4))})
    o = O.Model(p, fl)
    ref = o.moments()
    m = ms.Model(p, fl, ms.MS_FP64)
    for _ in range(2):
        got = _call(ms, torch, p, fl)
        assert np.array_equal(got[:, 0], ref[:, 0]), (got[:, 0], ref[:, 0])
        assert got[:, 0].tolist() == [0, 1, 0, 2, 0, 0, 1, 0, 0, 1, 0, 0, 2, 0, 0, 0]
        e = rel_errors(got, ref, p, 1e-12)
        assert e.max() <= TOL64, report(e)
        e = rel_errors(got, m.moments(), p, 1e-12)
        assert e.max() <= TOL64, report(e)
    m.close()
    o.close()


def test_noalloc_rejects_oversize():
    pytest.importorskip("torch")
    from paper_2303_07819_gb300 import msdem as ms
    p = {"nx": 256, "ny": 256, "Lx": 1e6, "Ly": 1e6, "rho_ice": 920.0}
    with pytest.raises(ms.MsError) as e:
        ms.cell_moments_noalloc(p, 10, *([0] * 9))
    assert e.value.code == -1 and "16384 cells" in str(e.value)
    p = {"nx": 4, "ny": 4, "Lx": 1e5, "Ly": 1e5, "rho_ice": 920.0}
    with pytest.raises(ms.MsError) as e:
        ms.cell_moments_noalloc(p, 1 << 19, *([0] * 9))
    assert e.value.code == -1 and "262144 floes" in str(e.value)
