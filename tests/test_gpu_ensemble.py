"""Ensemble batch: nens independent realizations (same grid and forcing, own
floes) advanced as one model must give what nens separate models give, and
each realization must match the oracle run on its own."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from tests.parity import rel_errors, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def realizations(R=3, nx=4):
    """The power-law workload's laws on nx x nx cells, one seed per realization, the first
    realization's ocean for all."""
    scens = [I.powerlaw_32x32(seed=100 + e, nx=nx) for e in range(R)]
    for sc in scens[1:]:
        sc["params"]["modes"] = scens[0]["params"]["modes"]
    return scens


@pytest.mark.parametrize("precision, variant", [(0, 4), (1, 0)])
def test_ensemble_equals_separate_models(ms, precision, variant):
    """Floes, moments and coarse state of the batched ensemble are those of
    the separate models through two coarse steps (graph path) and 50 single
    steps: bit for bit in FP32 (positions are fixed point of the cell, so the
    stacking offset e Ly leaves them unchanged); in FP64 the stacked y = y +
    e Ly rounds the offsets within the cell by an ulp of e Ly, so there the
    two agree to 1e-10.  FP32 with the warp-per-cell kernels (variant 4),
    whose sums over a cell do not depend on the other cells."""
    scens = realizations()
    ens = I.stack_ensemble(scens)
    dt, nsteps = ens["dt"], 250
    g = ms.Model(ens["params"], ens["floes"], precision)
    g.set_launch(variant, 128, 0, 1.3)
    g.step(dt, nsteps)
    fe, me, qe = g.floes(), g.moments(), g.coupling()["q"]
    nc = scens[0]["params"]["nx"] * scens[0]["params"]["ny"]
    off = 0
    for e, sc in enumerate(scens):
        m = ms.Model(sc["params"], sc["floes"], precision)
        m.set_launch(variant, 128, 0, 1.3)
        m.step(dt, nsteps)
        f = m.floes()
        n = f["x"].shape[0]
        for k in f:
            want = f[k] + (e * sc["params"]["Ly"] if k == "y" else 0.0)
            if precision == 0:
                assert np.array_equal(fe[k][off:off + n], want), (e, k)
            else:
                assert np.allclose(fe[k][off:off + n], want, rtol=1e-10, atol=1e-6 if k in "xy" else 1e-12), (e, k)
        if precision == 0:
            assert np.array_equal(me[e * nc:(e + 1) * nc], m.moments()), e
            assert np.array_equal(qe[:, e * nc:(e + 1) * nc], m.coupling()["q"]), e
        else:
            err = rel_errors(me[e * nc:(e + 1) * nc], m.moments(), sc["params"], 1e-12)
            assert err.max() <= 1e-10, report(err)
            q0, q1 = qe[:, e * nc:(e + 1) * nc], m.coupling()["q"]
            assert np.linalg.norm(q0 - q1) <= 1e-10 * np.linalg.norm(q1), e
        off += n
        m.close()


def test_ensemble_resident_blocks(ms):
    """The resident block kernels (variant 5, the default) pack cells of all
    realizations into shared blocks, differently from separate models.  A
    floe's arithmetic does not depend on its block and the per-cell sums are
    exact integer sums, so through coarse steps and gradual updates the
    ensemble's floes, moments and coarse states are the separate models'
    bit for bit."""
    scens = realizations()
    ens = I.stack_ensemble(scens)
    dt = ens["dt"]
    N0 = ens["params"]["N0"]
    g = ms.Model(ens["params"], ens["floes"], 0)
    assert g.info()["variant"] == 5
    seps = [ms.Model(sc["params"], sc["floes"], 0) for sc in scens]
    nc = scens[0]["params"]["nx"] * scens[0]["params"]["ny"]
    for nsteps in (N0 - 1, 2 * N0 + 51):
        g.step(dt, nsteps)
        fe, me, qe = g.floes(), g.moments(), g.coupling()["q"]
        off = 0
        for e, (sc, m) in enumerate(zip(scens, seps)):
            m.step(dt, nsteps)
            f = m.floes()
            n = f["x"].shape[0]
            for k in f:
                want = f[k] + (e * sc["params"]["Ly"] if k == "y" else 0.0)
                assert np.array_equal(fe[k][off:off + n], want), (e, k)
            assert np.array_equal(me[e * nc:(e + 1) * nc], m.moments()), e
            assert np.array_equal(qe[:, e * nc:(e + 1) * nc], m.coupling()["q"]), e
            off += n


def test_ensemble_matches_oracle(orc, ms):
    """FP64 ensemble against one oracle model per realization, 250 steps."""
    scens = realizations()
    ens = I.stack_ensemble(scens)
    g = ms.Model(ens["params"], ens["floes"], ms.MS_FP64)
    g.step(ens["dt"], 250)
    me = g.moments()
    nc = scens[0]["params"]["nx"] * scens[0]["params"]["ny"]
    for e, sc in enumerate(scens):
        o = orc.Model(sc["params"], sc["floes"])
        o.step(sc["dt"], 250)
        err = rel_errors(me[e * nc:(e + 1) * nc], o.moments(), sc["params"], 1e-12)
        assert err.max() <= 1e-10, report(err)


def test_ensemble_has_no_truth(ms):
    ens = I.stack_ensemble(realizations(R=2))
    g = ms.Model(ens["params"], ens["floes"], ms.MS_FP32)
    with pytest.raises(ms.MsError) as e:
        g.truth_step(ens["dt"], 1)
    assert e.value.code == -5
    with pytest.raises(ms.MsError):
        g.time_kernel(1, ens["dt"], 1)
    assert g.time_kernel(2, ens["dt"], 1) > 0


@pytest.mark.parametrize("variant", [2, 3])
def test_small_cell_ensemble_runs(ms, orc, variant):
    """Few floes per cell (the ensemble workload's law, 1 to 64; cells of up to 32 floes
    run packed several to a warp): 4 realizations of 16 x 16 cells through
    two coarse steps, one launch per step (variant 2) or per interval
    (variant 3), each realization's moments within the FP32 tolerance of its
    oracle model."""
    ens = I.ensemble_16x256x256(nreal=4, nx=16)
    p = ens["params"]
    g = ms.Model(p, ens["floes"], ms.MS_FP32)
    g.set_launch(variant, 128, 0, 1.3)
    g.step(ens["dt"], 200)
    me = g.moments()
    nc = p["nx"] * p["ny"]
    Ly = p["Ly"]
    for e in range(4):
        sel = (ens["floes"]["y"] >= e * Ly) & (ens["floes"]["y"] < (e + 1) * Ly)
        fl = {k: (v[sel] - (e * Ly if k == "y" else 0.0)) for k, v in ens["floes"].items()}
        o = orc.Model(dict(p, nens=1), fl)
        o.step(ens["dt"], 200)
        err = rel_errors(me[e * nc:(e + 1) * nc], o.moments(), p, 1e-6)
        assert err.max() <= 1e-4, report(err)
