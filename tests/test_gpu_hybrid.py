"""Closure plus particle fallback (the learned part of the method): training
data from the particle path, the trained network against held-out particle
data, and the coupled model with the closure against the particle-only model.

Workload: the batched workload's laws on 16 x 16 cells of 25 km (~31k floes), spun up
for 10 coarse intervals (the first gradual updates rescale radii by tens of
percent where neighbouring cells differ, and the contacts that follow need
several intervals to settle)."""
import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SPIN = 10


@pytest.fixture(scope="module")
def trained():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    Xs, Ys = [], []
    for sd in (201, 202, 203):
        s = I.batched_128x128(seed=sd, nx=16)
        m = msdem.Model(s["params"], s["floes"], 0)
        m.step(s["dt"], s["params"]["N0"] * SPIN)
        X, Y = m.closure_collect(30)
        Xs.append(X.reshape(-1, 16))
        Ys.append(Y.reshape(-1, 4))
        m.close()
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    norm = msdem.fit_norm(X, Y)
    net = msdem.MLP(I.mlp_init(), norm, max_batch=8192)
    losses = net.train(X, Y, epochs=120, batch=512, lr=2e-3, seed=11)
    box = np.stack([X.min(0) - 0.05 * np.abs(X.min(0)), X.max(0) + 0.05 * np.abs(X.max(0))])
    return msdem, net, X, Y, losses, box


def test_collect_targets_are_the_window_means(trained):
    """Targets 0-2 are the drag sums of the interval per unit mass/inertia, so
    for a cell without contacts they are the cell's mean drag acceleration:
    same sign convention as the velocity change it causes."""
    msdem, net, X, Y, losses, box = trained
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(Y))
    assert np.all(X[:, 0] > 0)                      # every cell holds ice
    assert np.all(X[:, 8] == 0)                     # a stream-function current has no divergence


def test_network_learns_translational_drag(trained):
    """Trained only on particle-generated data, the network predicts the
    interval-mean drag of unseen cells (another seed)."""
    msdem, net, X, Y, losses, box = trained
    assert losses[-1] < 0.5 * losses[0]
    s = I.batched_128x128(seed=204, nx=16)
    m = msdem.Model(s["params"], s["floes"], 0)
    m.step(s["dt"], s["params"]["N0"] * SPIN)
    Xh, Yh = m.closure_collect(10)
    Xh, Yh = Xh.reshape(-1, 16), Yh.reshape(-1, 4)
    P = net.predict(Xh)
    r2 = 1 - ((P - Yh) ** 2).sum(0) / ((Yh - Yh.mean(0)) ** 2).sum(0)
    assert r2[0] > 0.8 and r2[1] > 0.8, r2


def _run(msdem, s, mode, tol, net, box, K, variant=5):
    """Spin-up, then K coarse intervals with the closure attached (mode >= 0)
    or without; `variant` chooses the cell kernels (5, the default, or the
    warp-per-cell kernels of variant 4)."""
    p = s["params"]
    m = msdem.Model(p, s["floes"], 0)
    if variant != 5:
        m.set_launch(variant, 128, 0, 1.3)
    m.step(s["dt"], p["N0"] * SPIN)
    if mode >= 0:
        m.closure_attach(net if mode == 0 else None, mode, tol, box)
    m.step(s["dt"], p["N0"] * K)
    return m


@pytest.mark.parametrize("variant", [4, 5])
def test_zero_tolerance_is_the_particle_path(trained, variant):
    """With tol = 0 every cell fails the residual check and runs the particle
    step: the floes are bitwise those of the model without the closure."""
    msdem, net, X, Y, losses, box = trained
    s = I.batched_128x128(seed=205, nx=16)
    a = _run(msdem, s, -1, 0.0, net, box, 3, variant)
    b = _run(msdem, s, 0, 0.0, net, box, 3, variant)
    assert b.closure_stats()["closure_cell_intervals"] == 0
    fa, fb = a.floes(), b.floes()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_network_closure_beats_mean_field(trained):
    """What the trained network gains over the method without it: with every
    cell on a closure for the last 4 of 5 coarse intervals (the first after
    attaching runs the DEMs), the coarse momentum and angular momentum stay
    closer to the particle-only model with the network than with the
    mean-field drag of the cell-mean velocity and spin; mass stays within
    1e-3."""
    msdem, net, X, Y, losses, box = trained
    s = I.batched_128x128(seed=206, nx=16)
    K = 5
    qp = _run(msdem, s, -1, 0.0, net, box, K).coupling()["q"]
    qn = _run(msdem, s, 0, 1e9, net, None, K).coupling()["q"]
    qm = _run(msdem, s, 1, 0.0, None, None, K).coupling()["q"]
    err = lambda q: np.array([np.linalg.norm(q[f] - qp[f]) / np.linalg.norm(qp[f]) for f in range(4)])
    en, em = err(qn), err(qm)
    assert en[0] < 1e-3 and em[0] < 1e-3, (en, em)
    assert en[1] < em[1] and en[2] < em[2] and en[3] < em[3], (en, em)


def test_fallback_fraction_follows_tolerance(trained):
    msdem, net, X, Y, losses, box = trained
    s = I.batched_128x128(seed=207, nx=16)
    fr = []
    for tol in (0.02, 0.2, 1e9):
        # the first interval after attaching runs every DEM (the network needs
        # the tendencies of the interval before): count the two after it
        m = _run(msdem, s, 0, tol, net, box, 3)
        st = m.closure_stats()
        fr.append(st["closure_cell_intervals"] / (2 * st["cells"]))
    assert fr[0] <= fr[1] <= fr[2] and fr[2] > 0.5, fr


def test_closure_cells_skip_their_dem(trained):
    """One coarse interval with a mix of closure and particle cells (the
    resident kernels, variant 5): a closure cell's floes do not move (its
    DEM is skipped; the closure changed their velocities only), and every
    particle cell's floes are bitwise those of the particle-only model --
    cells sharing a block with skipped cells step exactly as before."""
    msdem, net, X, Y, losses, box = trained
    s = I.batched_128x128(seed=208, nx=16)
    p, dt, N0 = s["params"], s["dt"], s["params"]["N0"]
    a = _run(msdem, s, -1, 0.0, net, box, 2)
    b = _run(msdem, s, 0, 0.2, net, box, 1)
    assert b.closure_stats()["closure_cell_intervals"] == 0   # the first interval runs every DEM
    f1 = b.floes()
    b.step(dt, N0)
    f2, fa = b.floes(), a.floes()
    cells = msdem.floe_cells(p, s["floes"])
    still = (f1["x"] == f2["x"]) & (f1["y"] == f2["y"])
    ncell = p["nx"] * p["ny"]
    closure = np.zeros(ncell, bool)
    for c in range(ncell):
        sel = cells == c
        if sel.any() and still[sel].all():
            closure[c] = True
    nclos = b.closure_stats()["closure_cell_intervals"]
    assert 0 < nclos < ncell, nclos
    assert closure.sum() == nclos
    part = ~closure[cells]
    for k in fa:
        assert np.array_equal(f2[k][part], fa[k][part]), k
    a.close()
    b.close()


def test_ensemble_with_switching_closure_against_oracle(trained, orc):
    """Ensemble plus closure: two realizations of 32 x 32 cells (the batched
    workload's laws, about 98k floes each) in one model, the network
    attached after two coarse intervals, three more intervals in which cells
    switch between the closure and the particle path.  Each realization's
    coarse state against the FP64 oracle run of that realization alone
    (particle path only): mass within 1e-3, momentum and angular momentum
    within the closure's error scale; the same ensemble without the closure
    is within the FP32 tolerance."""
    msdem, net, X, Y, losses, box = trained
    scens = [I.batched_128x128(seed=301 + e, nx=32) for e in range(2)]
    for sc in scens[1:]:
        sc["params"]["modes"] = scens[0]["params"]["modes"]
    ens = I.stack_ensemble(scens)
    dt, N0 = ens["dt"], ens["params"]["N0"]
    nc = 32 * 32
    qs = {}
    for tol in (0.0, 0.1):
        g = msdem.Model(ens["params"], ens["floes"], 0)
        g.step(dt, 2 * N0)
        g.closure_attach(net, 0, tol, box)
        g.step(dt, 3 * N0)
        st = g.closure_stats()
        qs[tol] = (g.coupling()["q"], st["closure_cell_intervals"] / (2 * nc * 3))
        g.close()
    assert qs[0.0][1] == 0.0
    assert 0.0 < qs[0.1][1] < 1.0, qs[0.1][1]
    for e, sc in enumerate(scens):
        o = orc.Model(sc["params"], sc["floes"])
        o.step(dt, 5 * N0)
        qo = o.coupling()["q"]
        o.close()
        for tol, bounds in ((0.0, (1e-5, 1e-2, 1e-2, 1e-2)), (0.1, (1e-3, 0.15, 0.15, 0.3))):
            q = qs[tol][0][:, e * nc:(e + 1) * nc]
            err = [np.linalg.norm(q[f] - qo[f]) / np.linalg.norm(qo[f]) for f in range(4)]
            assert all(a <= b for a, b in zip(err, bounds)), (e, tol, err)
