"""The closure network's BF16 tensor-core forward, backward and Adam kernels
against the FP64 oracle (oracle/closure_oracle.py).  Training runs on either
engine: the tcgen05 GEMMs (engine 1, the default) or the mma.sync tiles
(engine 0); the training tests run on both."""
import numpy as np
import pytest

from oracle import closure_oracle as CO
from paper_2303_07819_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


def _data(seed, B):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, 16)) * np.linspace(0.5, 3.0, 16) + np.arange(16)
    Y = np.stack([np.sin(X[:, 0]), X[:, 1] * 0.1, np.tanh(X[:, 3] - 3), 0.01 * X[:, 4] ** 2], 1)
    Y = Y * np.array([1e-3, 2e-3, 1e-6, 5e-5])
    return X, Y


def _params(seed=5):
    rng = np.random.default_rng(seed)
    p = I.mlp_init(seed=seed)
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    return p


def test_fit_norm_matches_oracle(ms):
    """The library's own normalisation (device FP64 sums over FP32 inputs)
    against the oracle's NumPy mean and population sd of the same FP32
    values: equal to FP32 rounding; a constant column takes the floor."""
    X, Y = _data(4, 100003)
    X = X.astype(np.float32)
    Y = Y.astype(np.float32)
    X[:, 8] = 0.0                                   # a column without spread
    got = ms.fit_norm(X, Y)
    ref = CO.normalisation(X.astype(np.float64), Y.astype(np.float64))
    for k in ("mu_x", "mu_y"):
        sd = ref["sd_x" if k == "mu_x" else "sd_y"]
        assert np.all(np.abs(got[k] - ref[k]) <= 1e-6 * (np.abs(ref[k]) + sd)), k
    for k in ("sd_x", "sd_y"):
        assert np.all(np.abs(got[k] - ref[k]) <= 1e-6 * ref[k]), k
    assert got["sd_x"][8] == np.float32(1e-12)


def test_forward_matches_oracle(ms):
    X, Y = _data(0, 301)
    norm = CO.normalisation(X, Y)
    p = _params()
    net = ms.MLP(p, norm, max_batch=128)          # 3 batches, the last ragged
    got = net.predict(X)
    ref = CO.predict(p, X, norm)
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref - ref.mean(0), axis=0)
    assert err.max() < 2e-2, err
    # sample by sample, in the network's own (z-scored) output units: BF16
    # operands carry 8 significant bits through four layers
    ez = np.abs(got - ref) / norm["sd_y"]
    assert ez.max() < 0.1, ez.max(0)
    assert np.quantile(ez, 0.99) < 0.04, np.quantile(ez, 0.99, axis=0)


@pytest.mark.parametrize("n", [1, 127, 128, 301, 40000])
def test_tcgen05_forward_matches_oracle_and_mma(ms, n):
    """The tcgen05 inference kernel (the default engine) against the FP64
    oracle with the bounds of the tiled engine, and against the tiled
    engine itself: both round activations to BF16 between layers, so they
    differ only where an FP32 accumulation order flips a BF16 rounding.
    Sizes: one cell, a tile less one, one tile, a ragged tail, many tiles
    per CTA."""
    X, Y = _data(1, n)
    norm = CO.normalisation(_data(0, 301)[0], _data(0, 301)[1])
    p = _params()
    net = ms.MLP(p, norm, max_batch=65536)
    got = net.predict(X)
    net.set_engine(0)
    mma = net.predict(X)
    net.set_engine(1)
    ref = CO.predict(p, X, norm)
    ez = np.abs(got - ref) / norm["sd_y"]
    assert ez.max() < 0.1, ez.max(0)
    if n >= 128:
        assert np.quantile(ez, 0.99) < 0.04, np.quantile(ez, 0.99, axis=0)
    em = np.abs(got - mma) / norm["sd_y"]
    assert np.median(em) < 1e-3 and em.max() < 0.05, (np.median(em), em.max())
    net.close()


def test_engine_choice_is_checked(ms):
    X, Y = _data(0, 64)
    net = ms.MLP(_params(), CO.normalisation(X, Y), max_batch=64)
    with pytest.raises(ms.MsError):
        net.set_engine(2)
    net.close()


ENGINES = pytest.mark.parametrize("engine", [1, 0], ids=["tcgen05", "mma"])


@ENGINES
@pytest.mark.parametrize("B", [8, 64, 1000, 5000])
def test_gradients_match_oracle(ms, B, engine):
    """BF16 products with FP32 accumulation: each parameter's gradient within
    2e-2 of the FP64 gradient (normwise).  Batches below one 128-row tile,
    several tiles with a ragged tail, and split over k (5000 samples: 32
    slices of the weight-gradient products, added atomically)."""
    X, Y = _data(1, B)
    norm = CO.normalisation(X, Y)
    p = _params()
    net = ms.MLP(p, norm, max_batch=8192)
    net.set_engine(engine)
    loss, g = net.grad(X, Y)
    lref, gref = CO.loss_and_grads(p, X, Y, norm)
    assert abs(loss - lref) <= 2e-2 * lref
    for k in CO.NAMES:
        e = np.linalg.norm(g[k] - gref[k]) / np.linalg.norm(gref[k])
        assert e < 2e-2, (k, e)


def test_gradients_with_several_tiles_per_cta(ms):
    """40,000 samples are 313 tiles of 128, more than the SMs: the persistent
    tile kernel takes two or three tiles per CTA, and the weight-gradient
    kernel cuts the batch into 30 slices of 21 chunks of 64 samples.
    Within the oracle's 2e-2 and within 5e-3 of the mma.sync engine."""
    X, Y = _data(8, 40000)
    norm = CO.normalisation(X, Y)
    p = _params()
    net = ms.MLP(p, norm, max_batch=40000)
    l1, g1 = net.grad(X, Y)
    net.set_engine(0)
    l0, g0 = net.grad(X, Y)
    lref, gref = CO.loss_and_grads(p, X, Y, norm)
    assert abs(l1 - lref) <= 2e-2 * lref
    for k in CO.NAMES:
        e = np.linalg.norm(g1[k] - gref[k]) / np.linalg.norm(gref[k])
        assert e < 2e-2, (k, e)
        e = np.linalg.norm(g1[k] - g0[k]) / np.linalg.norm(g0[k])
        assert e < 5e-3, (k, e)
    net.close()


def test_gradients_of_the_two_engines_agree(ms):
    """Both engines round the same FP32 accumulations to BF16 between
    layers; they differ where the order of the FP32 sums flips a rounding:
    each gradient within 5e-3 of the other normwise."""
    X, Y = _data(6, 3001)
    norm = CO.normalisation(X, Y)
    net = ms.MLP(_params(), norm, max_batch=4096)
    l1, g1 = net.grad(X, Y)
    net.set_engine(0)
    l0, g0 = net.grad(X, Y)
    assert abs(l1 - l0) <= 1e-3 * l0
    for k in CO.NAMES:
        e = np.linalg.norm(g1[k] - g0[k]) / np.linalg.norm(g0[k])
        assert e < 5e-3, (k, e)
    net.close()


@ENGINES
def test_adam_first_step(ms, engine):
    """The first Adam step moves each parameter by lr * g / (|g| + eps): the
    same as the oracle's wherever the two gradients agree in sign."""
    X, Y = _data(2, 512)
    norm = CO.normalisation(X, Y)
    p = _params()
    net = ms.MLP(p, norm)
    net.set_engine(engine)
    _, gref = CO.loss_and_grads(p, X, Y, norm)
    net.step(X, Y, 1e-3)
    q = net.params()
    pr = {k: v.copy() for k, v in p.items()}
    CO.adam_step(pr, gref, {}, lr=1e-3)
    for k in CO.NAMES:
        big = np.abs(gref[k]) > 1e-2 * np.abs(gref[k]).max()
        d = np.abs(q[k] - pr[k])[big]
        assert np.mean(d < 1e-6) > 0.97, (k, np.mean(d < 1e-6))


@ENGINES
def test_training_on_gpu_reduces_loss(ms, engine):
    X, Y = _data(3, 20000)
    norm = CO.normalisation(X, Y)
    net = ms.MLP(I.mlp_init(), norm, max_batch=4096)
    net.set_engine(engine)
    losses = net.train(X, Y, epochs=25, batch=1024, lr=2e-3, seed=7)
    assert losses[-1] < 0.1 * losses[0], losses
    ref = CO.loss_and_grads(net.params(), X, Y, norm)[0]
    assert abs(ref - losses[-1]) < 0.5 * losses[-1] + 1e-3


@ENGINES
def test_every_epoch_visits_every_sample_once(ms, engine):
    """The device shuffle is a permutation: with a learning rate too small to
    move the weights, each epoch's mean loss is the loss of the whole set,
    to double rounding, although the set is gathered in a new order every
    epoch.  The samples' residuals span many magnitudes, so a sample seen
    twice or missed would move the mean far beyond that."""
    n = 8192
    X, Y = _data(9, n)
    norm = CO.normalisation(X, Y)
    Y = Y.copy()
    Y[:, 0] += norm["sd_y"][0] * np.geomspace(1e-3, 30.0, n)[np.random.default_rng(2).permutation(n)]
    net = ms.MLP(_params(), norm, max_batch=n)
    net.set_engine(engine)
    full = net.grad(X, Y)[0]
    losses = net.train(X, Y, epochs=3, batch=1024, lr=1e-30, seed=17)
    assert np.allclose(losses, full, rtol=1e-9, atol=0.0), (losses, full)
    net.close()
