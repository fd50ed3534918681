"""Tile sharding of the coarse grid (Sec. 3.1's processor grid), on CPU.

The partition and the exchange layout of paper_2303_07819_gb300.shard, and a
sharded run with gloo ranks (world sizes 2 and 3): each rank steps the
oracle's DEM of its own tile's cells only, the ranks all-gather the coarse
inputs through shard.gather at every coarse step, and every rank's floes,
moments and coarse state equal the unsharded oracle run bit for bit.  A run
whose ranks skip the exchange differs, so the comparison sees the
exchanged values."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2303_07819_gb300 import shard  # noqa: E402


def _cover(tiles, nx, ny):
    hit = np.zeros((ny, nx), dtype=int)
    for i0, i1, j0, j1 in tiles:
        assert 0 <= i0 < i1 <= nx and 0 <= j0 < j1 <= ny
        hit[j0:j1, i0:i1] += 1
    return hit


@pytest.mark.parametrize("nranks", [1, 2, 3, 4, 5, 7, 8, 16])
def test_partition_covers_once_and_balances(nranks):
    rng = np.random.default_rng(3)
    counts = np.clip(np.rint(96 * np.exp(0.69 * rng.standard_normal((64, 64)))), 8, 1024)
    w = 0.5 * counts * (counts - 1) + counts
    tiles = shard.partition(w, nranks)
    assert len(tiles) == nranks
    assert (_cover(tiles, 64, 64) == 1).all()
    loads = np.array([w[j0:j1, i0:i1].sum() for i0, i1, j0, j1 in tiles])
    # bisection on whole rows and columns: a cut moves a whole strip of a
    # tile (1/16 of a 16-wide tile's weight), so within 10 % of the mean
    assert loads.max() / loads.mean() < 1.10


def test_partition_follows_the_weight():
    """All the weight in the left quarter: the cut of two ranks falls inside
    it (balance by pair work, not by cell count)."""
    w = np.ones((16, 16))
    w[:, :4] = 1000.0
    (a, b) = shard.partition(w, 2)
    assert a[1] <= 4 and b[0] == a[1]


def test_partition_degenerate_grids():
    assert _cover(shard.partition(np.ones((1, 7)), 7), 7, 1).min() == 1
    assert _cover(shard.partition(np.ones((7, 1)), 7), 1, 7).min() == 1
    t = shard.partition(np.zeros((3, 5)), 4)           # no weight anywhere: split by cells
    assert (_cover(t, 5, 3) == 1).all()
    assert _cover(shard.partition(np.ones((3, 3)), 9), 3, 3).min() == 1
    with pytest.raises(ValueError):
        shard.partition(np.ones((2, 2)), 5)
    with pytest.raises(ValueError):
        shard.partition(np.ones((2, 2)), 0)


def test_partition_random_shapes():
    """Any grid and any rank count up to one rank per cell: the tiles are
    rectangles of at least one cell that cover the grid once."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        ny, nx = (int(v) for v in rng.integers(1, 13, 2))
        p = int(rng.integers(1, nx * ny + 1))
        w = rng.integers(0, 5, (ny, nx)).astype(float) ** 3
        t = shard.partition(w, p)
        assert len(t) == p
        assert (_cover(t, nx, ny) == 1).all()


def test_layout_rows_pack_unpack():
    rng = np.random.default_rng(5)
    counts = rng.integers(0, 50, size=(9, 11))
    lay = shard.layout(counts, 4)
    nc = 99
    assert sorted(lay.cells.tolist()) == list(range(nc))
    assert lay.rank_off[0] == 0 and lay.rank_off[-1] == nc
    for r in range(4):
        own = lay.own(r)
        assert (lay.owner[own] == r).all()
        i0, i1, j0, j1 = lay.tiles[r]
        assert own.size == (i1 - i0) * (j1 - j0)
        # row-major within the tile
        assert (np.diff(own) > 0).all()
    vals = rng.standard_normal((nc, shard.NCOL))
    gathered = np.concatenate([shard.pack(vals, lay, r) for r in range(4)])
    assert gathered.shape == (4 * lay.max_cells, shard.NCOL)
    cells, rows = shard.unpack(gathered, lay)
    assert np.array_equal(rows, vals[cells])
    # padding rows are zero and never read
    rows_used = set(lay.rows().tolist())
    pad = [k for k in range(gathered.shape[0]) if k not in rows_used]
    assert not np.any(gathered[pad])


# ----------------------------------------------------------- gloo ranks

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scenario(name):
    from paper_2303_07819_gb300 import inputs as I
    if name == "square":
        return I.square_4x4()
    return I.powerlaw_32x32(nx=8)


def _oracle_cells(O, s):
    """The oracle's cell of every floe (its own assignment rule)."""
    m = O.Model(s["params"], s["floes"])
    off, orig = m.layout()
    m.close()
    cell = np.empty(orig.shape[0], dtype=np.int64)
    for c in range(off.shape[0] - 1):
        cell[orig[off[c]:off[c + 1]]] = c
    return cell, np.diff(off)


def _run_rank(O, s, lay, rank, cell, nsteps, exchange):
    """Rank `rank`'s oracle run: the floes of its cells, held at every
    coarse step until the ranks have gathered each other's coarse inputs."""
    import torch.distributed as dist
    idx = np.flatnonzero(lay.owner[cell] == rank)
    own = {k: np.asarray(v)[idx] for k, v in s["floes"].items()}
    m = O.Model(s["params"], own)
    m.set_hold(True)
    dt = s["dt"]
    nexch = 0
    while True:
        if m.coarse_pending():
            vals = m.coarse_inputs()
            if exchange:
                send = torch.from_numpy(shard.pack(vals, lay, rank))
                cells, rows = shard.unpack(shard.gather(send, lay).numpy(), lay)
                m.set_coarse_inputs(cells, rows)
            else:
                dist.barrier()
            nexch += 1
            m.coarse()
            continue
        done = m.coupling()["steps"]
        if done >= nsteps:
            break
        m.step(dt, nsteps - done)
    out = {"idx": idx, "mom": m.moments(), "q": m.coupling()["q"], "tg": m.coupling()["targets"],
           "nexch": nexch}
    out.update({"f_" + k: v for k, v in m.floes().items()})
    m.close()
    return out


def _worker(rank, world, port, name, nsteps, exchange, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    O.set_threads(2)
    s = _scenario(name)
    cell, counts = _oracle_cells(O, s)
    p = s["params"]
    lay = shard.layout(counts.reshape(p["ny"], p["nx"]), world)
    res = _run_rank(O, s, lay, rank, cell, nsteps, exchange)
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), own=lay.own(rank), **res)
    dist.barrier()
    dist.destroy_process_group()


def _spawn(world, name, nsteps, exchange, outdir):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, nsteps, exchange, str(outdir)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    for p in procs:
        if p.exitcode is None:
            p.kill()
        assert p.exitcode == 0
    return [dict(np.load(os.path.join(outdir, f"rank{r}.npz"))) for r in range(world)]


def _unsharded(orc, name, nsteps):
    s = _scenario(name)
    m = orc.Model(s["params"], s["floes"])
    m.step(s["dt"], nsteps)
    out = {"mom": m.moments(), "q": m.coupling()["q"], "tg": m.coupling()["targets"], "floes": m.floes()}
    m.close()
    return out


@pytest.mark.parametrize("world,name", [(2, "powerlaw8"), (3, "square")])
def test_sharded_oracle_equals_unsharded(orc, tmp_path, world, name):
    """Two coarse steps (200 fine steps, N0 = 100) and the first gradual
    updates of a third interval: bitwise equal floes (each rank's own),
    moments (own cells) and the coarse state and targets (every cell, on
    every rank)."""
    nsteps = 250
    ref = _unsharded(orc, name, nsteps)
    ranks = _spawn(world, name, nsteps, True, tmp_path)
    seen = np.zeros(ref["mom"].shape[0], dtype=int)
    for r in ranks:
        assert r["nexch"] == 2
        own = r["own"]
        seen[own] += 1
        assert np.array_equal(r["mom"][own], ref["mom"][own])
        assert np.array_equal(r["q"], ref["q"])
        assert np.array_equal(r["tg"], ref["tg"])
        for k, v in ref["floes"].items():
            assert np.array_equal(r["f_" + k], v[r["idx"]]), k
    assert (seen == 1).all()
    assert sum(r["idx"].size for r in ranks) == ref["floes"]["x"].size


def test_sharded_oracle_without_exchange_differs(orc, tmp_path):
    """The same ranks with the all-gather left out (each rank's coarse step
    sees only its own cells): the coarse state departs from the unsharded
    one, so the equality above rests on the exchanged values."""
    nsteps = 150
    ref = _unsharded(orc, "powerlaw8", nsteps)
    ranks = _spawn(2, "powerlaw8", nsteps, False, tmp_path)
    assert any(not np.array_equal(r["q"], ref["q"]) for r in ranks)
