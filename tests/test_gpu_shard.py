"""Sharded grids on the GPU (ms_set_shard, Sec. 3.1's processor grid): a
grid split into tiles, one model per tile on this GPU, the coarse inputs
exchanged at every coarse step.

FP64 and FP32 shards give the unsharded model's floes, moments and coarse
state bit for bit.  The shards of a
test run in threads of one process (each thread steps its model; the
exchange meets at a barrier and copies on the models' streams) or in two
processes on this GPU that exchange through gloo on the host: in neither do
kernels of one shard wait on another's."""
import os
import socket
import threading

import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I
from paper_2303_07819_gb300 import shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ms():
    from paper_2303_07819_gb300 import msdem
    msdem.load()
    return msdem


class Shards:
    """nranks models of one grid in this process; step() runs each in its
    own thread and the exchange callbacks meet at a barrier."""

    def __init__(self, ms, scen, nranks, precision, lay=None):
        p, fl = scen["params"], scen["floes"]
        self.cells_of = ms.floe_cells(p, fl)
        nx, ny = int(p["nx"]), int(p["ny"]) * max(1, int(p.get("nens", 1)))
        counts = np.bincount(self.cells_of, minlength=nx * ny).reshape(ny, nx)
        self.lay = lay if lay is not None else shard.layout(counts, nranks)
        self.nranks = nranks
        self.bar = threading.Barrier(nranks, timeout=300)
        self.sent = [None] * nranks
        self.models, self.index, self.bufs = [], [], []
        self.exchanges = [0] * nranks
        for r in range(nranks):
            idx = np.flatnonzero(self.lay.owner[self.cells_of] == r)
            m = ms.Model(p, {k: np.asarray(v)[idx] for k, v in fl.items()}, precision)
            m.set_shard(nranks, r, self.lay.rank_off, self.lay.cells, self._exchange_of(r))
            snd, rcv, _ = m.shard_buffers()
            self.bufs.append((torch.as_tensor(snd, device="cuda"), torch.as_tensor(rcv, device="cuda")))
            self.models.append(m)
            self.index.append(idx)

    def _exchange_of(self, r):
        def ex(stream):
            st = torch.cuda.ExternalStream(stream)
            with torch.cuda.stream(st):
                self.sent[r] = self.bufs[r][0].clone()
            st.synchronize()
            self.bar.wait()
            with torch.cuda.stream(st):
                self.bufs[r][1].copy_(torch.cat(self.sent))
            st.synchronize()
            self.bar.wait()
            self.exchanges[r] += 1
        return ex

    def step(self, dt, nsteps, chunks=None):
        errs = []

        def run(m):
            try:
                for n in (chunks or [nsteps]):
                    m.step(dt, n)
            except BaseException as e:
                errs.append(e)
                self.bar.abort()

        th = [threading.Thread(target=run, args=(m,)) for m in self.models]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]

    def close(self):
        for m in self.models:
            m.close()


def _unsharded(ms, scen, precision, nsteps, chunks=None):
    m = ms.Model(scen["params"], scen["floes"], precision)
    for n in (chunks or [nsteps]):
        m.step(scen["dt"], n)
    out = {"floes": m.floes(), "mom": m.moments(), "c": m.coupling()}
    m.close()
    return out


def _check_bitwise(sh, ref):
    for r, m in enumerate(sh.models):
        own = sh.lay.own(r)
        f = m.floes()
        for k, v in ref["floes"].items():
            assert np.array_equal(f[k], v[sh.index[r]]), (r, k)
        assert np.array_equal(m.moments()[own], ref["mom"][own]), r
        c = m.coupling()
        for k in ("q", "targets"):
            assert np.array_equal(c[k], ref["c"][k]), (r, k)


@pytest.mark.parametrize("nranks", [2, 3])
def test_fp64_shards_equal_unsharded(ms, nranks):
    """Two coarse steps and part of a third interval, graph intervals and
    single steps mixed: bitwise equal on every rank."""
    scen = I.powerlaw_32x32(nx=8)
    chunks = [100, 37, 63, 50]
    ref = _unsharded(ms, scen, ms.MS_FP64, 250, chunks)
    sh = Shards(ms, scen, nranks, ms.MS_FP64)
    sh.step(scen["dt"], 250, chunks)
    assert sh.exchanges == [2] * nranks
    _check_bitwise(sh, ref)
    info = sh.models[0].info()
    assert info["shard_ranks"] == nranks and info["shard_rank"] == 0
    assert info["shard_cells"] == sh.lay.own(0).size
    sh.close()


def test_one_rank_is_the_unsharded_model(ms):
    """A one-rank shard (the exchange a plain copy): FP32 variant 5 bitwise
    equal to the unsharded model through coarse steps."""
    scen = I.powerlaw_32x32(nx=8)
    ref = _unsharded(ms, scen, ms.MS_FP32, 300)
    sh = shard.ShardedModel(scen["params"], scen["floes"], 1, 0)
    sh.step(scen["dt"], 300)
    assert sh.exchanges == 3
    f = sh.floes()
    for k, v in ref["floes"].items():
        assert np.array_equal(f[k], v), k
    assert np.array_equal(sh.moments(), ref["mom"])
    sh.close()


def test_fp32_shards_full_size(ms):
    """The batched 128 x 128 workload (about 2M floes) in four tiles, FP32
    variant 5, three coarse steps: floes, own cells' moments and the coarse
    state bitwise those of the unsharded model (a cell's floes run the code
    of its own size class, and its sums are exact integer sums whichever
    cells share its block)."""
    scen = I.batched_128x128()
    dt = scen["dt"]
    sh = Shards(ms, scen, 4, ms.MS_FP32)
    m0 = ms.Model(scen["params"], scen["floes"], ms.MS_FP32)
    m0.step(dt, 300)
    sh.step(dt, 300)
    ref = {"floes": m0.floes(), "mom": m0.moments(), "c": m0.coupling()}
    _check_bitwise(sh, ref)
    m0.close()
    sh.close()


def test_shard_errors(ms):
    scen = I.powerlaw_32x32(nx=4)
    p, fl = scen["params"], scen["floes"]
    nc = 16
    cells = np.arange(nc, dtype=np.int32)
    ok = lambda s: None  # noqa: E731
    m = ms.Model(p, fl, ms.MS_FP32)
    # the model holds floes of every cell: rank 0 of 2 may not own half
    with pytest.raises(ms.MsError, match="belongs to rank"):
        m.set_shard(2, 0, [0, 8, 16], cells, ok)
    with pytest.raises(ms.MsError, match="permutation"):
        m.set_shard(1, 0, [0, 16], np.r_[cells[:-1], 0], ok)
    with pytest.raises(ms.MsError, match="rank_off"):
        m.set_shard(1, 0, [0, 15], cells, ok)
    with pytest.raises(ms.MsError):
        m.set_shard(2, 2, [0, 8, 16], cells, ok)
    with pytest.raises(ms.MsError, match="not sharded"):
        m.shard_buffers()
    m.set_shard(1, 0, [0, 16], cells, ok)
    with pytest.raises(ms.MsError, match="already sharded"):
        m.set_shard(1, 0, [0, 16], cells, ok)
    mlp = ms.MLP(I.mlp_init(), {"mu_x": np.zeros(16), "sd_x": np.ones(16), "mu_y": np.zeros(4),
                                "sd_y": np.ones(4)})
    with pytest.raises(ms.MsError, match="no closure"):
        m.closure_attach(mlp, 0, 0.5)
    mlp.close()
    m.close()


def test_failed_exchange_stops_the_model(ms):
    scen = I.powerlaw_32x32(nx=4)
    m = ms.Model(scen["params"], scen["floes"], ms.MS_FP32)

    def bad(stream):
        raise RuntimeError("peer lost")

    m.set_shard(1, 0, [0, 16], np.arange(16, dtype=np.int32), bad)
    with pytest.raises(ms.MsError, match="exchange") as ei:
        m.step(scen["dt"], 100)
    assert isinstance(ei.value.__cause__, RuntimeError)
    with pytest.raises(ms.MsError) as e2:
        m.step(scen["dt"], 1)
    assert e2.value.code == -5
    m.close()


# ------------------------------------------- two processes, gloo on the host

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2303_07819_gb300 import msdem
    scen = I.powerlaw_32x32(nx=8)
    sh = shard.ShardedModel(scen["params"], scen["floes"], world, rank, precision=msdem.MS_FP64)
    sh.step(scen["dt"], 250)
    f = sh.floes()
    np.savez(os.path.join(outdir, f"r{rank}.npz"), idx=sh.index, own=sh.own_cells(), mom=sh.moments(),
             q=sh.model.coupling()["q"], nexch=sh.exchanges, **{"f_" + k: v for k, v in f.items()})
    sh.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_gloo(ms, tmp_path):
    """ShardedModel's host exchange (gloo) between two processes on this
    GPU: FP64 bitwise equal to the unsharded model."""
    import torch.multiprocessing as mp
    scen = I.powerlaw_32x32(nx=8)
    ref = _unsharded(ms, scen, ms.MS_FP64, 250)
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_proc, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
    for p in procs:
        if p.exitcode is None:
            p.kill()
        assert p.exitcode == 0
    for r in range(2):
        d = np.load(os.path.join(tmp_path, f"r{r}.npz"))
        assert int(d["nexch"]) == 2
        own = d["own"]
        assert np.array_equal(d["mom"][own], ref["mom"][own])
        assert np.array_equal(d["q"], ref["c"]["q"])
        for k, v in ref["floes"].items():
            assert np.array_equal(d["f_" + k], v[d["idx"]]), k
