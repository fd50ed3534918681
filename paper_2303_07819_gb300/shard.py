"""Tile sharding of the msDEM coarse grid over ranks (Sec. 3.1's processor
grid of cell blocks; Sec. 4.1's parallel runs).

Between coarse steps every cell's DEM is independent of every other cell's
(Algorithm 1: the particle steps of an interval touch only the cell's own
floes), so a rank steps the floes of a contiguous 2-D tile of cells and the
ranks meet once per coarse interval.  The coarse step needs, for each cell,
its moment columns 1-5 (mass, momentum, moment of inertia, angular momentum)
and its five window sums; every rank gathers those ten FP64 values of all
cells and takes the whole coarse step itself.  The coarse step is then the
same computation on the same inputs on every rank, so a sharded run gives
the unsharded run's floes and moments bit for bit.  An all-gather of the
whole grid (128 x 128 cells: 1.3 MB) instead of a one-cell halo keeps the
coarse step identical to the unsharded one and costs one collective.

This module holds the host side: the partition (recursive bisection into
rectangular tiles balanced by a per-cell weight, the number of floe pairs by
default), the exchange layout, and the all-gather through
``torch.distributed`` (NCCL for CUDA tensors, gloo for CPU tensors).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

NCOL = 10   # coarse inputs per cell: moment columns 1-5, window sums 0-4


def _split(weights: np.ndarray, parts_lo: int, parts: int) -> int:
    """Index k (1 <= k < len) splitting a 1-D weight profile so that the
    first k entries carry about parts_lo / parts of the total."""
    n = len(weights)
    if n < 2:
        return 1
    cum = np.cumsum(weights, dtype=np.float64)
    if cum[-1] <= 0.0:
        k = int(round(n * parts_lo / parts))
    else:
        # first k entries sum to cum[k - 1]; the k closest to the goal
        k = 1 + int(np.argmin(np.abs(cum[:-1] - cum[-1] * parts_lo / parts)))
    return min(max(k, 1), n - 1)


def partition(weight: np.ndarray, nranks: int) -> list[tuple[int, int, int, int]]:
    """Rectangular tiles (i0, i1, j0, j1), half-open in x (columns) and y
    (rows), one per rank, covering a grid whose per-cell weights are
    `weight[j, i]`.  Recursive bisection: the longer side of a tile is cut
    where the weight splits in the ratio of the ranks sent to each side.
    A tile is never empty of cells while the grid has at least nranks
    cells."""
    weight = np.asarray(weight, dtype=np.float64)
    ny, nx = weight.shape
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if nranks > nx * ny:
        raise ValueError(f"{nranks} ranks for {nx * ny} cells")
    out: list[tuple[int, int, int, int]] = []

    def cut(i0, i1, j0, j1, p):
        if p == 1:
            out.append((i0, i1, j0, j1))
            return
        w = weight[j0:j1, i0:i1]
        # cut across the longer side; a side of one cell cannot be cut
        along_x = (i1 - i0) >= (j1 - j0) if (i1 - i0) > 1 and (j1 - j0) > 1 else (i1 - i0) > 1
        prof = w.sum(axis=0) if along_x else w.sum(axis=1)
        n, strip = len(prof), (j1 - j0) if along_x else (i1 - i0)   # strips and cells per strip
        plo = p // 2
        k = _split(prof, plo, p)
        # every rank needs a cell: if this cut leaves a side too few cells
        # for its ranks, send it fewer ranks and cut again for those
        plo = min(max(plo, p - (n - k) * strip, 1), k * strip, p - 1)
        k = _split(prof, plo, p)
        k = min(max(k, -(-plo // strip)), n - (-(-(p - plo) // strip)))
        if along_x:
            cut(i0, i0 + k, j0, j1, plo)
            cut(i0 + k, i1, j0, j1, p - plo)
        else:
            cut(i0, i1, j0, j0 + k, plo)
            cut(i0, i1, j0 + k, j1, p - plo)

    cut(0, nx, 0, ny, nranks)
    return out


@dataclass
class Layout:
    """Exchange layout: rank r owns cells[rank_off[r]:rank_off[r+1]] (row-major
    within its tile); its rows of the gathered buffer are r * max_cells + k."""
    nx: int
    ny: int
    tiles: list
    rank_off: np.ndarray   # int32 [nranks + 1]
    cells: np.ndarray      # int32 [ncell], a permutation of the cells
    owner: np.ndarray      # int32 [ncell], the rank of each cell

    @property
    def nranks(self) -> int:
        return len(self.tiles)

    @property
    def max_cells(self) -> int:
        return int(np.diff(self.rank_off).max())

    def own(self, rank: int) -> np.ndarray:
        return self.cells[self.rank_off[rank]:self.rank_off[rank + 1]]

    def rows(self) -> np.ndarray:
        """Row of the gathered buffer holding each entry of `cells`."""
        r = np.repeat(np.arange(self.nranks), np.diff(self.rank_off))
        return (r * self.max_cells + (np.arange(len(self.cells)) - self.rank_off[r])).astype(np.int64)


def layout(counts: np.ndarray, nranks: int, weight: np.ndarray | None = None) -> Layout:
    """Layout of a grid of `counts[j, i]` floes per cell over nranks ranks,
    tiles balanced by `weight` (default: floe pairs, n (n - 1) / 2, plus n,
    so that cells of one floe still count)."""
    counts = np.asarray(counts)
    ny, nx = counts.shape
    if weight is None:
        c = counts.astype(np.float64)
        weight = 0.5 * c * (c - 1.0) + c
    tiles = partition(weight, nranks)
    owner = np.empty((ny, nx), dtype=np.int32)
    cells, off = [], [0]
    for r, (i0, i1, j0, j1) in enumerate(tiles):
        owner[j0:j1, i0:i1] = r
        jj, ii = np.meshgrid(np.arange(j0, j1), np.arange(i0, i1), indexing="ij")
        cells.append((jj * nx + ii).ravel())
        off.append(off[-1] + cells[-1].size)
    return Layout(nx, ny, tiles, np.asarray(off, dtype=np.int32),
                  np.concatenate(cells).astype(np.int32), owner.ravel())


def gather(send, lay: Layout, group=None, out=None):
    """All-gather the ranks' [max_cells][NCOL] coarse inputs into one
    [nranks * max_cells][NCOL] tensor (torch.distributed; the group's
    backend decides the transport).  `send` is a torch tensor; its padding
    rows are carried along and never read."""
    import torch
    import torch.distributed as dist
    if out is None:
        out = torch.empty((lay.nranks * lay.max_cells, NCOL), dtype=send.dtype, device=send.device)
    dist.all_gather_into_tensor(out, send.contiguous(), group=group)
    return out


def pack(values: np.ndarray, lay: Layout, rank: int) -> np.ndarray:
    """A rank's send rows from its [ncell][NCOL] coarse inputs (padding rows
    zero)."""
    own = lay.own(rank)
    out = np.zeros((lay.max_cells, NCOL))
    out[: own.size] = values[own]
    return out


def unpack(gathered: np.ndarray, lay: Layout) -> tuple[np.ndarray, np.ndarray]:
    """(cells, [ncell][NCOL] values in the order of `cells`) from the
    gathered buffer."""
    return lay.cells, np.asarray(gathered)[lay.rows()]


class ShardedModel:
    """This rank's part of a sharded msDEM model: the floes of its tile's
    cells in a model on the current CUDA device (ms_set_shard), the coarse
    inputs exchanged once per coarse interval through torch.distributed.
    With NCCL the all-gather is enqueued on the model's stream (no host
    synchronization); with another backend it goes through host memory.

    floes: the whole grid's floes (every rank passes the same); `index` holds
    the indices of those this rank steps, ascending, which keeps each cell's
    floes in their order of the unsharded model."""

    def __init__(self, params: dict, floes: dict, nranks: int, rank: int, group=None, precision=None,
                 lay: Layout | None = None, cells_of: np.ndarray | None = None):
        import torch
        import torch.distributed as dist
        from . import msdem
        if precision is None:
            precision = msdem.MS_FP32
        nx, ny = int(params["nx"]), int(params["ny"]) * max(1, int(params.get("nens", 1)))
        if cells_of is None:
            cells_of = msdem.floe_cells(params, floes)
        counts = np.bincount(cells_of, minlength=nx * ny).reshape(ny, nx)
        self.layout = lay if lay is not None else layout(counts, nranks)
        if self.layout.nranks != nranks:
            raise ValueError("layout has %d ranks, not %d" % (self.layout.nranks, nranks))
        self.rank, self.nranks, self.group = rank, nranks, group
        self.index = np.flatnonzero(self.layout.owner[cells_of] == rank)
        own = {k: np.asarray(floes[k], dtype=np.float64)[self.index] for k in msdem.FLOE_KEYS}
        self.model = msdem.Model(params, own, precision)
        self.model.set_shard(nranks, rank, self.layout.rank_off, self.layout.cells, self._exchange)
        send, recv, _ = self.model.shard_buffers()
        self._send = torch.as_tensor(send, device="cuda")
        self._recv = torch.as_tensor(recv, device="cuda")
        self._nccl = nranks > 1 and dist.get_backend(group) == "nccl"
        self.exchanges = 0

    def _exchange(self, stream: int) -> None:
        import torch
        import torch.distributed as dist
        ext = torch.cuda.ExternalStream(stream)
        if self.nranks == 1:
            with torch.cuda.stream(ext):
                self._recv.copy_(self._send)
        elif self._nccl:
            with torch.cuda.stream(ext):
                gather(self._send, self.layout, self.group, out=self._recv)
        else:
            ext.synchronize()
            out = gather(self._send.cpu(), self.layout, self.group)
            with torch.cuda.stream(ext):
                self._recv.copy_(out)
        self.exchanges += 1

    def step(self, dt: float, nsteps: int) -> None:
        self.model.step(dt, nsteps)

    def step_async(self, dt: float, nsteps: int) -> None:
        self.model.step_async(dt, nsteps)

    def sync(self) -> None:
        self.model.sync()

    def floes(self) -> dict:
        """This rank's floes, in the order of `index`."""
        return self.model.floes()

    def moments(self) -> np.ndarray:
        """[ncell][12]: the rows of this rank's cells (own_cells)."""
        return self.model.moments()

    def own_cells(self) -> np.ndarray:
        return self.layout.own(self.rank)

    def close(self) -> None:
        self.model.close()
