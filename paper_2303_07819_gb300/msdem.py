"""Thin ctypes binding of libmsdem.so (the C-ABI of include/msdem.h).

Argument marshalling only: every step of the model runs in the library's CUDA
kernels.  Importing this module loads the library and raises if it is missing
or no CUDA device is usable; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NMOM = 12
NWIN = 5
MAX_MODES = 16
MS_FP32, MS_FP64 = 0, 1
ERRORS = {0: "MS_OK", -1: "MS_ERR_ARG", -2: "MS_ERR_CUDA", -3: "MS_ERR_UNSTABLE", -4: "MS_ERR_TIMEOUT",
          -5: "MS_ERR_STATE"}
MOMENT_NAMES = ["n", "M", "Mu", "Mv", "I", "Iw", "area", "Muu", "Mvv", "Fdx", "Fdy", "Td"]
FLOE_KEYS = ("x", "y", "theta", "u", "v", "omega", "r", "h")

_dp = C.POINTER(C.c_double)
_ip32 = C.POINTER(C.c_int32)
SHARD_NCOL = 10
# int exchange(void *ctx, void *stream)
EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("Lx", C.c_double), ("Ly", C.c_double),
                ("nens", C.c_int32), ("walls", C.c_int32)]


class Floes(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, _dp) for k in FLOE_KEYS]


class Forcing(C.Structure):
    _fields_ = [
        ("uo_x", C.c_double), ("uo_y", C.c_double), ("n_modes", C.c_int32), ("modes", _dp),
        ("rho_o", C.c_double), ("Cd", C.c_double), ("rho_a", C.c_double), ("Ca", C.c_double),
        ("wind_x", C.c_double), ("wind_y", C.c_double), ("wind_period", C.c_double),
        ("rho_ice", C.c_double), ("E", C.c_double), ("G", C.c_double), ("eta", C.c_double),
        ("mu", C.c_double), ("h_ref", C.c_double), ("inertia_half", C.c_int32),
        ("couple", C.c_int32), ("N0", C.c_int32), ("n_t", C.c_int32), ("precision", C.c_int32),
        ("n_vmodes", C.c_int32), ("vmodes", _dp),
    ]


class MsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None
SYMBOLS = ["ms_init", "ms_step", "ms_step_async", "ms_sync", "ms_moments", "ms_get_floes", "ms_set_floes", "ms_coupling",
           "ms_truth_step", "ms_truth_moments", "ms_truth_get_floes", "ms_set_stream", "ms_autotune",
           "ms_time_kernel", "ms_set_launch", "ms_info", "ms_free", "ms_last_error", "ms_cell_moments_noalloc",
           "ms_mlp_create", "ms_mlp_predict", "ms_mlp_grad", "ms_mlp_step", "ms_mlp_train", "ms_mlp_get_params",
           "ms_mlp_forward_device", "ms_mlp_free", "ms_closure_attach", "ms_closure_collect", "ms_closure_stats",
           "ms_probe_fp32", "ms_save", "ms_load", "ms_mlp_fit_norm", "ms_set_resident",
           "ms_floe_cells", "ms_set_shard", "ms_shard_buffers", "ms_layout", "ms_mlp_set_engine",
           "ms_mlp_check"]


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libmsdem.so (building it if the sources are newer).  Raises when
    the library cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if path is None and not _build.up_to_date():
        _build.build()
    if not os.path.exists(p):
        raise RuntimeError(f"libmsdem.so not found at {p}; run __graft_entry__.build()")
    L = C.CDLL(p)
    vp = C.c_void_p
    L.ms_init.argtypes = [C.POINTER(vp), C.POINTER(Grid), C.POINTER(Floes), C.POINTER(Forcing)]
    L.ms_step.argtypes = [vp, C.c_double, C.c_int64]
    L.ms_step_async.argtypes = [vp, C.c_double, C.c_int64]
    L.ms_sync.argtypes = [vp]
    L.ms_moments.argtypes = [vp, _dp]
    L.ms_get_floes.argtypes = [vp, _dp]
    L.ms_set_floes.argtypes = [vp, C.POINTER(Floes)]
    L.ms_coupling.argtypes = [vp, _dp, _dp, _dp, C.POINTER(C.c_int64)]
    L.ms_truth_step.argtypes = [vp, C.c_double, C.c_int64]
    L.ms_truth_moments.argtypes = [vp, _dp]
    L.ms_truth_get_floes.argtypes = [vp, _dp]
    L.ms_set_stream.argtypes = [vp, vp]
    L.ms_autotune.argtypes = [vp, C.c_double, C.c_int32, _dp]
    L.ms_time_kernel.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, _dp]
    L.ms_set_launch.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_double]
    L.ms_set_resident.argtypes = [vp, C.c_double, C.c_int32]
    L.ms_info.argtypes = [vp, C.POINTER(C.c_int64)]
    L.ms_cell_moments_noalloc.argtypes = [C.POINTER(Grid), C.c_double, C.c_int32, C.c_int64] + [vp] * 10
    L.ms_closure_attach.argtypes = [vp, vp, C.c_int32, C.c_double, C.POINTER(C.c_float)]
    L.ms_closure_collect.argtypes = [vp, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.ms_closure_stats.argtypes = [vp, C.POINTER(C.c_int64)]
    L.ms_probe_fp32.argtypes = [C.c_int32, _dp]
    L.ms_save.argtypes = [vp, C.c_char_p]
    L.ms_load.argtypes = [vp, C.c_char_p]
    L.ms_floe_cells.argtypes = [C.POINTER(Grid), C.POINTER(Floes), _ip32]
    L.ms_layout.argtypes = [vp, _ip32, _ip32]
    L.ms_set_shard.argtypes = [vp, C.c_int32, C.c_int32, _ip32, _ip32, EXCHANGE_FN, vp]
    L.ms_shard_buffers.argtypes = [vp, C.POINTER(_dp), C.POINTER(_dp), _ip32]
    L.ms_free.argtypes = [vp]
    L.ms_free.restype = None
    L.ms_last_error.restype = C.c_char_p
    for name in SYMBOLS:
        if name not in ("ms_free", "ms_last_error", "ms_mlp_free"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise MsError(rc, load().ms_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_floes(floes: dict):
    arrs = [np.ascontiguousarray(floes[k], dtype=np.float64) for k in FLOE_KEYS]
    s = Floes()
    s.n = arrs[0].shape[0]
    for k, a in zip(FLOE_KEYS, arrs):
        setattr(s, k, _ptr(a))
    return s, arrs


def make_forcing(p: dict, precision: int):
    modes = np.ascontiguousarray(np.asarray(p.get("modes", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4))
    vmodes = np.ascontiguousarray(np.asarray(p.get("vmodes", np.zeros((0, 5))), dtype=np.float64).reshape(-1, 5))
    f = Forcing()
    f.uo_x, f.uo_y = float(p.get("uo_x", 0.0)), float(p.get("uo_y", 0.0))
    f.n_modes = modes.shape[0]
    f.modes = _ptr(modes) if modes.shape[0] else _dp()
    for k in ("rho_o", "Cd", "rho_a", "Ca", "wind_x", "wind_y", "wind_period", "rho_ice", "E", "G", "eta",
              "mu", "h_ref"):
        setattr(f, k, float(p.get(k, 0.0)))
    f.inertia_half = int(p.get("inertia_half", 0))
    f.couple, f.N0, f.n_t = int(p.get("couple", 0)), int(p.get("N0", 100)), int(p.get("n_t", 10))
    f.precision = int(precision)
    f.n_vmodes = vmodes.shape[0]
    f.vmodes = _ptr(vmodes) if vmodes.shape[0] else _dp()
    return f, (modes, vmodes)


def make_grid(params: dict) -> Grid:
    nens = max(1, int(params.get("nens", 1)))
    return Grid(int(params["nx"]), int(params["ny"]), float(params["Lx"]), float(params["Ly"]), nens,
                int(params.get("walls", 0)))


def floe_cells(params: dict, floes: dict) -> np.ndarray:
    """The cell ms_init assigns each floe to (int32, j * nx + i)."""
    L = load()
    g = make_grid(params)
    fl, keep = make_floes(floes)
    out = np.zeros(max(int(fl.n), 1), dtype=np.int32)
    _check(L.ms_floe_cells(C.byref(g), C.byref(fl), out.ctypes.data_as(_ip32)))
    return out[: int(fl.n)]


class DeviceArray:
    """A view of device memory the library owns, for consumers of
    __cuda_array_interface__ (torch.as_tensor(..., device="cuda"))."""

    def __init__(self, ptr: int, shape: tuple, typestr: str = "<f8"):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None,
                                         "stream": None}


class Model:
    """One msDEM model (plus its truth DEM) on the current CUDA device."""

    def __init__(self, params: dict, floes: dict, precision: int = MS_FP32):
        L = load()
        self.params = dict(params)
        self.precision = precision
        nens = max(1, int(params.get("nens", 1)))
        g = make_grid(params)
        fl, keep1 = make_floes(floes)
        fc, keep2 = make_forcing(params, precision)
        h = C.c_void_p()
        _check(L.ms_init(C.byref(h), C.byref(g), C.byref(fl), C.byref(fc)))
        self._h = h
        self.n = int(fl.n)
        self.ncell = g.nx * g.ny * nens

    def close(self):
        if getattr(self, "_h", None):
            load().ms_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _step_check(self, rc: int) -> None:
        err = getattr(self, "_exch_error", None)
        if rc != 0 and err is not None:
            self._exch_error = None
            raise MsError(rc, load().ms_last_error().decode()) from err
        _check(rc)

    def step(self, dt: float, nsteps: int) -> None:
        self._step_check(load().ms_step(self._h, float(dt), int(nsteps)))

    def step_async(self, dt: float, nsteps: int) -> None:
        self._step_check(load().ms_step_async(self._h, float(dt), int(nsteps)))

    def sync(self) -> None:
        _check(load().ms_sync(self._h))

    def moments(self) -> np.ndarray:
        out = np.zeros((self.ncell, NMOM))
        _check(load().ms_moments(self._h, _ptr(out)))
        return out

    def floes(self) -> dict:
        out = np.zeros((8, self.n))
        _check(load().ms_get_floes(self._h, _ptr(out)))
        return {k: out[i] for i, k in enumerate(FLOE_KEYS)}

    def set_floes(self, floes: dict) -> None:
        fl, keep = make_floes(floes)
        _check(load().ms_set_floes(self._h, C.byref(fl)))

    def coupling(self) -> dict:
        nc = self.ncell
        q = np.zeros((4, nc)); tg = np.zeros((4, nc)); win = np.zeros((NWIN, nc))
        fl = np.zeros(3, dtype=np.int64)
        _check(load().ms_coupling(self._h, _ptr(q), _ptr(tg), _ptr(win),
                                  fl.ctypes.data_as(C.POINTER(C.c_int64))))
        return {"q": q, "targets": tg, "window": win, "have_q": int(fl[0]), "have_targets": int(fl[1]),
                "steps": int(fl[2])}

    def truth_step(self, dt: float, nsteps: int) -> None:
        _check(load().ms_truth_step(self._h, float(dt), int(nsteps)))

    def truth_moments(self) -> np.ndarray:
        out = np.zeros((self.ncell, NMOM))
        _check(load().ms_truth_moments(self._h, _ptr(out)))
        return out

    def truth_floes(self) -> dict:
        out = np.zeros((8, self.n))
        _check(load().ms_truth_get_floes(self._h, _ptr(out)))
        return {k: out[i] for i, k in enumerate(FLOE_KEYS)}

    def set_stream(self, stream_handle: int | None) -> None:
        _check(load().ms_set_stream(self._h, C.c_void_p(stream_handle or 0)))

    def autotune(self, dt: float, reps: int = 5) -> float:
        best = C.c_double(0.0)
        _check(load().ms_autotune(self._h, float(dt), int(reps), C.byref(best)))
        return best.value

    def time_kernel(self, which: int, dt: float, reps: int = 10) -> float:
        out = C.c_double(0.0)
        _check(load().ms_time_kernel(self._h, int(which), float(dt), int(reps), C.byref(out)))
        return out.value

    def save(self, path: str) -> None:
        """Checkpoint the model's whole state to `path` (ms_save)."""
        _check(load().ms_save(self._h, os.fsencode(path)))

    def load_checkpoint(self, path: str) -> None:
        """Resume from a checkpoint written by save() (ms_load)."""
        _check(load().ms_load(self._h, os.fsencode(path)))

    def set_launch(self, variant: int = 0, threads: int = 128, persistent: int = 0,
                   bin_beta: float = 1.0) -> None:
        _check(load().ms_set_launch(self._h, int(variant), int(threads), int(persistent), float(bin_beta)))

    def closure_attach(self, mlp, mode: int = 0, tol: float = 0.5, box=None) -> None:
        """mode 0: network `mlp` (predicting the tendencies) with fallback;
        2: as 0 with `mlp` predicting their change from the interval before;
        1: mean-field closure; -1: off."""
        self._mlp_ref = mlp
        bx = None if box is None else np.ascontiguousarray(box, dtype=np.float32).reshape(2 * NFEAT)
        self._box = bx
        _check(load().ms_closure_attach(self._h, mlp._h if mlp is not None else None, int(mode), float(tol),
                                        bx.ctypes.data_as(C.POINTER(C.c_float)) if bx is not None else None))

    def closure_collect(self, nint: int):
        X = np.zeros((nint, self.ncell, NFEAT), dtype=np.float32)
        Y = np.zeros((nint, self.ncell, 4), dtype=np.float32)
        _check(load().ms_closure_collect(self._h, int(nint), X.ctypes.data_as(C.POINTER(C.c_float)),
                                         Y.ctypes.data_as(C.POINTER(C.c_float))))
        return X, Y

    def closure_stats(self) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(load().ms_closure_stats(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return {"closure_cell_intervals": int(out[0]), "cells": int(out[1]), "mode": int(out[2]),
                "intervals": int(out[3])}

    def set_resident(self, skin_steps: float = 32.0, block_floes: int = 256) -> None:
        _check(load().ms_set_resident(self._h, float(skin_steps), int(block_floes)))

    def layout(self):
        """(off [ncell + 1], orig [n]): each cell's first stored floe and the
        caller's index of every stored floe (ms_layout)."""
        off = np.zeros(self.ncell + 1, dtype=np.int32)
        orig = np.zeros(max(self.n, 1), dtype=np.int32)
        _check(load().ms_layout(self._h, off.ctypes.data_as(_ip32), orig.ctypes.data_as(_ip32)))
        return off, orig[: self.n]

    def set_shard(self, nranks: int, rank: int, rank_off, cells, exchange) -> None:
        """Make this model rank `rank` of a sharded grid (ms_set_shard).
        exchange(stream_handle) gathers every rank's send rows into recv
        (shard_buffers) ordered on that stream; an exception in it fails the
        step that called it and is re-raised from there."""
        rank_off = np.ascontiguousarray(rank_off, dtype=np.int32)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        self._exch_error = None

        def cb(ctx, stream):
            try:
                exchange(int(stream or 0))
                return 0
            except BaseException as e:  # reported through the failing step
                self._exch_error = e
                return 1

        fn = EXCHANGE_FN(cb)
        _check(load().ms_set_shard(self._h, int(nranks), int(rank), rank_off.ctypes.data_as(_ip32),
                                   cells.ctypes.data_as(_ip32), fn, None))
        self._exch_keep = (fn, rank_off, cells)
        self._shard = (int(nranks), int(rank))

    def shard_buffers(self):
        """(send, recv, max_cells): DeviceArray views of the exchange
        buffers, [max_cells][10] and [nranks * max_cells][10] FP64."""
        snd, rcv, mc = _dp(), _dp(), C.c_int32()
        _check(load().ms_shard_buffers(self._h, C.byref(snd), C.byref(rcv), C.byref(mc)))
        nranks = self._shard[0]
        addr = lambda p: C.cast(p, C.c_void_p).value
        return (DeviceArray(addr(snd), (mc.value, SHARD_NCOL)),
                DeviceArray(addr(rcv), (nranks * mc.value, SHARD_NCOL)), mc.value)

    def info(self) -> dict:
        out = np.zeros(21, dtype=np.int64)
        _check(load().ms_info(self._h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        keys = ["n", "ncell", "max_n", "precision", "variant", "threads", "bin_beta_milli",
                "launches_per_interval", "launches_per_coarse", "launches_per_truth_step", "steps",
                "truth_steps", "graph_replays", "deep_contacts", "persistent", "N1", "skin_steps_milli",
                "block_floes", "shard_ranks", "shard_rank", "shard_cells"]
        return {k: int(v) for k, v in zip(keys, out)}


def cell_moments_noalloc(params: dict, n: int, x: int, y: int, u: int, v: int, omega: int, r: int, h: int,
                         fd: int, out: int, stream: int | None = None) -> None:
    """Per-cell moments of floes in device memory (addresses as ints, FP64),
    computed without any device allocation (see ms_cell_moments_noalloc in
    include/msdem.h): for callers that must not allocate while they run.
    `out` receives ncell x 12 doubles; fd is [3][n] per-floe drag."""
    L = load()
    g = Grid(int(params["nx"]), int(params["ny"]), float(params["Lx"]), float(params["Ly"]),
             max(1, int(params.get("nens", 1))))
    ptrs = [C.c_void_p(a) for a in (x, y, u, v, omega, r, h, fd, out)]
    _check(L.ms_cell_moments_noalloc(C.byref(g), float(params["rho_ice"]), int(params.get("inertia_half", 0)),
                                     int(n), *ptrs, C.c_void_p(stream or 0)))


NFEAT = 16       # closure features per cell
MLP_SHAPES = [("W1", (128, NFEAT)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
              ("W3", (128, 128)), ("b3", (128,)), ("W4", (4, 128)), ("b4", (4,))]
NPARAM = sum(int(np.prod(shp)) for _, shp in MLP_SHAPES)
_fp = C.POINTER(C.c_float)


def probe_fp32(reps: int = 5) -> float:
    """FP32 FMA throughput of the current GPU in TFLOP/s (ms_probe_fp32)."""
    out = np.zeros(1)
    _check(load().ms_probe_fp32(int(reps), _ptr(out)))
    return float(out[0])


def pack_params(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1) for k, _ in MLP_SHAPES])


def unpack_params(flat: np.ndarray) -> dict:
    out, off = {}, 0
    for k, shp in MLP_SHAPES:
        n = int(np.prod(shp))
        out[k] = flat[off:off + n].reshape(shp)
        off += n
    return out


def _load_mlp():
    L = load()
    if getattr(L, "_mlp_ready", False):
        return L
    vp = C.c_void_p
    L.ms_mlp_create.argtypes = [C.POINTER(vp), _fp, _fp, C.c_int32]
    L.ms_mlp_predict.argtypes = [vp, _fp, C.c_int64, _fp]
    L.ms_mlp_grad.argtypes = [vp, _fp, _fp, C.c_int64, _fp, C.POINTER(C.c_double)]
    L.ms_mlp_step.argtypes = [vp, _fp, _fp, C.c_int64, C.c_float]
    L.ms_mlp_train.argtypes = [vp, _fp, _fp, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_uint64,
                               C.POINTER(C.c_double)]
    L.ms_mlp_get_params.argtypes = [vp, _fp]
    L.ms_mlp_forward_device.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.ms_mlp_fit_norm.argtypes = [_fp, _fp, C.c_int64, _fp]
    L.ms_mlp_set_engine.argtypes = [vp, C.c_int32]
    L.ms_mlp_check.argtypes = [vp]
    L.ms_mlp_free.argtypes = [vp]
    L.ms_mlp_free.restype = None
    for n in ("ms_mlp_create", "ms_mlp_predict", "ms_mlp_grad", "ms_mlp_step", "ms_mlp_train",
              "ms_mlp_get_params", "ms_mlp_forward_device", "ms_mlp_fit_norm", "ms_mlp_set_engine",
              "ms_mlp_check"):
        getattr(L, n).restype = C.c_int
    L._mlp_ready = True
    return L


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def fit_norm(X, Y) -> dict:
    """Per-column mean and population sd of a training set (features X[n][16],
    targets Y[n][4]), computed by the library on the device: the z-scoring the
    network's loss uses, as the dict MLP() takes."""
    X, Y = _f32(X), _f32(Y)
    if X.ndim != 2 or X.shape[1] != 16 or Y.shape != (X.shape[0], 4):
        raise ValueError("X must be [n][16] and Y [n][4]")
    out = np.zeros(40, dtype=np.float32)
    _check(_load_mlp().ms_mlp_fit_norm(X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0],
                                       out.ctypes.data_as(_fp)))
    return {"mu_x": out[:16].astype(np.float64), "sd_x": out[16:32].astype(np.float64),
            "mu_y": out[32:36].astype(np.float64), "sd_y": out[36:40].astype(np.float64)}


class MLP:
    """The closure network on the current CUDA device (see include/msdem.h)."""

    def __init__(self, params: dict, norm: dict, max_batch: int = 8192):
        L = _load_mlp()
        self._keep = [pack_params(params),
                      _f32(np.concatenate([norm["mu_x"], norm["sd_x"], norm["mu_y"], norm["sd_y"]]))]
        h = C.c_void_p()
        _check(L.ms_mlp_create(C.byref(h), self._keep[0].ctypes.data_as(_fp), self._keep[1].ctypes.data_as(_fp),
                               int(max_batch)))
        self._h = h
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "_h", None):
            _load_mlp().ms_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward_device(self, x_ptr: int, n: int, y_ptr: int, stream: int | None = None) -> None:
        """Device X[n][16] -> device Y[n][4] (addresses as ints) on `stream`,
        without waiting (ms_mlp_forward_device)."""
        _check(_load_mlp().ms_mlp_forward_device(self._h, C.c_void_p(x_ptr), int(n), C.c_void_p(y_ptr),
                                                 C.c_void_p(stream) if stream else None))

    def set_engine(self, engine: int) -> None:
        """1: the tcgen05 kernels for inference and training (default); 0: the mma.sync GEMMs."""
        _check(_load_mlp().ms_mlp_set_engine(self._h, int(engine)))

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        Y = np.zeros((X.shape[0], 4), dtype=np.float32)
        _check(_load_mlp().ms_mlp_predict(self._h, X.ctypes.data_as(_fp), X.shape[0], Y.ctypes.data_as(_fp)))
        return Y

    def grad(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        g = np.zeros(NPARAM, dtype=np.float32)
        loss = C.c_double(0.0)
        _check(_load_mlp().ms_mlp_grad(self._h, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0],
                                       g.ctypes.data_as(_fp), C.byref(loss)))
        return loss.value, unpack_params(g)

    def step(self, X, Y, lr: float) -> None:
        X, Y = _f32(X), _f32(Y)
        _check(_load_mlp().ms_mlp_step(self._h, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0],
                                       float(lr)))

    def train(self, X, Y, epochs: int, batch: int, lr: float, seed: int = 1) -> np.ndarray:
        X, Y = _f32(X), _f32(Y)
        losses = np.zeros(epochs)
        _check(_load_mlp().ms_mlp_train(self._h, X.ctypes.data_as(_fp), Y.ctypes.data_as(_fp), X.shape[0],
                                        int(epochs), int(batch), float(lr), int(seed),
                                        losses.ctypes.data_as(C.POINTER(C.c_double))))
        return losses

    def params(self) -> dict:
        flat = np.zeros(NPARAM, dtype=np.float32)
        _check(_load_mlp().ms_mlp_get_params(self._h, flat.ctypes.data_as(_fp)))
        return {k: v.astype(np.float64) for k, v in unpack_params(flat).items()}
