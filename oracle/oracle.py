"""Python access to the FP64 CPU oracle (``ms_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (``paper_2303_07819_gb300``) never imports this module and shares
no code with it; both sides only read the seeded inputs of
``paper_2303_07819_gb300.inputs``.

``build()`` compiles the C oracle with gcc (``-ffp-contract=off`` so that x86
and Arm hosts round identically; OpenMP over cells when available).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libms_oracle.so")
NMOM = 12
NWIN = 5

MOMENT_NAMES = ["n", "M", "Mu", "Mv", "I", "Iw", "area", "Muu", "Mvv", "Fdx", "Fdy", "Td"]


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("Lx", C.c_double), ("Ly", C.c_double),
        ("uo_x", C.c_double), ("uo_y", C.c_double), ("n_modes", C.c_int32),
        ("modes", C.POINTER(C.c_double)),
        ("rho_o", C.c_double), ("Cd", C.c_double), ("rho_a", C.c_double), ("Ca", C.c_double),
        ("wind_x", C.c_double), ("wind_y", C.c_double), ("wind_period", C.c_double),
        ("rho_ice", C.c_double), ("E", C.c_double), ("G", C.c_double), ("eta", C.c_double),
        ("mu", C.c_double), ("h_ref", C.c_double), ("inertia_half", C.c_int32),
        ("couple", C.c_int32), ("N0", C.c_int32), ("n_t", C.c_int32),
        ("n_vmodes", C.c_int32), ("vmodes", C.POINTER(C.c_double)),
        ("walls", C.c_int32),
    ]


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "ms_oracle.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", LIB, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int64)
        ip32 = C.POINTER(C.c_int32)
        P = C.POINTER(Params)
        L.orc_forcing.argtypes = [P, C.c_double, C.c_double, C.c_double, dp]
        L.orc_pair.argtypes = [P, C.c_double, C.c_double] + [C.c_double] * 14 + [dp]
        L.orc_pair.restype = C.c_int
        L.orc_contacts.argtypes = [P, C.c_double, C.c_double, C.c_int64, dp, dp, dp, ip, C.c_int64]
        L.orc_contacts.restype = C.c_int64
        L.orc_lf.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, dp, dp, dp,
                             C.c_double, C.c_int32]
        L.orc_lf_bc.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, dp, dp, dp,
                                C.c_double, C.c_int32, C.c_int32]
        L.orc_wall.argtypes = [P, C.c_double] + [C.c_double] * 6 + [dp]
        L.orc_wall.restype = C.c_int
        L.orc_model_create.argtypes = [P, C.c_int64] + [dp] * 8
        L.orc_model_create.restype = C.c_void_p
        L.orc_model_free.argtypes = [C.c_void_p]
        L.orc_model_step.argtypes = [C.c_void_p, C.c_double, C.c_int64]
        L.orc_model_step.restype = C.c_int
        L.orc_model_moments.argtypes = [C.c_void_p, dp]
        L.orc_model_floes.argtypes = [C.c_void_p, dp]
        L.orc_model_coupling.argtypes = [C.c_void_p, dp, dp, dp, ip]
        L.orc_model_layout.argtypes = [C.c_void_p, ip, ip]
        L.orc_model_set_hold.argtypes = [C.c_void_p, C.c_int32]
        L.orc_model_set_hold.restype = None
        L.orc_model_pending.argtypes = [C.c_void_p]
        L.orc_model_pending.restype = C.c_int32
        L.orc_model_coarse_inputs.argtypes = [C.c_void_p, dp]
        L.orc_model_coarse_inputs.restype = None
        L.orc_model_set_coarse_inputs.argtypes = [C.c_void_p, C.c_int32, ip32, dp]
        L.orc_model_set_coarse_inputs.restype = None
        L.orc_model_coarse.argtypes = [C.c_void_p]
        L.orc_model_coarse.restype = C.c_int
        L.orc_truth_create.argtypes = [P, C.c_int64] + [dp] * 8
        L.orc_truth_create.restype = C.c_void_p
        L.orc_truth_free.argtypes = [C.c_void_p]
        L.orc_truth_step.argtypes = [C.c_void_p, C.c_double, C.c_int64]
        L.orc_truth_step.restype = C.c_int
        L.orc_truth_moments.argtypes = [C.c_void_p, dp]
        L.orc_truth_floes.argtypes = [C.c_void_p, dp]
        L.orc_truth_set_brute.argtypes = [C.c_void_p, C.c_int32]
        L.orc_l2_diff.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, dp, dp]
        L.orc_l2_diff.restype = C.c_double
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_get_threads.restype = C.c_int32
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def make_params(p: dict):
    """Build the C parameter struct from a scenario parameter dict.  Returns
    (struct, keep-alive arrays of the stream and velocity modes)."""
    modes = np.ascontiguousarray(np.asarray(p.get("modes", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4))
    vmodes = np.ascontiguousarray(np.asarray(p.get("vmodes", np.zeros((0, 5))), dtype=np.float64).reshape(-1, 5))
    s = Params()
    s.nx, s.ny = int(p["nx"]), int(p["ny"])
    s.Lx, s.Ly = float(p["Lx"]), float(p["Ly"])
    s.uo_x, s.uo_y = float(p.get("uo_x", 0.0)), float(p.get("uo_y", 0.0))
    s.n_modes = modes.shape[0]
    s.modes = _dp(modes) if modes.shape[0] else C.POINTER(C.c_double)()
    for k in ("rho_o", "Cd", "rho_a", "Ca", "wind_x", "wind_y", "wind_period", "rho_ice",
              "E", "G", "eta", "mu", "h_ref"):
        setattr(s, k, float(p.get(k, 0.0)))
    s.inertia_half = int(p.get("inertia_half", 0))
    s.couple, s.N0, s.n_t = int(p.get("couple", 0)), int(p.get("N0", 100)), int(p.get("n_t", 10))
    s.n_vmodes = vmodes.shape[0]
    s.vmodes = _dp(vmodes) if vmodes.shape[0] else C.POINTER(C.c_double)()
    s.walls = int(p.get("walls", 0))
    return s, (modes, vmodes)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def forcing(p: dict, X: float, Y: float, t: float = 0.0) -> np.ndarray:
    s, keep = make_params(p)
    out = np.zeros(5)
    lib().orc_forcing(C.byref(s), X, Y, t, _dp(out))
    return out


def pair(p: dict, Px: float, Py: float, fl: tuple, fj: tuple):
    """fl, fj = (x, y, u, v, omega, r, h).  Returns (contact, out[16])."""
    s, keep = make_params(p)
    out = np.zeros(16)
    hit = lib().orc_pair(C.byref(s), Px, Py, *[float(a) for a in fl], *[float(a) for a in fj], _dp(out))
    return bool(hit), out


def wall(p: dict, Lx: float, fl: tuple):
    """Floe fl = (x, u, v, omega, r, h) against the walls X = 0 and X = Lx.
    Returns (walls touched, out[16])."""
    s, keep = make_params(p)
    out = np.zeros(16)
    hit = lib().orc_wall(C.byref(s), Lx, *[float(a) for a in fl], _dp(out))
    return int(hit), out


def contacts(p: dict, Px: float, Py: float, x, y, r) -> set:
    s, keep = make_params(p)
    x, y, r = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, r))
    n = x.shape[0]
    mx = n * (n - 1) // 2 + 1
    pairs = np.zeros(2 * mx, dtype=np.int64)
    cnt = lib().orc_contacts(C.byref(s), Px, Py, n, _dp(x), _dp(y), _dp(r), _ip(pairs), mx)
    return {(int(pairs[2 * k]), int(pairs[2 * k + 1])) for k in range(cnt)}


def lf(nx, ny, dx, dy, q, V, S, dtau, nsub) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    V = np.ascontiguousarray(V, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    lib().orc_lf(nx, ny, dx, dy, _dp(q), _dp(V), _dp(S), dtau, nsub)
    return q


def lf_bc(nx, ny, dx, dy, q, V, S, dtau, nsub, walls) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    V = np.ascontiguousarray(V, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    lib().orc_lf_bc(nx, ny, dx, dy, _dp(q), _dp(V), _dp(S), dtau, nsub, int(walls))
    return q


def l2_diff(nx, ny, dx, dy, a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib().orc_l2_diff(nx, ny, dx, dy, _dp(a), _dp(b)))


FLOE_KEYS = ("x", "y", "theta", "u", "v", "omega", "r", "h")


class _Base:
    _create = _free = _step = _moments = _floes = None

    def __init__(self, params: dict, floes: dict):
        self.params = dict(params)
        self._p, self._keep = make_params(self.params)
        arrs = [np.ascontiguousarray(floes[k], dtype=np.float64) for k in FLOE_KEYS]
        self.n = arrs[0].shape[0]
        L = lib()
        self._h = getattr(L, self._create)(C.byref(self._p), self.n, *[_dp(a) for a in arrs])
        self.ncell = int(params["nx"]) * int(params["ny"])

    def close(self):
        if self._h:
            getattr(lib(), self._free)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt: float, nsteps: int) -> None:
        rc = getattr(lib(), self._step)(self._h, dt, int(nsteps))
        if rc != 0:
            raise ValueError(f"oracle step rejected its arguments (rc={rc})")

    def moments(self) -> np.ndarray:
        out = np.zeros((self.ncell, NMOM))
        getattr(lib(), self._moments)(self._h, _dp(out))
        return out

    def floes(self) -> dict:
        out = np.zeros((8, self.n))
        getattr(lib(), self._floes)(self._h, _dp(out))
        return {k: out[i] for i, k in enumerate(FLOE_KEYS)}


class Model(_Base):
    """msDEM: one doubly periodic DEM per coarse cell + Algorithm 1 coupling."""
    _create, _free, _step = "orc_model_create", "orc_model_free", "orc_model_step"
    _moments, _floes = "orc_model_moments", "orc_model_floes"

    def coupling(self):
        nc = self.ncell
        q = np.zeros((4, nc)); tg = np.zeros((4, nc)); win = np.zeros((NWIN, nc))
        fl = np.zeros(3, dtype=np.int64)
        lib().orc_model_coupling(self._h, _dp(q), _dp(tg), _dp(win), _ip(fl))
        return {"q": q, "targets": tg, "window": win, "have_q": int(fl[0]),
                "have_targets": int(fl[1]), "steps": int(fl[2])}

    def layout(self):
        off = np.zeros(self.ncell + 1, dtype=np.int64)
        orig = np.zeros(max(self.n, 1), dtype=np.int64)
        lib().orc_model_layout(self._h, _ip(off), _ip(orig))
        return off, orig[: self.n]

    # sharded runs: stop before each coarse step, exchange its inputs
    NCI = 10

    def set_hold(self, hold: bool) -> None:
        lib().orc_model_set_hold(self._h, 1 if hold else 0)

    def coarse_pending(self) -> bool:
        return bool(lib().orc_model_pending(self._h))

    def coarse_inputs(self) -> np.ndarray:
        """[ncell][10]: moment columns 1-5 and the window sums of every cell."""
        out = np.zeros((self.ncell, self.NCI))
        lib().orc_model_coarse_inputs(self._h, _dp(out))
        return out

    def set_coarse_inputs(self, cells, vals) -> None:
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64).reshape(cells.shape[0], self.NCI)
        lib().orc_model_set_coarse_inputs(self._h, int(cells.shape[0]), cells.ctypes.data_as(C.POINTER(C.c_int32)),
                                          _dp(vals))

    def coarse(self) -> None:
        if lib().orc_model_coarse(self._h) != 0:
            raise ValueError("no coarse step is pending")


class Truth(_Base):
    """The un-localised DEM over the whole periodic domain."""
    _create, _free, _step = "orc_truth_create", "orc_truth_free", "orc_truth_step"
    _moments, _floes = "orc_truth_moments", "orc_truth_floes"

    def set_brute(self, brute: bool) -> None:
        """True: contact forces by the plain all-pairs loop (the definition);
        False (default): the binned search, identical bit for bit."""
        lib().orc_truth_set_brute(self._h, int(bool(brute)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
