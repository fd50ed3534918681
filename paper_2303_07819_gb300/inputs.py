"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path, the oracle and the tests, so it holds
none of the method's arithmetic: no forces, drag, integration, moments, coarse
solver or coupling.  It only draws floe fields, ocean-mode coefficients and
physical constants.

Every scenario is a dict::

    {"name", "params": {...}, "floes": {x, y, theta, u, v, omega, r, h}, "dt", "nsteps", "meta"}

``params`` uses SI units (the paper's Sec. 4 scenarios are non-dimensional and
keep the paper's units).  Ocean current: uniform part ``uo_x, uo_y`` plus the
stream function ``psi = sum A sin(2 pi (kx X/Lx + ky Y/Ly) + phi)`` given as
rows ``modes[m] = (A, kx, ky, phi)``.

Constants the paper leaves open (contact stiffness E, shear coefficient G,
normal dashpot eta, densities) are chosen here; E makes the contact time of
the smallest floe pair several fine steps, and eta = 2.5 E dt keeps forward
Euler from gaining energy in a contact (the linearised gain per step is
w^2 dt^2, the dashpot loss 2 zeta w dt, and 2 zeta / (w dt) = eta / (1.5 E dt)
for the chord-length law).
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20230314

RHO_ICE = 920.0
RHO_O = 1026.0
RHO_A = 1.3


def _phys(dt: float, E: float = 4.0e3, G: float = 5.0e3) -> dict:
    return {
        "rho_o": RHO_O, "Cd": 5.5e-3, "rho_a": RHO_A, "Ca": 0.0,
        "wind_x": 0.0, "wind_y": 0.0, "wind_period": 0.0,
        "rho_ice": RHO_ICE, "E": E, "G": G, "eta": 2.5 * E * dt, "mu": 0.3, "h_ref": 1.0,
        "inertia_half": 0, "couple": 1, "N0": 100, "n_t": 10,
        "uo_x": 0.0, "uo_y": 0.0,
    }


def psi_sin_sin_modes(U: float, L: float) -> np.ndarray:
    """psi = U L sin(2 pi x / L) sin(2 pi y / L) written as two modes:
    sin a sin b = (sin(a - b + pi/2) - sin(a + b + pi/2)) / 2."""
    A = 0.5 * U * L
    return np.array([[A, 1.0, -1.0, 0.5 * math.pi], [-A, 1.0, 1.0, 0.5 * math.pi]])


def random_modes(rng: np.random.Generator, n_modes: int, Lx: float, Ly: float,
                 rms_speed: float, kmax: int = 4) -> np.ndarray:
    """n_modes distinct integer wave vectors with 1 <= max(|kx|,|ky|) <= kmax
    (no two opposite), random phases, amplitudes scaled so the domain-mean
    speed^2 of the current equals rms_speed^2 (Parseval: sum A^2 |k|^2 / 2)."""
    cand = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
            if max(abs(kx), abs(ky)) >= 1 and (kx > 0 or (kx == 0 and ky > 0))]
    pick = rng.choice(len(cand), size=n_modes, replace=False)
    ks = np.array([cand[i] for i in pick], dtype=np.float64)
    A = rng.uniform(0.5, 1.5, size=n_modes) * rng.choice([-1.0, 1.0], size=n_modes)
    phi = rng.uniform(0.0, 2 * math.pi, size=n_modes)
    k2 = (2 * math.pi * ks[:, 0] / Lx) ** 2 + (2 * math.pi * ks[:, 1] / Ly) ** 2
    scale = rms_speed / math.sqrt(np.sum(A * A * k2) / 2.0)
    return np.stack([A * scale, ks[:, 0], ks[:, 1], phi], axis=1)


def power_law_radii(rng: np.random.Generator, n: int, rmin: float, rmax: float) -> np.ndarray:
    """p(r) ~ r^-2 on [rmin, rmax] by inverse CDF."""
    u = rng.uniform(0.0, 1.0, size=n)
    return 1.0 / (1.0 / rmin - u * (1.0 / rmin - 1.0 / rmax))


def lognormal_mean_sd(rng: np.random.Generator, n: int, mean: float, sd: float) -> np.ndarray:
    s2 = math.log(1.0 + (sd / mean) ** 2)
    return rng.lognormal(math.log(mean) - 0.5 * s2, math.sqrt(s2), size=n)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def place_floes(rng: np.random.Generator, nx: int, ny: int, Lx: float, Ly: float,
                radii: list, domain_check: bool, max_tries: int = 300,
                shrink: float = 0.9) -> tuple:
    """Random sequential placement, largest floe first, of the floes of every
    coarse cell, with no overlap under the cell-periodic metric and, when
    domain_check, under the domain-periodic metric as well.  Cells of the same
    2x2 colour are placed together (they cannot touch while 2 r_max < cell
    side).  A floe that finds no room after max_tries is shrunk by `shrink` and
    tried again.  Returns (x, y, r, cell) in global coordinates, floes grouped
    by cell (cell = iy * nx + ix)."""
    ncell = nx * ny
    Lcx, Lcy = Lx / nx, Ly / ny
    counts = np.array([len(r) for r in radii], dtype=np.int64)
    nmax = int(counts.max()) if ncell else 0
    R = np.zeros((ncell, max(nmax, 1)))
    for c in range(ncell):
        R[c, : counts[c]] = np.sort(radii[c])[::-1]
    X = np.full((ncell, max(nmax, 1)), np.nan)
    Y = np.full((ncell, max(nmax, 1)), np.nan)
    cx = (np.arange(ncell) % nx).astype(np.float64)
    cy = (np.arange(ncell) // nx).astype(np.float64)
    if domain_check:
        ix = np.arange(ncell) % nx
        iy = np.arange(ncell) // nx
        groups = [np.nonzero((ix % 2 == a) & (iy % 2 == b))[0] for a in (0, 1) for b in (0, 1)]
        nb = np.stack([((iy + dy) % ny) * nx + (ix + dx) % nx
                       for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)], axis=1)
    else:
        groups = [np.arange(ncell)]
    for k in range(nmax):
        for g in groups:
            pend = g[counts[g] > k]
            while pend.size:
                for _ in range(max_tries):
                    if not pend.size:
                        break
                    px = rng.uniform(0.0, Lcx, size=pend.size)
                    py = rng.uniform(0.0, Lcy, size=pend.size)
                    rk = R[pend, k]
                    dx = _min_image(px[:, None] - X[pend, :k], Lcx)
                    dy = _min_image(py[:, None] - Y[pend, :k], Lcy)
                    bad = np.any(dx * dx + dy * dy < (rk[:, None] + R[pend, :k]) ** 2, axis=1)
                    if domain_check:
                        nbc = nb[pend]                                   # [p, 8]
                        gx = X[nbc] + (cx[nbc] * Lcx)[:, :, None]        # [p, 8, nmax]
                        gy = Y[nbc] + (cy[nbc] * Lcy)[:, :, None]
                        qx = (px + cx[pend] * Lcx)[:, None, None]
                        qy = (py + cy[pend] * Lcy)[:, None, None]
                        ddx = _min_image(qx - gx, Lx)
                        ddy = _min_image(qy - gy, Ly)
                        rr = (rk[:, None, None] + R[nbc]) ** 2
                        bad |= np.any((ddx * ddx + ddy * ddy < rr).reshape(pend.size, -1), axis=1)
                    ok = ~bad
                    X[pend[ok], k] = px[ok]
                    Y[pend[ok], k] = py[ok]
                    pend = pend[bad]
                if pend.size:
                    R[pend, k] *= shrink
    xs, ys, rs, cs = [], [], [], []
    for c in range(ncell):
        n = counts[c]
        xs.append(X[c, :n] + cx[c] * Lcx)
        ys.append(Y[c, :n] + cy[c] * Lcy)
        rs.append(R[c, :n])
        cs.append(np.full(n, c, dtype=np.int64))
    cat = (lambda a, dt=np.float64: np.concatenate(a).astype(dt) if a else np.zeros(0, dt))
    return cat(xs), cat(ys), cat(rs), cat(cs, np.int64)


def _floes(x, y, r, h, u=None, v=None, omega=None) -> dict:
    n = x.shape[0]
    z = np.zeros(n)
    return {"x": x, "y": y, "theta": z.copy(), "u": z.copy() if u is None else u,
            "v": z.copy() if v is None else v, "omega": z.copy() if omega is None else omega,
            "r": r, "h": h}


def _rescale_cells(radii: list, Ac: float, target: float) -> tuple:
    """Per cell, scale radii by min(1, sqrt(target A_c / sum pi r^2))."""
    out, scales = [], []
    for r in radii:
        a = float(np.sum(np.pi * r * r))
        s = min(1.0, math.sqrt(target * Ac / a)) if a > 0 else 1.0
        out.append(r * s)
        scales.append(s)
    return out, np.array(scales)


def square_4x4(seed: int | None = None) -> dict:
    """Plain msDEM, FP64: periodic 100 km square, 4 x 4 cells, 16 floes per cell,
    r ~ U[1, 2.5] km, h = 1 m; psi = U L sin sin with U = 0.1 m/s; no wind;
    dt = 10 s, 1000 steps; the truth DEM runs on the same floes."""
    rng = np.random.default_rng(BASE_SEED if seed is None else seed)
    nx = ny = 4
    L = 100e3
    radii = [rng.uniform(1000.0, 2500.0, size=16) for _ in range(nx * ny)]
    x, y, r, cell = place_floes(rng, nx, ny, L, L, radii, domain_check=True)
    h = np.ones_like(x)
    p = _phys(dt=10.0)
    p.update({"nx": nx, "ny": ny, "Lx": L, "Ly": L, "modes": psi_sin_sin_modes(0.1, L)})
    return {"name": "periodic 100 km, 4x4 cells, 16 floes/cell (256 floes)", "params": p,
            "floes": _floes(x, y, r, h), "dt": 10.0, "nsteps": 1000,
            "meta": {"cell": cell}}


def _powerlaw_config(rng, nx, ny, L, counts, dt, nsteps, wind, wind_period, domain_check,
                     name, conc=0.55):
    Ac = (L / nx) * (L / ny)
    radii = [power_law_radii(rng, int(n), 200.0, 3000.0) for n in counts]
    radii, scales = _rescale_cells(radii, Ac, conc)
    x, y, r, cell = place_floes(rng, nx, ny, L, L, radii, domain_check=domain_check)
    h = lognormal_mean_sd(rng, x.shape[0], 1.5, 0.5)
    p = _phys(dt=dt)
    p.update({"nx": nx, "ny": ny, "Lx": L, "Ly": L,
              "modes": random_modes(rng, 8, L, L, 0.1),
              "Ca": 1.2e-3, "wind_x": wind[0], "wind_y": wind[1], "wind_period": wind_period})
    return {"name": name, "params": p, "floes": _floes(x, y, r, h), "dt": dt, "nsteps": nsteps,
            "meta": {"cell": cell, "radius_scale": scales}}


def powerlaw_32x32(seed: int | None = None, nx: int = 32) -> dict:
    """32 x 32 cells over a periodic 400 km square (L_c = 12.5 km), floes per cell
    ~ Poisson(64), power-law radii 0.2-3 km, lognormal thickness (1.5, 0.5) m,
    8-mode ocean with 0.1 m/s RMS, uniform 10 m/s wind with Ca = 1.2e-3,
    dt = 5 s, 2000 steps.  `nx` < 32 keeps L_c and the laws on a smaller
    square (used for quick parity cases)."""
    rng = np.random.default_rng((BASE_SEED + 1) if seed is None else seed)
    L = 12.5e3 * nx
    counts = np.maximum(rng.poisson(64, size=nx * nx), 1)
    return _powerlaw_config(rng, nx, nx, L, counts, 5.0, 2000, (10.0, 0.0), 0.0, True,
                            f"periodic {L/1e3:.0f} km, {nx}x{nx} cells, Poisson(64) floes/cell")


def lognormal_counts(rng, ncell: int, median: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    n = np.rint(median * np.exp(sigma * rng.standard_normal(ncell)))
    return np.clip(n, lo, hi).astype(np.int64)


def batched_128x128(seed: int | None = None, nx: int = 128) -> dict:
    """128 x 128 cells of 25 km (3200 km periodic square), floes per cell
    lognormal(median 96, sigma 0.69) clipped to [8, 1024] (~2.0M floes),
    radius/thickness/ocean laws of powerlaw_32x32, wind of 10 m/s rotating with a
    6 h period, dt = 5 s, 5000 steps.  No truth run, so only the cell metric
    is kept overlap-free."""
    rng = np.random.default_rng((BASE_SEED + 2) if seed is None else seed)
    L = 25e3 * nx
    counts = lognormal_counts(rng, nx * nx, 96.0, 0.69, 8, 1024)
    return _powerlaw_config(rng, nx, nx, L, counts, 5.0, 5000, (10.0, 0.0), 6 * 3600.0, False,
                            f"periodic {L/1e3:.0f} km, {nx}x{nx} cells, lognormal(96, 0.69) floes/cell")


def stack_ensemble(scens: list) -> dict:
    """An ensemble of realizations of one grid and forcing (different floes)
    as one model input: realization e's floes move to y + e Ly (the stacking
    of ms_grid.nens); params from the first realization with nens set."""
    p = dict(scens[0]["params"], nens=len(scens))
    Ly = p["Ly"]
    fl = {k: np.concatenate([sc["floes"][k] + (e * Ly if k == "y" else 0.0) for e, sc in enumerate(scens)])
          for k in scens[0]["floes"]}
    return {"name": f"{len(scens)} realizations of {scens[0]['name']}", "params": p, "floes": fl,
            "dt": scens[0]["dt"], "nsteps": scens[0]["nsteps"], "meta": {}}


def ensemble_16x256x256(nreal: int = 16, nx: int = 256, seed: int | None = None) -> dict:
    """Ensemble batch: nreal seeded realizations of an nx x nx grid of 25 km
    cells with few floes per cell, lognormal(median 6, sigma 0.69) clipped to
    [1, 64] (about 7.6 on average; 16 x 256^2 cells hold about 8M floes),
    radius/thickness laws of powerlaw_32x32, one ocean (8 modes) and one wind (10 m/s
    turning with a 6 h period) for all realizations, dt = 5 s."""
    base = (BASE_SEED + 4) if seed is None else seed
    L = 25e3 * nx
    forcing = random_modes(np.random.default_rng(base), 8, L, L, 0.1)
    scens = []
    for e in range(nreal):
        rng = np.random.default_rng(base + 1 + e)
        counts = lognormal_counts(rng, nx * nx, 6.0, 0.69, 1, 64)
        sc = _powerlaw_config(rng, nx, nx, L, counts, 5.0, 10000, (10.0, 0.0), 6 * 3600.0, False,
                              f"periodic {L/1e3:.0f} km, {nx}x{nx} cells, lognormal(6, 0.69) floes/cell")
        sc["params"]["modes"] = forcing
        scens.append(sc)
    return stack_ensemble(scens)


def scenario41(nfx: int = 480, nfy: int = 240, nx: int = 48, ny: int = 24,
               uo: tuple = (0.3, 0.0)) -> dict:
    """Sec. 4.1 of the paper (non-dimensional): domain [0,4] x [0,2], one floe at
    the centre of each of nfx x nfy fine cells, r = r_c (0.2 + 0.8 sin(pi x / 4))
    with 2 r_c the fine cell side, initial velocity = the uniform current
    (0.3, 0), no spin, periodic; coarse grid nx x ny; dt = 1e-4, dT = 0.01."""
    Lx, Ly = 4.0, 2.0
    fx, fy = Lx / nfx, Ly / nfy
    rc = 0.5 * fy
    gx, gy = np.meshgrid((np.arange(nfx) + 0.5) * fx, (np.arange(nfy) + 0.5) * fy)
    x, y = gx.ravel(), gy.ravel()
    r = rc * (0.2 + 0.8 * np.sin(0.25 * np.pi * x))
    n = x.shape[0]
    p = {"nx": nx, "ny": ny, "Lx": Lx, "Ly": Ly, "uo_x": uo[0], "uo_y": uo[1],
         "modes": np.zeros((0, 4)), "rho_o": 1.0, "Cd": 1.0, "rho_a": 0.0, "Ca": 0.0,
         "wind_x": 0.0, "wind_y": 0.0, "wind_period": 0.0, "rho_ice": 1.0, "E": 1.0e3,
         "G": 0.0, "eta": 0.0, "mu": 0.3, "h_ref": 1.0, "inertia_half": 0, "couple": 1,
         "N0": 100, "n_t": 10}
    fl = _floes(x, y, r, np.ones(n), u=np.full(n, uo[0]), v=np.full(n, uo[1]))
    return {"name": f"Sec. 4.1 uniform drift, {nfx}x{nfy} floes, {nx}x{ny} coarse", "params": p,
            "floes": fl, "dt": 1e-4, "nsteps": 2000, "meta": {}}


# Ocean drag constant of the non-dimensional Secs. 4.2-4.3 runs (the paper
# gives none): with rho_o = rho_ice = h = 1 the drag acceleration is
# Cd (u_o - v)|u_o - v|.  Reading: one length unit = 100 km (a 400 x 200 km
# domain) and 1 m thick ice with Cd = 5.5e-3, rho_o = 1026, rho_ice = 920,
# i.e. Cd rho_o / (rho_ice h) = 6.1e-3 per metre = 613 per length unit; floes
# then follow the current within a few hundredths of a time unit.
SEC4_DRAG = 613.0


def sec42_vmodes() -> np.ndarray:
    """Sec. 4.2 current u_o = (0.3 - 0.1 cos(pi x), 0): the uniform part plus
    one velocity mode (Au, Av, kx, ky, phi) = (-0.1, 0, pi, 0, 0)."""
    return np.array([[-0.1, 0.0, np.pi, 0.0, 0.0]])


def sec43_vmodes() -> np.ndarray:
    """Sec. 4.3 current u_o = (0.3 - 0.1 sin(0.1 pi x) cos(pi y),
    0.05 cos(0.1 pi x) sin(pi y)) as velocity modes: with a = 0.1 pi x and
    b = pi y, sin(a) cos(b) = (sin(a + b) + sin(a - b))/2 and cos(a) sin(b) =
    (sin(a + b) - sin(a - b))/2, and sin(t) = cos(t - pi/2)."""
    k = 0.1 * np.pi
    return np.array([[-0.05, 0.025, k, np.pi, -0.5 * np.pi],
                     [-0.05, -0.025, k, -np.pi, -0.5 * np.pi]])


def scenario4x(which: int, nfx: int = 480, nfy: int = 240, nx: int = 48, ny: int = 24) -> dict:
    """Secs. 4.2 and 4.3: the floes, domain, grid, time step, drag and
    initial state of Sec. 4.1 (both sections keep that setting; floes start
    with velocity (0.3, 0) and no spin) with the compressible currents of
    those sections (uniform part (0.3, 0) plus velocity modes)."""
    s = scenario41(nfx=nfx, nfy=nfy, nx=nx, ny=ny)
    s["params"]["vmodes"] = sec42_vmodes() if which == 2 else sec43_vmodes()
    s["params"]["Cd"] = SEC4_DRAG
    s["name"] = f"Sec. 4.{which} compressible current, {nfx}x{nfy} floes, {nx}x{ny} coarse"
    return s


def scenario44(nfx: int = 480, nfy: int = 240, nx: int = 48, ny: int = 24) -> dict:
    """Sec. 4.4: the floes, domain, grid, time step and initial state of Sec.
    4.1 driven by the uniform current u_o = (0.3, 0) into rigid walls at x = 0
    and x = 4 (periodic in y); the drag constant of Secs. 4.2-4.3 (a
    reading, see SEC4_DRAG)."""
    s = scenario41(nfx=nfx, nfy=nfy, nx=nx, ny=ny)
    s["params"]["Cd"] = SEC4_DRAG
    s["params"]["walls"] = 1
    s["name"] = f"Sec. 4.4 floes against a wall, {nfx}x{nfy} floes, {nx}x{ny} coarse"
    return s


def random_cell_floes(rng: np.random.Generator, n: int, L: float, rmin: float, rmax: float,
                      vscale: float = 0.2, wscale: float = 1e-4, overlap_ok: bool = True) -> dict:
    """n floes in one periodic square of side L with random radii, velocities
    and spins; overlaps allowed (for contact-law and search tests)."""
    x = rng.uniform(0, L, n)
    y = rng.uniform(0, L, n)
    r = rng.uniform(rmin, rmax, n)
    return {"x": x, "y": y, "theta": rng.uniform(0, 6.28, n), "u": rng.normal(0, vscale, n),
            "v": rng.normal(0, vscale, n), "omega": rng.normal(0, wscale, n), "r": r,
            "h": rng.uniform(0.5, 2.0, n)}


WORKLOADS = {f.__name__: f for f in (square_4x4, powerlaw_32x32, batched_128x128, ensemble_16x256x256)}


def mlp_init(seed: int = BASE_SEED + 3, layers=((16, 128), (128, 128), (128, 128), (128, 4))) -> dict:
    """Initial closure weights (uniform Glorot: U(-a, a), a = sqrt(6/(fan_in +
    fan_out)); zero biases), drawn here so both sides start from the same
    network.  W[out][in]."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (fi, fo) in enumerate(layers, start=1):
        a = math.sqrt(6.0 / (fi + fo))
        p[f"W{i}"] = rng.uniform(-a, a, size=(fo, fi))
        p[f"b{i}"] = np.zeros(fo)
    return p
