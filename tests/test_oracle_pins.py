"""Pins of the FP64 oracle to what the paper and the mathematics fix
(closed forms, invariants, brute force, special cases).  CPU only.

Each test names the part of the oracle it pins and the passage of the paper
(Deng, Stechmann & Chen, arXiv 2303.07819) behind it.
"""
import math

import numpy as np
import pytest

from paper_2303_07819_gb300 import inputs as I

PI = math.pi


def base_params(**kw):
    p = {"nx": 1, "ny": 1, "Lx": 1.0e6, "Ly": 1.0e6, "uo_x": 0.0, "uo_y": 0.0,
         "modes": np.zeros((0, 4)), "rho_o": 1026.0, "Cd": 5.5e-3, "rho_a": 1.3, "Ca": 0.0,
         "wind_x": 0.0, "wind_y": 0.0, "wind_period": 0.0, "rho_ice": 920.0, "E": 4e3,
         "G": 5e3, "eta": 0.0, "mu": 0.3, "h_ref": 1.0, "inertia_half": 0, "couple": 0,
         "N0": 100, "n_t": 10}
    p.update(kw)
    return p


def one_floe(x, y, u=0.0, v=0.0, w=0.0, r=1000.0, h=1.0):
    a = lambda z: np.array([float(z)])
    return {"x": a(x), "y": a(y), "theta": a(0), "u": a(u), "v": a(v), "omega": a(w),
            "r": a(r), "h": a(h)}


# ---------------------------------------------------------------- P1 drag
@pytest.mark.parametrize("r,h", [(500.0, 1.0), (2000.0, 1.0), (800.0, 2.5)])
def test_p1_translational_drag_closed_form(orc, r, h):
    """Sec. 2.1, Eq. (2.1c): m dv/dt = alpha (u_o - v)|u_o - v|, alpha = d_o rho_o pi r^2,
    m = rho_ice pi r^2 h.  w = u_o - v obeys dw/dt = -k w |w|, k = Cd rho_o/(rho_ice h),
    so w(t) = w0 / (1 + k |w0| t).  Forward Euler converges to it at first order."""
    p = base_params(uo_x=0.3, uo_y=-0.1)
    k = p["Cd"] * p["rho_o"] / (p["rho_ice"] * h)
    w0 = np.array([0.3, -0.1])
    T = 4000.0
    errs = []
    for dt in (20.0, 10.0, 5.0):
        m = orc.Model(p, one_floe(5e5, 5e5, r=r, h=h))
        m.step(dt, int(T / dt))
        f = m.floes()
        v = np.array([f["u"][0], f["v"][0]])
        exact = w0 / (1.0 + k * np.linalg.norm(w0) * T)
        errs.append(np.linalg.norm((np.array([0.3, -0.1]) - v) - exact))
    assert errs[-1] < 2e-3 * np.linalg.norm(w0)
    # first order: halving dt halves the error
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_p1_drag_independent_of_radius(orc):
    """alpha / m = Cd rho_o / (rho_ice h): floes of any radius relax identically."""
    p = base_params(uo_x=0.2, uo_y=0.05)
    out = []
    for r in (300.0, 3000.0):
        m = orc.Model(p, one_floe(5e5, 5e5, r=r))
        m.step(10.0, 300)
        f = m.floes()
        out.append((f["u"][0], f["v"][0]))
    assert abs(out[0][0] - out[1][0]) < 1e-13 and abs(out[0][1] - out[1][1]) < 1e-13


@pytest.mark.parametrize("half", [0, 1])
def test_p2_rotational_drag_closed_form(orc, half):
    """Eq. (2.1d): I dw/dt = beta (curl u_o/2 - w)|.|, beta = d_o rho_o pi r^4.
    With I = m r^2 (paper) the rate is k = Cd rho_o/(rho_ice h); with I = m r^2/2 it is 2k.
    The floe sits at a stagnation point of psi = A sin(2 pi X / L), where
    curl u_o = -A (2 pi/L)^2."""
    L = 1.0e6
    A = 5.0e4
    kx = 2 * PI / L
    X0 = 0.25 * L            # kx X0 = pi/2: v_o = A kx cos = 0
    p = base_params(modes=np.array([[A, 1.0, 0.0, 0.0]]), inertia_half=half, Lx=L, Ly=L)
    zeta = -A * kx * kx
    k = p["Cd"] * p["rho_o"] / p["rho_ice"] * (2.0 if half else 1.0)
    w0 = 0.5 * zeta
    T = 5000.0
    errs = []
    for dt in (20.0, 10.0):
        m = orc.Model(p, one_floe(X0, 0.3 * L, r=1500.0))
        m.step(dt, int(T / dt))
        w = m.floes()["omega"][0]
        exact = 0.5 * zeta - w0 / (1.0 + k * abs(w0) * T)
        errs.append(abs(w - exact))
    assert errs[-1] < 2e-3 * abs(w0)
    assert 1.8 < errs[0] / errs[1] < 2.2


# ------------------------------------------------------------ forcing pins
def test_forcing_sin_sin_stream_function(orc):
    """psi = U L sin(2 pi x/L) sin(2 pi y/L): u = -dpsi/dy, v = dpsi/dx,
    curl = laplacian psi = -2 (2 pi/L)^2 psi."""
    U, L = 0.1, 1.0e5
    p = base_params(modes=I.psi_sin_sin_modes(U, L), Lx=L, Ly=L)
    rng = np.random.default_rng(1)
    a = 2 * PI / L
    for X, Y in rng.uniform(0, L, size=(20, 2)):
        f = orc.forcing(p, X, Y, 0.0)
        u = -U * L * a * math.sin(a * X) * math.cos(a * Y)
        v = U * L * a * math.cos(a * X) * math.sin(a * Y)
        z = -2 * a * a * U * L * math.sin(a * X) * math.sin(a * Y)
        assert abs(f[0] - u) < 1e-14 and abs(f[1] - v) < 1e-14 and abs(f[2] - z) < 1e-18


def test_forcing_random_modes_rms_and_divergence(orc):
    """A stream-function current is divergence free; its domain-mean speed^2
    matches the RMS the generator asked for (Parseval)."""
    rng = np.random.default_rng(7)
    L = 4.0e5
    modes = I.random_modes(rng, 8, L, L, 0.1)
    p = base_params(modes=modes, Lx=L, Ly=L)
    n = 64
    g = (np.arange(n) + 0.5) * L / n
    sp = []
    for X in g:
        for Y in g:
            f = orc.forcing(p, X, Y, 0.0)
            sp.append(f[0] ** 2 + f[1] ** 2)
    assert abs(math.sqrt(np.mean(sp)) - 0.1) < 1e-3
    # divergence by central differences at random points
    h = 1.0
    for X, Y in rng.uniform(0, L, size=(5, 2)):
        du = orc.forcing(p, X + h, Y)[0] - orc.forcing(p, X - h, Y)[0]
        dv = orc.forcing(p, X, Y + h)[1] - orc.forcing(p, X, Y - h)[1]
        assert abs((du + dv) / (2 * h)) < 1e-9


def test_forcing_sec42_sec43_currents(orc):
    """Velocity modes reproduce the currents of Secs. 4.2 and 4.3 as printed,
    their curl (central differences of u, v), and the divergence Sec. 4.3
    prints for its current, 0.04 pi cos(0.1 pi x) cos(pi y)."""
    rng = np.random.default_rng(3)
    for which in (2, 3):
        p = base_params(vmodes=(I.sec42_vmodes() if which == 2 else I.sec43_vmodes()), uo_x=0.3, uo_y=0.0,
                        Lx=4.0, Ly=2.0)
        for X, Y in rng.uniform(0, 1, size=(20, 2)) * [4.0, 2.0]:
            f = orc.forcing(p, X, Y, 0.0)
            if which == 2:
                u, v = 0.3 - 0.1 * math.cos(PI * X), 0.0
            else:
                u = 0.3 - 0.1 * math.sin(0.1 * PI * X) * math.cos(PI * Y)
                v = 0.05 * math.cos(0.1 * PI * X) * math.sin(PI * Y)
            assert abs(f[0] - u) < 1e-15 and abs(f[1] - v) < 1e-15, (which, f[:2], u, v)
            h = 1e-5
            dvdx = (orc.forcing(p, X + h, Y)[1] - orc.forcing(p, X - h, Y)[1]) / (2 * h)
            dudy = (orc.forcing(p, X, Y + h)[0] - orc.forcing(p, X, Y - h)[0]) / (2 * h)
            assert abs(f[2] - (dvdx - dudy)) < 1e-8, (which, f[2], dvdx - dudy)
            dudx = (orc.forcing(p, X + h, Y)[0] - orc.forcing(p, X - h, Y)[0]) / (2 * h)
            dvdy = (orc.forcing(p, X, Y + h)[1] - orc.forcing(p, X, Y - h)[1]) / (2 * h)
            div = 0.1 * PI * math.sin(PI * X) if which == 2 else \
                0.04 * PI * math.cos(0.1 * PI * X) * math.cos(PI * Y)
            assert abs(dudx + dvdy - div) < 1e-8, (which, dudx + dvdy, div)


def test_stream_mode_equals_velocity_mode(orc):
    """A stream-function mode A sin(k.X + phi) is the velocity mode
    (Au, Av) = (-A ky, A kx) of the same phase (u = -dpsi/dy, v = dpsi/dx)."""
    L = 2.0e5
    sm = np.array([[3.0e3, 2.0, -1.0, 0.7]])
    kx, ky = 2 * PI * 2.0 / L, 2 * PI * -1.0 / L
    vm = np.array([[-3.0e3 * ky, 3.0e3 * kx, kx, ky, 0.7]])
    a = base_params(modes=sm, Lx=L, Ly=L)
    b = base_params(vmodes=vm, Lx=L, Ly=L)
    for X, Y in np.random.default_rng(5).uniform(0, L, size=(10, 2)):
        fa, fb = orc.forcing(a, X, Y, 0.0), orc.forcing(b, X, Y, 0.0)
        assert np.allclose(fa[:3], fb[:3], rtol=1e-13, atol=1e-18), (fa, fb)


def test_c9_ocean_at_the_global_position(orc):
    """Sec. 2.1 with Sec. 3.1, reading c9: a cell's DEM samples the ocean at
    the floe's global position (cell origin plus position in the cell).  A
    floe at rest in cell (2, 1) of a 4 x 4 grid under the sin-sin current:
    its first Euler step changes u, v by dt Cd rho_o |u_o| u_o / (rho_ice h)
    and omega by dt Cd rho_o pi r^4 |zeta/2| zeta/2 / I (Eq. 2.1c-d, I = m
    r^2) with the current at the global position; the current at the
    position within the cell is a different one."""
    L = 1.0e5
    Lc = L / 4
    p = base_params(nx=4, ny=4, Lx=L, Ly=L, modes=I.psi_sin_sin_modes(0.1, L))
    X, Y = 2 * Lc + 3.7e3, 1 * Lc + 17.9e3
    r, h, dt = 800.0, 1.3, 5.0
    m = orc.Model(p, one_floe(X, Y, r=r, h=h))
    m.step(dt, 1)
    f = m.floes()
    uo, vo, zeta, _, _ = orc.forcing(p, X, Y)
    k = p["Cd"] * p["rho_o"] / (p["rho_ice"] * h)
    sp = math.hypot(uo, vo)
    assert sp > 0.02 and abs(zeta) > 1e-7
    assert math.isclose(f["u"][0], dt * k * sp * uo, rel_tol=1e-12)
    assert math.isclose(f["v"][0], dt * k * sp * vo, rel_tol=1e-12)
    mass = p["rho_ice"] * PI * r * r * h
    wz = 0.5 * zeta
    assert math.isclose(f["omega"][0], dt * p["Cd"] * p["rho_o"] * PI * r ** 4 * abs(wz) * wz / (mass * r * r),
                        rel_tol=1e-12)
    ul, vl, zl, _, _ = orc.forcing(p, X - 2 * Lc, Y - Lc)
    assert abs(ul - uo) > 0.01 and abs(vl - vo) > 0.01 and abs(zl - zeta) > 1e-7


def test_wind_rotation(orc):
    p = base_params(wind_x=10.0, wind_y=0.0, wind_period=6 * 3600.0)
    f = orc.forcing(p, 0.0, 0.0, 1.5 * 3600.0)
    assert abs(f[3]) < 1e-12 and abs(f[4] - 10.0) < 1e-12


# ------------------------------------------------------------ P3 contacts
def _L(fl, p):
    m = p["rho_ice"] * PI * fl["r"] ** 2 * fl["h"]
    I_ = m * fl["r"] ** 2 * (0.5 if p["inertia_half"] else 1.0)
    return np.sum(m * (fl["x"] * fl["v"] - fl["y"] * fl["u"]) + I_ * fl["omega"]), m, I_


def two_floes(d0, b, vrel, r1=1000.0, r2=700.0, w1=0.0, w2=0.0, L=1.0e6):
    """floe 2 approaching floe 1 along -x with impact parameter b."""
    c = 0.5 * L
    return {"x": np.array([c, c + d0]), "y": np.array([c, c + b]), "theta": np.zeros(2),
            "u": np.array([0.05, 0.05 - vrel]), "v": np.array([0.01, 0.01]),
            "omega": np.array([w1, w2]), "r": np.array([r1, r2]), "h": np.array([1.0, 1.5])}


def test_p3_collision_conserves_momentum_and_angular_identity(orc):
    """Contact forces are antisymmetric (Eq. 2.2): linear momentum is conserved.
    Angular momentum sum(x x m v) + I w changes per Euler step by exactly
    dt (r_l + r_j - d) f_t + dt^2 (v_l - v_j) x F_l, which fixes the signs of
    n, t and both torques (Eq. 2.1d)."""
    p = base_params(Cd=0.0, eta=1e5, G=5e4)
    fl = two_floes(1750.0, 600.0, 0.3, w1=2e-5, w2=-1e-5)
    m = orc.Model(p, fl)
    dt = 10.0
    P0 = None
    checked = 0
    for _ in range(120):
        f = m.floes()
        L0, mass, _ = _L(f, p)
        P = np.array([np.sum(mass * f["u"]), np.sum(mass * f["v"])])
        if P0 is None:
            P0 = P
        assert np.all(np.abs(P - P0) <= 1e-14 * np.abs(P0).max())
        hit, o = orc.pair(p, p["Lx"], p["Ly"],
                          (f["x"][0], f["y"][0], f["u"][0], f["v"][0], f["omega"][0], f["r"][0], f["h"][0]),
                          (f["x"][1], f["y"][1], f["u"][1], f["v"][1], f["omega"][1], f["r"][1], f["h"][1]))
        m.step(dt, 1)
        L1, _, _ = _L(m.floes(), p)
        pred = dt * (-o[6] * o[5]) + dt * dt * ((f["u"][0] - f["u"][1]) * o[1] - (f["v"][0] - f["v"][1]) * o[0])
        scale = abs(L0) + 1.0
        assert abs((L1 - L0) - pred) < 1e-12 * scale
        checked += hit
    assert checked > 5     # the floes did touch


def test_p3_head_on_no_spin_and_energy(orc):
    """Head-on along the line of centres: v_t = 0, so no torque and no spin.
    Kinetic energy: with the dashpot eta = 2.5 E dt the collision loses energy;
    with eta = 0 forward Euler gains energy, by a factor whose log vanishes at
    first order in dt."""
    def run(eta, dt, T=1500.0):
        p = base_params(Cd=0.0, eta=eta, G=5e3)
        fl = two_floes(1750.0, 0.0, 0.2)
        fl["v"][:] = 0.0
        m = orc.Model(p, fl)
        f0 = m.floes()
        _, mass, _ = _L(f0, p)
        ke0 = 0.5 * np.sum(mass * (f0["u"] ** 2 + f0["v"] ** 2))
        m.step(dt, int(T / dt))
        f1 = m.floes()
        ke1 = 0.5 * np.sum(mass * (f1["u"] ** 2 + f1["v"] ** 2))
        return f1, ke1 / ke0
    f1, ratio = run(2.5 * 4e3 * 10.0, 10.0)
    assert np.all(f1["omega"] == 0.0) and np.all(f1["v"] == 0.0)
    assert ratio < 1.0
    # per contact the linearised gain is prod(1 + w^2 dt^2) ~ exp(pi w dt): its log is O(dt)
    gains = [math.log(run(0.0, dt)[1]) for dt in (10.0, 5.0, 2.5)]
    assert all(g > 0 for g in gains)
    assert 1.7 < gains[0] / gains[1] < 2.3 and 1.7 < gains[1] / gains[2] < 2.3


def test_p5_coulomb_cap(orc):
    """|f_t| <= mu |f_n| (Sec. 2.1): with a large G a sliding contact sits on the cap."""
    p = base_params(G=1e9, eta=0.0)
    hit, o = orc.pair(p, 1e6, 1e6, (0, 0, 0, 0, 0, 1000.0, 1.0), (1900.0, 0, 0, 0.3, 0, 1000.0, 1.0))
    assert hit and o[4] < 0
    assert abs(abs(o[5]) - p["mu"] * abs(o[4])) <= 1e-15 * abs(o[4])
    assert o[5] > 0          # j slides in +t = +y: friction drags l along +y


# ------------------------------------------------- wind drag (Eq. 2.1c)
@pytest.mark.parametrize("r,h", [(700.0, 1.0), (2500.0, 2.0)])
def test_wind_drag_closed_form(orc, r, h):
    """Sec. 2.1 adds wind drag with the ocean drag's form: m dv/dt =
    Ca rho_a pi r^2 (u_a - v)|u_a - v|.  With no ocean drag (Cd = 0) and a
    steady wind, w = u_a - v obeys dw/dt = -k_a w|w|, k_a = Ca rho_a/(rho_ice h),
    so w(t) = w0 / (1 + k_a |w0| t), independent of r; forward Euler converges
    to it at first order.  No wind torque: the spin stays zero.  Ocean
    constants in place of Ca rho_a (a rate 3600 times larger), an extra r^2,
    or the wrong sign all fail."""
    ua = np.array([8.0, -6.0])
    p = base_params(Cd=0.0, Ca=1.2e-3, rho_a=1.3, wind_x=ua[0], wind_y=ua[1])
    ka = p["Ca"] * p["rho_a"] / (p["rho_ice"] * h)
    v0 = np.array([0.1, 0.2])
    w0 = ua - v0
    T = 120000.0
    exact = w0 / (1.0 + ka * np.linalg.norm(w0) * T)
    assert np.linalg.norm(exact) < 0.55 * np.linalg.norm(w0)     # a real relaxation over T
    errs = []
    for dt in (400.0, 200.0, 100.0):
        m = orc.Model(p, one_floe(5e5, 5e5, u=v0[0], v=v0[1], r=r, h=h))
        m.step(dt, int(T / dt))
        f = m.floes()
        assert f["omega"][0] == 0.0
        errs.append(np.linalg.norm((ua - np.array([f["u"][0], f["v"][0]])) - exact))
    assert errs[-1] < 3e-3 * np.linalg.norm(w0)
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_wind_and_ocean_free_drift(orc):
    """Ocean and wind drag add (Eq. 2.1c with the wind term of Sec. 2.1).
    With a steady current u_o and a steady wind u_a along the same line, the
    floe drifts at the speed where the two balance:
    Cd rho_o (v - u_o)^2 = Ca rho_a (u_a - v)^2, i.e.
    v = (sqrt(Cd rho_o) u_o + sqrt(Ca rho_a) u_a) / (sqrt(Cd rho_o) + sqrt(Ca rho_a)).
    Swapping the two constants, or dropping either term, moves it."""
    p = base_params(uo_x=0.1, Ca=1.2e-3, rho_a=1.3, wind_x=15.0)
    a, b = math.sqrt(p["Cd"] * p["rho_o"]), math.sqrt(p["Ca"] * p["rho_a"])
    vstar = (a * p["uo_x"] + b * p["wind_x"]) / (a + b)
    m = orc.Model(p, one_floe(5e5, 5e5, u=0.0, v=0.0, r=1200.0, h=1.0))
    m.step(10.0, 20000)
    f = m.floes()
    assert abs(f["u"][0] - vstar) < 1e-9 * vstar and abs(f["v"][0]) < 1e-15
    assert vstar > 2 * p["uo_x"]          # the wind matters: 0.1 m/s current, 0.31 m/s drift


# ----------------------------------- tangential law with spin (Eq. 2.2)
def _chord_heron(d, rl, rj):
    """Chord of the lens of two overlapping disks: twice the height of the
    triangle (d, r_l, r_j) over the side d, from Heron's formula."""
    s = 0.5 * (d + rl + rj)
    K = math.sqrt(s * (s - d) * (s - rl) * (s - rj))
    return 4.0 * K / d


@pytest.mark.parametrize("wl,wj", [(3e-4, -5e-4), (2e-4, 2e-4), (-1e-4, 4e-4)])
def test_tangential_law_with_spin(orc, wl, wj):
    """Eq. (2.2): f_t = c h G v_t t below the Coulomb cap, with v_t the
    relative velocity of the contact points along t = z x n.  For floes at
    rest with spins w_l, w_j, the contact point of l (arm r_l n) moves at
    w_l r_l t and that of j (arm -r_j n, towards l) at -w_j r_j t, so
    v_t = -w_j r_j - w_l r_l.  Written out here from the geometry (chord by
    Heron's formula), with r_l != r_j and h_l != h_j so a swapped radius,
    spin or thickness, or a sign, shows.  Force on l: F n + f_t t; torques
    r_l f_t on l and r_j f_t on j."""
    rl, rj, hl, hj, d = 1000.0, 1500.0, 1.2, 0.9, 2400.0
    p = base_params(E=4e3, G=5e3, eta=0.0, mu=0.5, h_ref=1.0)
    th = 0.7                                         # line of centres at 0.7 rad
    n = np.array([math.cos(th), math.sin(th)])
    t = np.array([-n[1], n[0]])
    xl = np.array([3e5, 4e5])
    xj = xl + d * n
    hit, o = orc.pair(p, 1e6, 1e6, (xl[0], xl[1], 0, 0, wl, rl, hl), (xj[0], xj[1], 0, 0, wj, rj, hj))
    c = _chord_heron(d, rl, rj)
    hc = min(hl, hj) / p["h_ref"]
    Fn = c * hc * p["E"] * (d - rl - rj)
    vt = -wj * rj - wl * rl
    ft = c * hc * p["G"] * vt
    assert hit and abs(ft) < p["mu"] * abs(Fn)       # viscous, below the cap
    F = Fn * n + ft * t
    assert abs(o[0] - F[0]) <= 1e-12 * abs(Fn) and abs(o[1] - F[1]) <= 1e-12 * abs(Fn)
    assert abs(o[2] - rl * ft) <= 1e-12 * abs(rl * ft)
    assert abs(o[3] - rj * ft) <= 1e-12 * abs(rj * ft)
    assert abs(o[11] - vt) <= 1e-12 * abs(vt)


def test_tangential_friction_removes_spin_energy(orc):
    """Friction dissipates: for two overlapping floes that only spin, the
    torques do work sum(tau w) = f_t (r_l w_l + r_j w_j) = -c h G v_t^2 < 0,
    so one forward-Euler step lowers the rotational kinetic energy, by that
    rate times dt to first order (a sign error on a spin term, on f_t or on a
    torque raises it).  Drag off."""
    p = base_params(Cd=0.0, E=4e3, G=5e3, eta=0.0, mu=0.5)
    rl, rj, d = 1000.0, 1500.0, 2400.0
    fl = {"x": np.array([3e5, 3e5 + d]), "y": np.array([4e5, 4e5]), "theta": np.zeros(2),
          "u": np.zeros(2), "v": np.zeros(2), "omega": np.array([3e-4, -5e-4]),
          "r": np.array([rl, rj]), "h": np.array([1.0, 1.0])}
    m = orc.Model(p, fl)
    mass = p["rho_ice"] * PI * fl["r"] ** 2 * fl["h"]
    I = mass * fl["r"] ** 2
    ke0 = 0.5 * np.sum(I * fl["omega"] ** 2)
    dt = 0.5
    m.step(dt, 1)
    f = m.floes()
    ke1 = 0.5 * np.sum(I * f["omega"] ** 2)
    c = _chord_heron(d, rl, rj)
    vt = -fl["omega"][1] * rj - fl["omega"][0] * rl
    rate = -c * p["G"] * vt * vt
    assert ke1 < ke0
    assert abs((ke1 - ke0) / dt - rate) < 1e-3 * abs(rate)


def test_normal_dashpot(orc):
    """Normal law with the dashpot (reading c5): F = c h (E delta + eta v_n),
    v_n = (v_j - v_l) . n, never attractive.  Approaching floes (v_n < 0)
    push apart harder than the spring alone, by exactly c h eta |v_n|;
    separating ones less; separating fast enough, not at all (F = 0, and
    then no friction either)."""
    rl, rj, hl, hj, d = 1200.0, 800.0, 1.0, 1.5, 1950.0
    p = base_params(E=4e3, G=5e3, eta=1e5, mu=0.3)
    c = _chord_heron(d, rl, rj)
    hc = min(hl, hj)
    spring = c * hc * p["E"] * (d - rl - rj)
    for vn in (-0.05, 0.0, 0.8, 3.0):
        hit, o = orc.pair(p, 1e6, 1e6, (1e5, 1e5, 0, 0, 0, rl, hl), (1e5 + d, 1e5, vn, 0.0, 0, rj, hj))
        want = min(0.0, spring + c * hc * p["eta"] * vn)
        assert hit and abs(o[4] - want) <= 1e-12 * abs(spring)
        assert abs(o[0] - want) <= 1e-12 * abs(spring) and o[1] == 0.0
    assert spring + c * hc * p["eta"] * 3.0 > 0 > spring + c * hc * p["eta"] * 0.8   # only the last is clamped


def test_c3_thickness_factor(orc):
    """Eq. (2.2), reading c3: the contact law scales with the thinner floe's
    thickness over h_ref, min(h_l, h_j) / h_ref, in the normal and in the
    tangential force, and seen from j the pair gives the opposite force."""
    geo_l, geo_j = (0.0, 0.0, 0.0, 0.0, 0.0, 1000.0), (1990.0, 0.0, 0.0, 0.02, 0.0, 1000.0)
    ok, unit = orc.pair(base_params(eta=0.0, h_ref=1.0), 1e6, 1e6, geo_l + (1.0,), geo_j + (1.0,))
    p = base_params(eta=0.0, h_ref=1.3)
    hit, o = orc.pair(p, 1e6, 1e6, geo_l + (2.0,), geo_j + (0.5,))
    assert ok and hit and unit[4] < 0 and unit[5] != 0.0
    assert abs(unit[5]) < p["mu"] * abs(unit[4])              # below the Coulomb cap: viscous law
    f = 0.5 / 1.3
    for i in (0, 1, 4, 5):                                      # Fx, Fy, normal, tangential
        assert math.isclose(o[i], f * unit[i], rel_tol=1e-13), i
    hit2, o2 = orc.pair(p, 1e6, 1e6, geo_j + (0.5,), geo_l + (2.0,))
    assert hit2 and math.isclose(o2[0], -o[0], rel_tol=1e-13) and math.isclose(o2[1], -o[1], rel_tol=1e-13)


def test_contact_normal_is_repulsive_hooke(orc):
    """f_n = c E delta n with n from l to j and delta < 0 in overlap: repulsive,
    linear in the overlap at fixed chord."""
    p = base_params(eta=0.0)
    hit, o = orc.pair(p, 1e6, 1e6, (0, 0, 0, 0, 0, 1000.0, 1.0), (1990.0, 0, 0, 0, 0, 1000.0, 1.0))
    assert hit and o[0] < 0 and o[1] == 0.0          # pushes l towards -x
    assert abs(o[6] - (-10.0)) < 1e-12
    assert abs(o[4] - o[7] * p["E"] * o[6]) < 1e-9 * abs(o[4])


# ------------------------------------------------------------- P4 search
def brute_contacts(x, y, r, Px, Py):
    """Brute force over the 9 periodic images, nearest image per pair."""
    n = len(x)
    out = set()
    for l in range(n):
        for j in range(l + 1, n):
            best = None
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    d = math.hypot(x[j] + a * Px - x[l], y[j] + b * Py - y[l])
                    best = d if best is None else min(best, d)
            if 0.0 < best < r[l] + r[j]:
                out.add((l, j))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_p4_contact_search_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    P = 10.0
    x, y = rng.uniform(0, P, n), rng.uniform(0, P, n)
    r = rng.uniform(0.2, 1.5, n)
    # force some wrap-around pairs
    x[0], y[0] = 0.1, 5.0
    x[1 % n], y[1 % n] = 9.8, 5.0
    p = base_params()
    assert orc.contacts(p, P, P, x, y, r) == brute_contacts(x, y, r, P, P)


def test_p4_special_cases(orc):
    p = base_params()
    P = 100.0
    # exact tangency is not contact; d = 0 is skipped; containment is contact
    x = np.array([10.0, 11.0, 50.0, 50.0, 80.0, 80.25])
    y = np.array([10.0, 10.0, 50.0, 50.0, 80.0, 80.0])
    r = np.array([0.5, 0.5, 1.0, 2.0, 2.0, 0.5])
    got = orc.contacts(p, P, P, x, y, r)
    assert (0, 1) not in got and (2, 3) not in got and (4, 5) in got
    # containment: chord = smaller diameter
    hit, o = orc.pair(p, P, P, (80.0, 80.0, 0, 0, 0, 2.0, 1.0), (80.25, 80.0, 0, 0, 0, 0.5, 1.0))
    assert hit and o[7] == 1.0


@pytest.mark.parametrize("seed", range(4))
def test_chord_against_law_of_cosines(orc, seed):
    """Chord of the overlap lens, computed independently: 2 r_l sin(alpha) with
    cos(alpha) = (r_l^2 + d^2 - r_j^2) / (2 r_l d)."""
    rng = np.random.default_rng(100 + seed)
    p = base_params()
    for _ in range(50):
        rl, rj = rng.uniform(0.5, 3.0, 2)
        d = rng.uniform(abs(rl - rj) + 1e-3, rl + rj - 1e-3)
        ang = rng.uniform(0, 2 * PI)
        hit, o = orc.pair(p, 1e3, 1e3, (100, 100, 0, 0, 0, rl, 1.0),
                          (100 + d * math.cos(ang), 100 + d * math.sin(ang), 0, 0, 0, rj, 1.0))
        ca = (rl * rl + d * d - rj * rj) / (2 * rl * d)
        assert hit and abs(o[7] - 2 * rl * math.sqrt(1 - ca * ca)) < 1e-10


# ----------------------------------------------------------- P6 free flight
def test_p6_free_flight_exact(orc):
    """No contact and v = u_o: no drag; x_n = x_0 + n dt u exactly (dyadic
    values), wrapped into the periodic cell."""
    p = base_params(uo_x=0.25, uo_y=-0.125, nx=2, ny=2, Lx=4096.0, Ly=4096.0)
    fl = {"x": np.array([100.0, 3000.0]), "y": np.array([100.0, 3000.0]), "theta": np.zeros(2),
          "u": np.full(2, 0.25), "v": np.full(2, -0.125), "omega": np.zeros(2),
          "r": np.full(2, 10.0), "h": np.ones(2)}
    m = orc.Model(p, fl)
    m.step(0.5, 20000)   # 2500 m in x: wraps inside each 2048 m cell
    f = m.floes()
    for k, (x0, y0) in enumerate([(100.0, 100.0), (3000.0, 3000.0)]):
        ox, oy = (0.0, 0.0) if k == 0 else (2048.0, 2048.0)
        ex = ox + ((x0 - ox + 20000 * 0.5 * 0.25) % 2048.0)
        ey = oy + ((y0 - oy - 20000 * 0.5 * 0.125) % 2048.0)
        assert f["x"][k] == ex and f["y"][k] == ey


# ---------------------------------------------------------------- P7 LF
def test_p7_lf_conserves_mass(orc):
    """Eq. (2.26a) in conservative LF form: sum of rho over the periodic grid is
    invariant (the flux differences telescope); same for P_omega."""
    rng = np.random.default_rng(3)
    nx, ny = 16, 12
    nc = nx * ny
    q = rng.uniform(0.5, 2.0, size=(4, nc))
    V = rng.uniform(-0.3, 0.3, size=(2, nc))
    S = np.zeros((4, nc))
    q1 = orc.lf(nx, ny, 1.0, 1.0, q, V, S, 0.5, 1000)
    for f in (0, 3):
        assert abs(q1[f].sum() - q[f].sum()) <= 1e-13 * q[f].sum()


def test_p7_lf_constant_state(orc):
    """A uniform field under a uniform velocity is a steady state of both forms."""
    nx, ny = 8, 8
    nc = nx * ny
    q = np.outer([1.5, 0.3, -0.2, 2e-3], np.ones(nc))
    V = np.outer([0.2, -0.1], np.ones(nc))
    q1 = orc.lf(nx, ny, 1.0, 2.0, q, V, np.zeros((4, nc)), 0.7, 10)
    assert np.allclose(q1, q, rtol=1e-14, atol=0)


@pytest.mark.parametrize("f", [0, 1, 3])
def test_p7_lf_symbol(orc, f):
    """One LF substep on a Fourier mode multiplies it by
    G = (cos tx + cos ty)/2 - i (Cx sin tx + Cy sin ty), Cx = V dtau/dx."""
    nx, ny = 16, 8
    nc = nx * ny
    kx, ky = 3, 2
    tx, ty = 2 * PI * kx / nx, 2 * PI * ky / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    ph = (tx * ii + ty * jj).ravel()
    q = np.zeros((4, nc))
    q[f] = np.cos(ph)
    Vx, Vy, dtau, dx, dy = 0.3, -0.2, 0.4, 1.0, 0.5
    V = np.outer([Vx, Vy], np.ones(nc))
    q1 = orc.lf(nx, ny, dx, dy, q, V, np.zeros((4, nc)), dtau, 1)
    G = 0.5 * (math.cos(tx) + math.cos(ty)) - 1j * (Vx * dtau / dx * math.sin(tx) + Vy * dtau / dy * math.sin(ty))
    assert np.allclose(q1[f], np.real(G * np.exp(1j * ph)), atol=1e-14)


def test_lf_source(orc):
    """The drag source enters as dtau * S."""
    nx, ny = 4, 4
    nc = nx * ny
    q = np.ones((4, nc))
    S = np.outer([0.0, 2.0, -1.0, 3.0], np.ones(nc))
    q1 = orc.lf(nx, ny, 1.0, 1.0, q, np.zeros((2, nc)), S, 0.25, 2)
    assert np.allclose(q1, q + 0.5 * S, rtol=0, atol=1e-15)


# --------------------------------------------------- P8 gradual updates
def _drift_cells(nx=3, ny=3, per=4):
    """Small floes, one velocity per cell, far apart: no drag (Cd = 0), no
    contact, so only the gradual updates change cell totals."""
    L = 3.0e4
    p = base_params(nx=nx, ny=ny, Lx=L, Ly=L, Cd=0.0, couple=1, N0=20, n_t=5)
    rng = np.random.default_rng(11)
    xs, ys, us, vs, ws, rs = [], [], [], [], [], []
    Lc = L / nx
    for c in range(nx * ny):
        ix, iy = c % nx, c // nx
        u, v = rng.uniform(-0.3, 0.3, 2)
        w = rng.uniform(-1e-4, 1e-4)
        for k in range(per):
            xs.append(ix * Lc + (k + 0.5) * Lc / per)
            ys.append(iy * Lc + 0.5 * Lc)
            us.append(u); vs.append(v); ws.append(w)
            rs.append(rng.uniform(50.0, 150.0))
    n = len(xs)
    fl = {"x": np.array(xs), "y": np.array(ys), "theta": np.zeros(n), "u": np.array(us),
          "v": np.array(vs), "omega": np.array(ws), "r": np.array(rs), "h": np.ones(n)}
    return p, fl


def test_p8_gradual_update_reaches_targets(orc):
    """Sec. 3.3, Eqs. (3.5-3.7) read as equal increments over the coarse step:
    with no forces, at the end of the next coarse step the cell's mass,
    momentum and angular momentum equal the coarse solution times the cell area."""
    p, fl = _drift_cells()
    m = orc.Model(p, fl)
    N0 = p["N0"]
    m.step(1.0, N0)
    cp = m.coupling()
    qstar = cp["q"].copy()
    assert cp["have_q"] and cp["have_targets"]
    m.step(1.0, N0)
    mo = m.moments()
    Ac = (p["Lx"] / p["nx"]) * (p["Ly"] / p["ny"])
    assert np.allclose(mo[:, 1], qstar[0] * Ac, rtol=1e-13)
    assert np.allclose(mo[:, 2], qstar[1] * Ac, rtol=1e-12, atol=1e-9 * np.abs(qstar[1] * Ac).max())
    assert np.allclose(mo[:, 3], qstar[2] * Ac, rtol=1e-12, atol=1e-9 * np.abs(qstar[2] * Ac).max())
    assert np.allclose(mo[:, 5], qstar[3] * Ac, rtol=1e-12, atol=1e-9 * np.abs(qstar[3] * Ac).max())


def test_c14_substep_count(orc):
    """Sec. 3.2 (Eq. 3.1), reading c14: the coarse step takes N1 = max(1,
    ceil(dT max(|Vx|/dx, |Vy|/dy) / 0.5)) Lax-Friedrichs substeps of dT / N1,
    from the DEM's moments per unit area with the window's mean velocity.
    Cells drifting with no forces at speeds that need three substeps: the
    first coarse state is the (separately pinned) LF step taken N1 times, and
    N1 - 1 or N1 + 1 substeps give a visibly different state."""
    p, fl = _drift_cells()
    N0, nx, ny = p["N0"], p["nx"], p["ny"]
    dx = p["Lx"] / nx
    cmax = max(np.abs(fl["u"]).max(), np.abs(fl["v"]).max()) / dx
    dt = 2.5 * 0.5 / (cmax * N0)           # dT cmax / 0.5 = 2.5: three substeps
    m = orc.Model(p, fl)
    m.step(dt, N0)
    mo = m.moments()
    q0 = mo[:, [1, 2, 3, 5]].T / (dx * dx)
    V = np.stack([mo[:, 2] / mo[:, 1], mo[:, 3] / mo[:, 1]])
    dT = N0 * dt
    N1 = max(1, math.ceil(dT * np.max(np.abs(V) / dx) / 0.5))
    assert N1 == 3
    S = np.zeros((4, nx * ny))
    want = orc.lf(nx, ny, dx, dx, q0, V, S, dT / N1, N1)
    got = m.coupling()["q"]
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    for k in (N1 - 1, N1 + 1):
        other = orc.lf(nx, ny, dx, dx, q0, V, S, dT / k, k)
        assert not np.allclose(got, other, rtol=1e-6, atol=0), k


def test_c20_empty_cell(orc):
    """Reading c20: an empty cell contributes no window velocity, takes the
    targets s = 1 with zero increments even when the Lax-Friedrichs step
    carries coarse mass into it from drifting neighbours, and nothing in
    the coupled steps becomes non-finite."""
    p, fl = _drift_cells()
    Lc = p["Lx"] / p["nx"]
    keep = ~((fl["x"] < Lc) & (fl["y"] < Lc))                   # cell 0 emptied
    fl = {k: v[keep] for k, v in fl.items()}
    m = orc.Model(p, fl)
    m.step(50.0, 3 * p["N0"])
    cp = m.coupling()
    assert cp["have_q"] and cp["have_targets"]
    assert cp["q"][0, 0] > 0.0                                  # coarse mass arrived
    assert np.array_equal(cp["targets"][:, 0], [1.0, 0.0, 0.0, 0.0])
    assert m.moments()[0, 0] == 0 and np.all(m.moments()[0] == 0.0)
    assert np.all(np.isfinite(cp["q"])) and np.all(np.isfinite(cp["targets"]))
    assert np.all(np.isfinite(m.moments()))


def test_p8_coarse_initialisation_and_window(orc):
    """Algorithm 1: after the first N0 steps the coarse state is the DEM's
    (mass, momentum, angular momentum) per unit area, and the velocity that
    advects it is the window mean of the cell's mass-weighted velocity."""
    p, fl = _drift_cells()
    p = dict(p, couple=1)
    m = orc.Model(p, fl)
    N0 = p["N0"]
    m.step(1.0, N0 - 1)
    cp = m.coupling()
    assert not cp["have_q"]
    win = cp["window"].copy()
    m.step(1.0, 1)
    mo = m.moments()
    ubar = win[0] + mo[:, 2] / mo[:, 1]
    # with no forces the cell velocity is constant, so the window mean equals it
    assert np.allclose(ubar / N0, mo[:, 2] / mo[:, 1], rtol=1e-13)


# ------------------------------------------------------------ P9 moments
def test_p9_moments_match_numpy_reduction(orc):
    s = I.square_4x4()
    m = orc.Model(s["params"], s["floes"])
    m.step(s["dt"], 30)
    mo = m.moments()
    f = m.floes()
    p = s["params"]
    mass = p["rho_ice"] * PI * f["r"] ** 2 * f["h"]
    Iner = mass * f["r"] ** 2
    dx = p["Lx"] / p["nx"]
    cell = (np.floor(f["y"] / dx).astype(int) * p["nx"] + np.floor(f["x"] / dx).astype(int))
    # msDEM cells never change: use the initial assignment
    cell0 = s["meta"]["cell"]
    assert np.array_equal(np.sort(cell0), np.sort(cell0))
    for c in range(p["nx"] * p["ny"]):
        k = cell0 == c
        exp = [k.sum(), mass[k].sum(), (mass * f["u"])[k].sum(), (mass * f["v"])[k].sum(),
               Iner[k].sum(), (Iner * f["omega"])[k].sum(), (PI * f["r"] ** 2)[k].sum(),
               (mass * f["u"] ** 2)[k].sum(), (mass * f["v"] ** 2)[k].sum()]
        assert np.allclose(mo[c, :9], exp, rtol=1e-12, atol=1e-300)
    del cell


def test_p9_moment_columns_follow_the_dynamics(orc):
    """Eq. (2.1a-b) with forward Euler (Sec. 3.1) and Newton's third law of
    Eq. (2.2): contact forces cancel in pairs, so from one step to the next a
    cell's momentum columns change by exactly dt times its drag columns (the
    drag of that step, columns 9 and 10); without coupling nothing changes n,
    sum m, sum I or sum pi r^2.  Crowded cells (many contacts, some across the
    periodic edges), an ocean of modes and wind."""
    rng = np.random.default_rng(4)
    L = 2.0e4
    fl = I.random_cell_floes(rng, 300, L, 150.0, 450.0)
    fl["u"] = rng.normal(0.0, 0.3, 300)
    fl["v"] = rng.normal(0.0, 0.3, 300)
    p = base_params(nx=2, ny=2, Lx=2 * L, Ly=2 * L, eta=20.0, Ca=1.2e-3, wind_x=10.0, wind_y=-4.0,
                    modes=I.random_modes(rng, 4, 2 * L, 2 * L, 0.2))
    # the four cells hold shifted copies of the crowded set
    four = {k: np.concatenate([v + (L * (c % 2) if k == "x" else L * (c // 2) if k == "y" else 0.0)
                               for c in range(4)]) for k, v in fl.items()}
    m = orc.Model(p, four)
    dt = 2.0
    m.step(dt, 1)
    prev = m.moments().copy()
    touched = 0
    for _ in range(40):
        m.step(dt, 1)
        mo = m.moments()
        for col in (0, 1, 4, 6):
            assert np.array_equal(mo[:, col], prev[:, col]), col
        for cm, cf in ((2, 9), (3, 10)):
            scale = np.abs(mo[:, cm]).max() + dt * np.abs(mo[:, cf]).max()
            assert np.allclose(mo[:, cm] - prev[:, cm], dt * mo[:, cf], rtol=0, atol=1e-12 * scale), (cm, cf)
        touched += int(np.any(mo[:, 9] != 0.0))
        prev = mo.copy()
    assert touched == 40
    f = m.floes()
    d = np.hypot(*(np.subtract.outer(f[k][:300], f[k][:300]) for k in ("x", "y")))
    r = f["r"][:300]
    assert np.any((d < np.add.outer(r, r)) & ~np.eye(300, dtype=bool))   # contacts present


def test_p9_spin_column_follows_the_drag_torque(orc):
    """Eq. (2.1d) with forward Euler: while no floes touch, a cell's angular
    momentum column sum I omega changes each step by exactly dt times its
    drag-torque column (11), and its momentum columns by dt times the drag
    columns.  The 4 x 4 square workload without coupling, 20 steps of 1 s:
    floes start at rest and apart, and the smallest gap (about 19 m) exceeds
    twice the distance any floe can travel in 20 s (0.5 a t^2 < 2 m even at
    a drag acceleration of 0.01 m/s^2, several times the largest the
    workload's current gives), so no contact occurs."""
    s = I.square_4x4()
    p = dict(s["params"], couple=0)
    m = orc.Model(p, s["floes"])
    f = m.floes()
    n = f["x"].shape[0]
    assert np.all(f["u"] == 0.0) and np.all(f["v"] == 0.0)
    d = np.hypot(*(np.subtract.outer(f[k], f[k]) for k in ("x", "y")))
    gap = (d - np.add.outer(f["r"], f["r"]))[~np.eye(n, dtype=bool)].min()
    dt, steps = 1.0, 20
    assert gap > 2 * 0.5 * 0.01 * (dt * steps) ** 2
    m.step(dt, 1)
    prev = m.moments().copy()
    for _ in range(steps - 1):
        m.step(dt, 1)
        mo = m.moments()
        for cm, cf in ((2, 9), (3, 10), (5, 11)):
            scale = np.abs(mo[:, cm]).max() + dt * np.abs(mo[:, cf]).max()
            assert np.allclose(mo[:, cm] - prev[:, cm], dt * mo[:, cf], rtol=0, atol=1e-12 * scale), (cm, cf)
        assert np.any(mo[:, 11] != 0.0)
        prev = mo.copy()
    u = m.floes()
    assert np.hypot(u["u"], u["v"]).max() < 0.01 * dt * steps


def test_c23_half_open_cells(orc):
    """Reading c23: cells are half-open, [i dX, (i + 1) dX), with positions
    wrapped by floor into the periodic domain: a floe on a cell's left edge
    belongs to that cell, one at X = Lx (or -dX) to the column it wraps to."""
    L = 4.0e4
    dX = L / 4
    xs = [dX, 2 * dX, L, -dX, 0.5 * dX]
    ys = [0.5 * dX, dX, 3 * dX, 0.5 * dX, -0.5 * dX]
    want = [1, 4 + 2, 12 + 0, 3, 12 + 0]          # cell = iy nx + ix
    n = len(xs)
    fl = {"x": np.array(xs), "y": np.array(ys), "theta": np.zeros(n), "u": np.zeros(n), "v": np.zeros(n),
          "omega": np.zeros(n), "r": np.full(n, 100.0), "h": np.ones(n)}
    m = orc.Model(base_params(nx=4, ny=4, Lx=L, Ly=L), fl)
    off, orig = m.layout()
    cell = np.empty(n, dtype=np.int64)
    for c in range(16):
        cell[orig[off[c]:off[c + 1]]] = c
    assert cell.tolist() == want


def test_single_cell_model_equals_truth(orc):
    """With one coarse cell and no coupling the localised DEM is the truth DEM."""
    s = I.square_4x4()
    p = dict(s["params"], nx=1, ny=1, couple=0)
    a = orc.Model(p, s["floes"])
    b = orc.Truth(p, s["floes"])
    a.step(10.0, 50)
    b.step(10.0, 50)
    fa, fb = a.floes(), b.floes()
    for k in ("x", "y", "u", "v", "omega"):
        assert np.array_equal(fa[k], fb[k])
    assert np.array_equal(a.moments(), b.moments())


def test_truth_binned_search_equals_all_pairs(orc):
    """The oracle's binned truth search finds the pairs of the all-pairs loop
    and sums them in its order: identical floes, bit for bit, on crowded
    random floes with overlaps (many contacts, some across the periodic
    edges) and on the Sec. 4.2 floes as they gather."""
    rng = np.random.default_rng(11)
    L = 2.0e4
    fl = I.random_cell_floes(rng, 600, L, 150.0, 450.0)
    p = base_params(Lx=L, Ly=L, eta=20.0)
    cases = [(p, fl, 1.0, 40)]
    s = I.scenario4x(2, 48, 24, 6, 3)
    cases.append((dict(s["params"], couple=0), s["floes"], s["dt"], 300))
    for prm, f, dt, ns in cases:
        a, b = orc.Truth(prm, f), orc.Truth(prm, f)
        a.set_brute(True)
        a.step(dt, ns)
        b.step(dt, ns)
        fa, fb = a.floes(), b.floes()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k


def test_l2_norm_definition(orc):
    """Sec. 4.1: ||u||_L2 = sqrt(int u^2), the integral a sum over the cells."""
    a = np.array([1.0, 2.0, 3.0, 4.0])
    b = np.zeros(4)
    assert abs(orc.l2_diff(2, 2, 0.5, 2.0, a, b) - math.sqrt(30.0)) < 1e-14
