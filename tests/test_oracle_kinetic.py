"""Pins of the oracle's kinetic electron model (Sec. 5.2, Eq. 20-24 and the
printed f_1x / Jx update).

The checks: velocity-grid quadratures against the Maxwellian moments they
approximate; the driven single cell against brute-force geometric sums and the
Crank-Nicolson steady-state conductivity; the reduction of the kinetic update
to a Drude current when nu is constant; the discrete cold-plasma dispersion of
a plasma-filled cavity; particle-number conservation; and the paper's plasma
frequency for Table 3's density.
"""
import json
import os

import numpy as np
import pytest

from tests.physics import C0, EPS0, ME, QE, discrete_conductivity, plasma_omega, yee_omega

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
LAM0 = 0.03
OMEGA0 = 2 * np.pi * C0 / LAM0

GRIDS = [
    dict(vgrid="signed1d", nv=64),
    dict(vgrid="speed3d", nv=31),
    dict(vgrid="cart2d", nv=32, nv_perp=32),
]


def _vth(te=1.0):
    return np.sqrt(QE * te / ME)


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g["vgrid"])
def test_velocity_quadrature_moments(oracle_lib, g):
    """-sum_j w_j F0'_j is the Drude weight omega_eff^2/omega_p^2 (exact 1 for
    a Maxwellian); sum F0 dV = 1; the mean of nu is nu0; nu is proportional
    to the speed (Eq. 23, s constant)."""
    O = oracle_lib
    p = O.params(te_ev=1.0, vmax_vth=6.0, nu0=1e8, **g)
    t = O.vtables(p, 1e-12)
    assert abs(-np.sum(t["w"] * t["f0p"]) - 1.0) < 2e-6
    assert abs(np.sum(t["f0"] * t["dV"]) - 1.0) < 2e-6
    assert np.sum(t["nu"] * t["f0"] * t["dV"]) / np.sum(t["f0"] * t["dV"]) == pytest.approx(1e8, rel=1e-12)
    vth = _vth()
    if g["vgrid"] == "signed1d":
        # second moment of the 1-D Maxwellian is vth^2
        assert np.sum(t["v"] ** 2 * t["f0"] * t["dV"]) == pytest.approx(vth ** 2, rel=2e-6)
        r = t["nu"] / np.abs(t["v"])
        assert np.allclose(r, r[0], rtol=1e-13)
        assert np.allclose(t["v"], -t["v"][::-1], rtol=0, atol=0)   # exact mirror nodes
    if g["vgrid"] == "speed3d":
        assert np.sum(t["v"] ** 2 * t["f0"] * t["dV"]) == pytest.approx(3 * vth ** 2, rel=2e-6)
        r = t["nu"] / t["v"]
        assert np.allclose(r, r[0], rtol=1e-13)
    # Crank-Nicolson coefficients (Sec. 5.2): alpha = (2-dt nu)/(2+dt nu)
    dt = 1e-12
    assert np.allclose(t["alpha"] * (2 + dt * t["nu"]), 2 - dt * t["nu"], rtol=1e-14)


def test_quadrature_paper_vdim(oracle_lib):
    """The paper's v_dim = 31 speed grid (Sec. 5.2) reaches the Drude weight to 1e-6."""
    O = oracle_lib
    nv = GOLD["v_dim"]["value"]
    t = O.vtables(O.params(vgrid="speed3d", nv=nv, te_ev=1.0), 1e-12)
    assert abs(-np.sum(t["w"] * t["f0p"]) - 1.0) < 1e-6


@pytest.mark.parametrize("g", GRIDS[:2], ids=lambda g: g["vgrid"])
def test_driven_cell_geometric_sums(oracle_lib, g):
    """df_j^{m+1/2} = sum_l alpha_j^{m-l} beta_j n E^l exactly (P-f), with nu(v) != const."""
    O = oracle_lib
    dt = (LAM0 / 20) * 0.5 / C0
    p = O.params(te_ev=1.0, nu0=0.05 * OMEGA0, nu_model="nsv", **g)
    t = O.vtables(p, dt)
    n = 3e17
    M = 400
    E = np.cos(0.9 * OMEGA0 * dt * np.arange(M)) + 0.3 * np.sin(2.1 * OMEGA0 * dt * np.arange(M))
    J, df = O.kinetic_drive(p, dt, n, E)
    # brute force, independent of the recursion
    m = np.arange(M)
    pw = t["alpha"][None, :] ** (M - 1 - m)[:, None]          # alpha^{M-1-l}
    df_bf = np.sum(pw * (t["beta"][None, :] * n * E[:, None]), axis=0)
    assert np.abs(df - df_bf).max() <= 1e-12 * np.abs(df_bf).max()
    Jbf = np.array([-QE * np.sum(t["w"] * np.sum((t["alpha"][None, :] ** (k - np.arange(k + 1))[:, None]) *
                                                 (t["beta"][None, :] * n * E[: k + 1, None]), axis=0))
                    for k in range(0, M, 37)])
    assert np.abs(J[::37] - Jbf).max() <= 1e-12 * np.abs(Jbf).max()


def test_driven_cell_steady_state_conductivity(oracle_lib):
    """Late-time J of a cell driven at one frequency equals the discrete
    Crank-Nicolson conductivity (derived from the scheme, not the code), and
    that tends to the Drude conductivity eps0 wp^2/(nu - i w) as dt -> 0."""
    O = oracle_lib
    dt = (LAM0 / 40) * 0.5 / C0
    nu0 = 0.2 * OMEGA0
    p = O.params(vgrid="signed1d", nv=64, te_ev=1.0, nu0=nu0, nu_model="const")
    t = O.vtables(p, dt)
    n = 5e17
    w = 0.8 * OMEGA0
    M = 6000
    m = np.arange(M)
    E = np.cos(w * dt * m)
    J, _ = O.kinetic_drive(p, dt, n, E)
    sig = discrete_conductivity(w, dt, n, t["nu"], t["w"], t["f0p"])
    ref = np.real(sig * np.exp(-1j * w * (m + 0.5) * dt))
    tail = slice(M - 800, M)
    assert np.abs(J[tail] - ref[tail]).max() < 1e-10 * np.abs(ref).max()
    # continuous limit (Drude)
    wp2 = plasma_omega(n) ** 2
    sig_c = EPS0 * wp2 / (nu0 - 1j * w)
    small = discrete_conductivity(w, dt / 1000, n, t["nu"], t["w"], t["f0p"])
    assert abs(small - sig_c) / abs(sig_c) < 1e-5


def _slab_1d(O, **kw):
    dz = LAM0 / 40
    nz = 2000
    dens = np.zeros(nz + 1)
    n = (0.5 ** 2) * EPS0 * ME * OMEGA0 ** 2 / QE ** 2
    dens[1000:1500] = n
    base = dict(ndim=1, nz=nz, dx=dz, courant=0.5, mur=1, src_kind="gauss_sine", src_amp=1.0,
                src_fc=C0 / LAM0, src_tau=0.96 * LAM0 / C0, src_t0=4.52 * 0.96 * LAM0 / C0, src_k=100,
                vgrid="signed1d", nv=64, te_ev=1.0, nu0=0.01 * OMEGA0)
    base.update(kw)
    return O.Sim(O.params(**base), dens), n


def test_kinetic_reduces_to_drude(oracle_lib):
    """With nu constant, J obeys J^{n+1/2} = rho J^{n-1/2} + 2dt/(2+dt nu) eps0 w_eff^2 E^n (P-d)."""
    O = oracle_lib
    s, n = _slab_1d(O, nu_model="const")
    dt = s.dt
    nu = 0.01 * OMEGA0
    cells = s.slot_cells()
    q = 7
    c = cells[q]
    t = O.vtables(s.p, dt)
    weff2 = plasma_omega(n) ** 2 * (-np.sum(t["w"] * t["f0p"]))
    rho = (2 - dt * nu) / (2 + dt * nu)
    Jprev = 0.0
    worst, scale = 0.0, 0.0
    s.step(1500)
    Jprev = s.get("j")[q]
    for _ in range(1200):
        En = s.get("ex")[c]
        s.step(1)
        Jn = s.get("j")[q]
        pred = rho * Jprev + 2 * dt / (2 + dt * nu) * EPS0 * weff2 * En
        worst = max(worst, abs(Jn - pred))
        scale = max(scale, abs(Jn))
        Jprev = Jn
    assert scale > 0
    assert worst <= 1e-12 * scale


def test_cold_plasma_cavity_dispersion(oracle_lib):
    """A PEC cavity filled with collisionless plasma rings at the discrete
    cold-plasma frequency (2/dt)^2 sin^2(w dt/2) = w_eff^2 + c^2 K^2 (P-e)."""
    O = oracle_lib
    nz, dz = 60, LAM0 / 20
    n = (0.8 ** 2) * EPS0 * ME * OMEGA0 ** 2 / QE ** 2
    dens = np.full(nz + 1, n)
    s = O.Sim(O.params(ndim=1, nz=nz, dx=dz, courant=0.5, vgrid="signed1d", nv=64, te_ev=1.0,
                       nu0=0.0, nu_model="const"), dens)
    dt = s.dt
    k = 3 * np.pi / (nz * dz)
    s.set("ex", np.sin(k * np.arange(nz + 1) * dz))
    t = O.vtables(s.p, dt)
    weff = plasma_omega(n) * np.sqrt(-np.sum(t["w"] * t["f0p"]))
    w = yee_omega(dt, dz, [k], omega_eff=weff)
    M = 4000
    rec = np.zeros(M)
    for m in range(M):
        rec[m] = s.get("ex")[11]
        s.step(1)
    tt = np.arange(M) * dt
    A = np.stack([np.ones(M), np.cos(w * tt), np.sin(w * tt)], 1)
    coef, *_ = np.linalg.lstsq(A, rec, rcond=None)
    res = rec - A @ coef
    assert np.sqrt(np.mean(res ** 2)) < 1e-9 * np.sqrt(np.mean(rec ** 2))
    # the vacuum frequency does not fit: the plasma term is really there
    w_vac = yee_omega(dt, dz, [k])
    A2 = np.stack([np.ones(M), np.cos(w_vac * tt), np.sin(w_vac * tt)], 1)
    c2, *_ = np.linalg.lstsq(A2, rec, rcond=None)
    assert np.sqrt(np.mean((rec - A2 @ c2) ** 2)) > 1e-2 * np.sqrt(np.mean(rec ** 2))


def test_particle_number_linear_and_nonlinear(oracle_lib):
    """Linear mode: sum_j df_j dv vanishes per cell (odd source).  Nonlinear
    flux form: the sum is conserved while the even part develops (P-h)."""
    O = oracle_lib
    for nl in (0, 1):
        s, _ = _slab_1d(O, nonlinear=nl, src_amp=3e5)
        s.step(2600)
        d = s.diag()
        assert d["number_abs"] > 0
        assert abs(d["number"]) <= 1e-13 * d["number_abs"]
        assert d["number_max_cell"] <= 1e-13 * d["number_abs"]
        df = s.get("df")
        even = 0.5 * (df + df[:, ::-1])
        if nl == 0:
            assert np.abs(even).max() <= 1e-14 * np.abs(df).max()
        else:
            assert np.abs(even).max() > 1e-6 * np.abs(df).max()


def test_nonlinear_mode_weak_field_limit(oracle_lib):
    """The advection of delta f is second order in E: at weak fields the
    nonlinear mode's current matches the linear one to the field ratio."""
    O = oracle_lib
    js = []
    for nl in (0, 1):
        s, _ = _slab_1d(O, nonlinear=nl, src_amp=1e-3)
        s.step(2400)
        js.append(s.get("j"))
    rel = np.linalg.norm(js[1] - js[0]) / np.linalg.norm(js[0])
    assert rel < 1e-6


def test_zero_density_equals_vacuum(oracle_lib):
    """n = 0 everywhere gives exactly the pure Yee run (P-i)."""
    O = oracle_lib
    s0, _ = _slab_1d(O)
    p = s0.p
    a = O.Sim(p, np.zeros(p.nz + 1))
    b = O.Sim(p, None)
    a.step(900); b.step(900)
    assert a.nslots == 0
    assert np.array_equal(a.get("ex"), b.get("ex"))
    assert np.array_equal(a.get("hy"), b.get("hy"))


def test_paper_plasma_frequency():
    """f_p for Table 3's n = 1e19 m^-3 is the ~28.5 GHz of the S-parameter discussion (P-n)."""
    n = GOLD["plasma_density_m3"]["value"]
    fp = plasma_omega(n) / (2 * np.pi)
    g = GOLD["plasma_frequency_hz"]
    assert abs(fp - g["value"]) / g["value"] < g["rel_tol"]
    assert fp == pytest.approx(28.39e9, rel=1e-3)
