"""Pins of the oracle's isotropic F0 models and tabulated cross-section.

Sec. 5.2 takes F0 as a Druyvesteyn distribution (no formula printed) and the
elastic collision frequency as nu = N s(v) v with a measured s(v) (Eq. 23).
The oracle's Druyvesteyn F0 is A exp(-(eps/eps0)^2) with mean energy
(3/2) e Te; on each velocity grid it enters as the distribution (3-D, or its
1-D / 2-D marginal) and its v_par derivative.  Checks:
  * normalisation, <v_par^2> = v_th^2 (mean energy 3/2 e Te) and the Drude
    weight -sum w F0' = 1 (integration by parts, any isotropic F0), per grid;
  * the shape: <v^4>/<v^2>^2 = Gamma(3/4) Gamma(7/4) / Gamma(5/4)^2 in 3-D,
    9/5 of that for one Cartesian component (5/3 and 3 for the Maxwellian);
  * F0' against finite differences of F0 on fine grids (the two come from
    separate formulas: erfc vs -2 pi u F0 on the signed grid, two separate
    quadratures on the Cartesian grid);
  * the s(v) table: a constant table reproduces N s |v|, s = c/v at the node
    speeds gives constant nu, a linear s(v) is interpolated exactly, the ends
    are held constant; and with constant nu the kinetic current of a
    Druyvesteyn plasma obeys the same Drude recursion as a Maxwellian one."""
import math

import numpy as np
import pytest

from tests.physics import EPS0, ME, QE, plasma_omega

DT = 1.0e-12
GRIDS = [dict(vgrid="signed1d", nv=256), dict(vgrid="cart2d", nv=96, nv_perp=96), dict(vgrid="speed3d", nv=256)]
KURT3 = math.gamma(0.75) * math.gamma(1.75) / math.gamma(1.25) ** 2


def _tables(O, **kw):
    p = O.params(te_ev=2.0, vmax_vth=8.0, nu0=1e9, **kw)
    return O.vtables(p, DT), math.sqrt(QE * 2.0 / ME)


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g["vgrid"])
@pytest.mark.parametrize("f0", ["maxwell", "druyvesteyn"])
def test_f0_moments_and_drude_weight(oracle_lib, g, f0):
    t, vth = _tables(oracle_lib, f0_model=f0, **g)
    m0 = np.sum(t["f0"] * t["dV"])
    m2 = np.sum(t["v"] ** 2 * t["f0"] * t["dV"])
    m4 = np.sum(t["v"] ** 4 * t["f0"] * t["dV"])
    drude = -np.sum(t["w"] * t["f0p"])
    tol = 1e-12 if f0 == "druyvesteyn" else 1e-11
    assert abs(m0 - 1) <= tol and abs(drude - 1) <= tol
    if g["vgrid"] == "speed3d":       # v is the speed here
        assert abs(m2 / (3 * vth ** 2) - 1) <= tol
        want = KURT3 if f0 == "druyvesteyn" else 5.0 / 3.0
    else:                             # v is v_par
        assert abs(m2 / vth ** 2 - 1) <= tol
        want = 9.0 / 5.0 * KURT3 if f0 == "druyvesteyn" else 3.0
    assert abs(m4 / m2 ** 2 / want - 1) <= 1e-9


@pytest.mark.parametrize("g", [dict(vgrid="signed1d", nv=4096), dict(vgrid="cart2d", nv=2048, nv_perp=3),
                               dict(vgrid="speed3d", nv=4096)], ids=lambda g: g["vgrid"])
def test_druyvesteyn_derivative_matches_finite_differences(oracle_lib, g):
    t, vth = _tables(oracle_lib, f0_model="druyvesteyn", **g)
    nperp = g.get("nv_perp", 1)
    v = t["v"].reshape(-1, nperp)[:, 0]
    f = t["f0"].reshape(-1, nperp)[:, 1 if nperp > 1 else 0]
    fp = t["f0p"].reshape(-1, nperp)[:, 1 if nperp > 1 else 0]
    fd = (f[2:] - f[:-2]) / (v[2:] - v[:-2])
    err = np.abs(fd - fp[1:-1]).max() / np.abs(fp).max()
    print(f"{g['vgrid']}: max |FD - F0'| / max |F0'| = {err:.2e}")
    assert err <= 5e-5


def test_fraction_above_speed_closed_forms(oracle_lib):
    """Share of electrons faster than V = 3 v_th: Gamma(3/4, Y^4) / Gamma(3/4)
    with Y = V sqrt(m / (2 eps0)) for the Druyvesteyn F0 (0.0038: the flat top
    starves the tail), erfc(V / (sqrt 2 v_th)) + sqrt(2/pi) (V/v_th)
    exp(-V^2 / (2 v_th^2)) for the Maxwellian (0.029).  The cut falls on a
    cell edge of the midpoint grid, so the sums converge as the cell width^2."""
    sp = pytest.importorskip("scipy.special")
    out = {}
    for f0 in ("druyvesteyn", "maxwell"):
        t, vth = _tables(oracle_lib, f0_model=f0, vgrid="speed3d", nv=2048)
        tail = t["v"] > 3 * vth
        out[f0] = np.sum((t["f0"] * t["dV"])[tail])
    eps0 = 1.5 * QE * 2.0 * math.gamma(0.75) / math.gamma(1.25)
    Y = 3 * vth * math.sqrt(ME / (2 * eps0))
    want_d = sp.gammaincc(0.75, Y ** 4)
    want_m = math.erfc(3 / math.sqrt(2)) + math.sqrt(2 / math.pi) * 3 * math.exp(-4.5)
    print(f"tail share above 3 v_th: Druyvesteyn {out['druyvesteyn']:.6e} (closed form {want_d:.6e}), "
          f"Maxwellian {out['maxwell']:.6e} ({want_m:.6e})")
    assert abs(out["druyvesteyn"] / want_d - 1) <= 1e-4
    assert abs(out["maxwell"] / want_m - 1) <= 1e-4


def test_table_constant_sigma_is_nsv(oracle_lib):
    for g in GRIDS:
        sp = np.array([0.0, 1e5, 7e6])
        t1, _ = _tables(oracle_lib, nu_model="nsv", **g)
        t2, _ = _tables(oracle_lib, nu_model="table", s_table=(sp, np.full(3, 3.7e-20)), **g)
        assert np.allclose(t2["nu"], t1["nu"], rtol=1e-13, atol=0)


def test_table_inverse_speed_gives_constant_nu(oracle_lib):
    g = dict(vgrid="speed3d", nv=40)
    t0, _ = _tables(oracle_lib, **g)
    sp = t0["v"].copy()                       # table points at the node speeds: interpolation is exact there
    t, _ = _tables(oracle_lib, nu_model="table", s_table=(sp, 1.0 / sp), **g)
    assert np.allclose(t["nu"], 1e9, rtol=1e-13, atol=0)


def test_table_linear_sigma_and_clamped_ends(oracle_lib):
    """s(v) = a + b v given at a few irregular points inside the grid range:
    nu_j / nu_k = s(v_j) v_j / (s(v_k) v_k) with s linear inside the table and
    held at the end values outside it."""
    g = dict(vgrid="signed1d", nv=64)
    t0, vth = _tables(oracle_lib, **g)
    a, b = 2.0, 3.0 / vth
    sp = np.array([0.3, 0.9, 2.2, 4.1]) * vth
    t, _ = _tables(oracle_lib, nu_model="table", s_table=(sp, a + b * sp), **g)
    speed = np.abs(t["v"])
    s = np.clip(a + b * speed, a + b * sp[0], a + b * sp[-1])
    ratio = t["nu"] / (s * speed)
    assert np.allclose(ratio, ratio[0], rtol=1e-13, atol=0)
    # the F0-weighted mean of nu is nu0
    assert abs(np.sum(t["nu"] * t["f0"] * t["dV"]) / np.sum(t["f0"] * t["dV"]) / 1e9 - 1) <= 1e-13


def test_druyvesteyn_drude_recursion(oracle_lib):
    """Constant nu: J^{n+1/2} = rho J^{n-1/2} + 2dt/(2+dt nu) eps0 wp^2 E^n
    with the Drude weight 1, for a Druyvesteyn plasma on the Cartesian grid."""
    O = oracle_lib
    n = 3e17
    p = O.params(vgrid="cart2d", nv=24, nv_perp=24, te_ev=1.0, f0_model="druyvesteyn", nu0=5e8, nu_model="const")
    rng = np.random.default_rng(3)
    E = rng.standard_normal(300)
    dt = 1.2e-12
    J, _ = O.kinetic_drive(p, dt, n, E)
    t = O.vtables(p, dt)
    weff2 = plasma_omega(n) ** 2 * (-np.sum(t["w"] * t["f0p"]))
    nu = 5e8
    rho = (2 - dt * nu) / (2 + dt * nu)
    pred = np.zeros_like(J)
    prev = 0.0
    for m in range(E.size):
        prev = rho * prev + 2 * dt / (2 + dt * nu) * EPS0 * weff2 * E[m]
        pred[m] = prev
    assert np.abs(J - pred).max() <= 1e-12 * np.abs(J).max()
