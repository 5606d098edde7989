"""Pins of the oracle's closure-data transform (oracle/closure_data.py): the
Drude part it subtracts is the paper's velocity-space update (Sec. 5.2,
Eq. 22-24) in the case where that update has a closed form.

* With a speed-independent collision frequency the kinetic current of a
  driven cell obeys the Crank-Nicolson Drude recursion, so the residual the
  network would learn vanishes (to the grid's Drude weight, 1 - 7e-8).
* With nu = N s v it does not: the residual is the kinetic correction.
* n_c is the density whose plasma frequency is w0 (closed form).
"""
import numpy as np

from oracle import closure_data as CD
from tests.physics import EPS0, plasma_omega

OMEGA0 = 2 * np.pi * 299792458.0 / 0.03


def _driven(O, nu_model, n_dens=3.0e17, steps=600, seed=4):
    p = O.params(ndim=1, nz=4, dx=0.03 / 40, vgrid="signed1d", nv=64, nu0=0.01 * OMEGA0, nu_model=nu_model)
    dt = 0.5 * 0.03 / 40 / 299792458.0
    rng = np.random.default_rng(seed)
    m = np.arange(steps)
    E = np.cos(OMEGA0 * m * dt) * np.exp(-((m - 250) / 120.0) ** 2) + 0.05 * rng.standard_normal(steps)
    J, _ = O.kinetic_drive(p, dt, n_dens, E)
    return CD.samples_from_series(E, J, n_dens), dt, p


def test_critical_density_closed_form():
    n_c = CD.critical_density(OMEGA0)
    assert abs(plasma_omega(n_c) / OMEGA0 - 1) < 1e-14
    assert abs(n_c / 1.2387e18 - 1) < 1e-4          # lambda0 = 3 cm


def test_residual_vanishes_for_constant_collision_frequency(oracle_lib):
    s, dt, p = _driven(oracle_lib, "const")
    rho, beta = CD.drude_coefficients(dt, p.nu0)
    r = CD.residual(s, rho, beta)
    drude = beta * s[:, 16] * s[:, 15]
    assert np.abs(drude).max() > 0
    assert np.abs(r).max() <= 1e-6 * np.abs(drude).max(), np.abs(r).max() / np.abs(drude).max()
    # a wrong coefficient leaves a residual of the size of the current
    r_bad = CD.residual(s, rho, beta * (1 + 1e-3))
    assert np.abs(r_bad).max() > 1e-4 * np.abs(drude).max()


def test_residual_is_the_kinetic_correction_for_speed_dependent_nu(oracle_lib):
    s, dt, p = _driven(oracle_lib, "nsv")
    rho, beta = CD.drude_coefficients(dt, p.nu0)
    r = CD.residual(s, rho, beta)
    assert np.abs(r).max() > 2e-4 * np.abs(s[:, 17]).max()      # 7.8e-4 here; 5e-9 with constant nu


def test_scales_and_dataset(oracle_lib):
    s, dt, p = _driven(oracle_lib, "nsv")
    sc = CD.scales(s, OMEGA0, dt, p.nu0)
    x, t = CD.dataset(s, sc)
    assert abs(np.sqrt(np.mean(x[:, :16] ** 2)) - 1) < 1e-12      # E_s is the RMS of the history
    assert abs(np.sqrt(np.mean(t ** 2)) - 1) < 1e-12              # unit-variance targets
    assert np.allclose(x[:, 16], s[:, 16] / sc["n_scale"])
    # constant history +-A gives E_s = A; a zero residual falls back to eps0 w0 E_s
    c = np.zeros((4, 19))
    c[:, :16] = 2.5 * np.where(np.arange(16) % 2, 1, -1)
    sc0 = CD.scales(c, OMEGA0, dt, 0.0, increment=False)
    assert sc0["e_scale"] == 2.5 and sc0["j_scale"] == EPS0 * OMEGA0 * 2.5 and sc0["rho"] == 0.0
