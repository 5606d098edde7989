"""Closed forms the oracle and the CUDA path are pinned to.

Everything here is derived from the mathematics of the continuous and the
discrete (Yee / Crank-Nicolson) equations, not from either implementation:
discrete plane-wave dispersion relations, the discrete Drude response that the
kinetic update reduces to, Airy (Fabry-Perot) slab coefficients and the like.
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C0 * C0)
ETA0 = MU0 * C0


def plasma_omega(n: float) -> float:
    """Electron plasma angular frequency sqrt(n e^2 / (eps0 m))."""
    return np.sqrt(n * QE * QE / (EPS0 * ME))


def yee_omega(dt: float, dx: float, ks, omega_eff: float = 0.0) -> float:
    """Real frequency of a discrete Yee mode with wavenumbers ``ks`` (one per
    axis) in a uniform collisionless Drude plasma:
    (2/dt)^2 sin^2(w dt/2) = w_eff^2 + c^2 sum (2/dx)^2 sin^2(k dx/2)."""
    K2 = sum((2.0 / dx * np.sin(k * dx / 2.0)) ** 2 for k in ks)
    s = 0.5 * dt * np.sqrt(C0 * C0 * K2 + omega_eff ** 2)
    return 2.0 / dt * np.arcsin(s)


def maxwellian_moments_signed(vth, vmax, nv):
    """Midpoint quadrature of -int v dF0/dv dv for the 1-D Maxwellian (exact: 1)."""
    dv = 2 * vmax / nv
    v = (np.arange(nv) + 0.5 - nv / 2) * dv
    f0 = np.exp(-v * v / (2 * vth * vth)) / np.sqrt(2 * np.pi * vth * vth)
    return float(np.sum(v * v / vth ** 2 * f0 * dv))


def discrete_conductivity(omega, dt, density, nu, w, f0p):
    """Steady-state response J = sigma_d E of the Crank-Nicolson kinetic
    update driven by E^m = E e^{-i w m dt}.  With df_j^{m+1/2} = D_j e^{-i w (m+1/2) dt}
    and theta = w dt / 2:
      D_j ((2 + dt nu_j) e^{-i theta} - (2 - dt nu_j) e^{i theta}) = 2 dt (e/m) F0'_j n E
      D_j (-4 i sin theta + 2 dt nu_j cos theta)               = 2 dt (e/m) F0'_j n E
    so sigma_d = -e n sum_j w_j (e/m) F0'_j / (-i Om + nu_j cos theta),
    Om = (2/dt) sin theta, with J^{m+1/2} referred to t^{m+1/2}."""
    Om = 2.0 / dt * np.sin(omega * dt / 2.0)
    return -QE * density * np.sum(w * (QE / ME) * f0p / (-1j * Om + nu * np.cos(omega * dt / 2.0)))


def drude_eps(omega, omega_p, nu):
    """Relative permittivity of a cold collisional plasma, e^{-i w t} convention."""
    return 1.0 - omega_p ** 2 / (omega * (omega + 1j * nu))


def slab_rt(omega, eps, d):
    """Complex reflection / transmission amplitudes of a slab of thickness d
    and relative permittivity eps between two vacuum half-spaces (normal
    incidence, e^{-i w t}); transmission is referred to the vacuum wave at the
    same exit plane, so |T| is its magnitude relative to no slab."""
    k0 = omega / C0
    n = np.sqrt(eps + 0j)
    if np.imag(n) < 0:
        n = -n
    r = (1 - n) / (1 + n)
    ph = np.exp(2j * k0 * n * d)
    R = r * (1 - ph) / (1 - r * r * ph)
    T = (1 - r * r) * np.exp(1j * k0 * n * d) / (1 - r * r * ph) * np.exp(-1j * k0 * d)
    return R, T


def mur1_reflection(omega, dt, dz):
    """Reflection coefficient of the discrete first-order Mur condition for a
    discrete Yee plane wave: substitute E_k^n = Z^n (X^k + R X^{-k}) with
    Z = e^{-i w dt}, X = e^{-i kappa} (kappa from the discrete dispersion,
    wave incident on node 0) into E_0^{n+1} = E_1^n + m (E_1^{n+1} - E_0^n)."""
    S = C0 * dt / dz
    kap = 2 * np.arcsin(np.sin(omega * dt / 2) / S)
    Z = np.exp(-1j * omega * dt)
    X = np.exp(-1j * kap)
    m = (S - 1) / (S + 1)
    # Z (1 + R) = X + R/X + m Z (X + R/X) - m (1 + R)
    num = X + m * Z * X - m - Z
    den = Z - 1 / X - m * Z / X + m
    return num / den
