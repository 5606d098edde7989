"""FP64 reference of the learned closure's training-data transform.

TEST INFRASTRUCTURE ONLY (imported by tests; never by the product library).

The closure is not in the paper.  It keeps the Crank-Nicolson update of a
Drude plasma with the mean collision frequency nu -- what the Sec. 5.2 f_1x
update and Jx sum (Eq. 22-24) reduce to when nu does not depend on the speed --
and a network learns the remaining kinetic correction:
    rho  = (2 - dt nu) / (2 + dt nu)
    beta = 2 dt (e^2 / m) / (2 + dt nu)
    r    = J^{n+1/2} - rho J^{n-1/2} - beta n E^n
    x    = [E^{n-15} .. E^n] / E_s ++ [n / n_c],   target = r / J_s
with E_s the RMS of the recorded E values, n_c = eps0 m w0^2 / e^2 the
critical density at the carrier frequency and J_s the RMS of r.  A sample is
the 19-vector [E^{n-15} .. E^n, n, J^{n+1/2}, J^{n-1/2}].
"""
from __future__ import annotations

import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def critical_density(omega0: float) -> float:
    """n_c = eps0 m w0^2 / e^2: the density whose plasma frequency is w0."""
    return EPS0 * ME * omega0 * omega0 / (QE * QE)


def drude_coefficients(dt: float, nu: float) -> tuple[float, float]:
    """(rho, beta) of the Crank-Nicolson Drude current update
    (2 + dt nu) J^{n+1/2} = (2 - dt nu) J^{n-1/2} + 2 dt (e^2/m) n E^n."""
    return (2.0 - dt * nu) / (2.0 + dt * nu), 2.0 * dt * (QE * QE / ME) / (2.0 + dt * nu)


def residual(samples: np.ndarray, rho: float, beta: float) -> np.ndarray:
    s = np.asarray(samples, dtype=np.float64)
    return s[:, 17] - rho * s[:, 18] - beta * s[:, 16] * s[:, 15]


def scales(samples: np.ndarray, omega0: float, dt: float, nu_mean: float, increment: bool = True) -> dict:
    s = np.asarray(samples, dtype=np.float64)
    e_s = float(np.sqrt(np.mean(s[:, :16] ** 2)))
    rho, beta = drude_coefficients(dt, nu_mean) if increment else (0.0, 0.0)
    j_s = float(np.sqrt(np.mean(residual(s, rho, beta) ** 2)))
    if j_s == 0.0:
        j_s = EPS0 * omega0 * e_s
    return dict(e_scale=e_s, j_scale=j_s, n_scale=critical_density(omega0), rho=rho, beta=beta)


def dataset(samples: np.ndarray, sc: dict) -> tuple[np.ndarray, np.ndarray]:
    """FP64 inputs [N, 17] and targets [N]."""
    s = np.asarray(samples, dtype=np.float64)
    x = np.empty((s.shape[0], 17))
    x[:, :16] = s[:, :16] / sc["e_scale"]
    x[:, 16] = s[:, 16] / sc["n_scale"]
    return x, residual(s, sc["rho"], sc["beta"]) / sc["j_scale"]


def samples_from_series(E: np.ndarray, J: np.ndarray, density: float) -> np.ndarray:
    """Samples of a driven cell: step m gives [E^{m-15..m} (0 before the
    start), n, J^{m+1/2}, J^{m-1/2} (0 at m = 0)]."""
    N = E.size
    out = np.zeros((N, 19))
    for m in range(N):
        h = E[max(0, m - 15):m + 1]
        out[m, 16 - h.size:16] = h
        out[m, 16] = density
        out[m, 17] = J[m]
        out[m, 18] = J[m - 1] if m > 0 else 0.0
    return out
