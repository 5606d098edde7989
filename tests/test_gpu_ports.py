"""Running-DFT ports (Sec. 5.3 S-parameters) on the GPU, through the C ABI,
against the oracle's port spectra, and the slab's S11 / S21 against the Airy
formula for a Drude slab (the kinetic update with constant nu is Drude)."""
import numpy as np
import pytest

from fdtd_inputs import C0, EPS0, ME, QE, spec_1d_slab, spec_2d_cylinder
from tests.adapters import oracle_sim

pytestmark = pytest.mark.gpu

LAM0 = 0.03
F0 = C0 / LAM0


def _solver(spec):
    from paper_2211_05647_gb300 import Solver
    return Solver.from_spec(spec)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_ports_match_oracle_1d(oracle_lib, prec, tol):
    spec = spec_1d_slab(nz=900, slab=(400, 520), src_k=60, precision=prec, steps=1500, nv=32)
    ports = [[200], [700], [300, 301, 650]]
    freqs = np.linspace(0.4, 1.6, 33) * F0
    s = _solver(spec)
    s.set_ports(ports, freqs)
    s.step(1500)
    got = s.port_spectra()
    (want,) = oracle_lib.port_spectra([oracle_sim(oracle_lib, spec)], ports, freqs, 1500)
    err = np.abs(got - want).max() / np.abs(want).max()
    print(f"1-D ports {prec}: max |X - X_oracle| / max |X| = {err:.2e}")
    assert err <= tol


def test_ports_match_oracle_2d(oracle_lib):
    spec = spec_2d_cylinder(n=120, ny=96, R=20, center=(70, 48), src=(30, 48), nv=8, nv_perp=8, steps=300,
                            precision="f64", f_dtype="f64", seed=4)
    nx = 120
    line = [j * nx + 100 for j in range(30, 66)]          # an Ez line behind the cylinder
    ports = [[48 * nx + 20], line]
    freqs = np.linspace(0.5, 1.5, 17) * F0
    s = _solver(spec)
    s.set_ports(ports, freqs)
    s.step(120)
    s.step(180)                                            # two graph launches: the step index carries on
    got = s.port_spectra()
    (want,) = oracle_lib.port_spectra([oracle_sim(oracle_lib, spec)], ports, freqs, 300)
    err = np.abs(got - want).max() / np.abs(want).max()
    print(f"2-D ports f64: {err:.2e}")
    assert err <= 1e-11


def test_slab_s_parameters_on_gpu():
    """The uniform-slab experiment of the oracle pin, on the FP32 GPU path:
    |S11|, |S21| from the port spectra of a plasma run and a vacuum run."""
    from tests.physics import drude_eps, plasma_omega, slab_rt
    dz, nz = LAM0 / 40, 2400
    k1, k2 = 1200, 1279
    n = (0.8 ** 2) * EPS0 * ME * (2 * np.pi * F0) ** 2 / QE ** 2
    nu = 0.02 * 2 * np.pi * F0
    spec = spec_1d_slab(nz=nz, ppw=40, slab=(k1, k2 + 1), src_k=200, precision="f32", steps=12000, nv=64)
    spec["source"].update(tau=0.5 / F0, t0=3 / F0, fc=F0, amp=1.0)
    spec["plasma"].update(nu_model="const", nu0=nu)
    dens = np.zeros(nz + 1)
    dens[k1:k2 + 1] = n
    spec["plasma"]["density"] = dens
    vac = dict(spec, plasma=None)
    freqs = np.linspace(0.55, 1.55, 21) * F0
    X = []
    for sp in (vac, spec):
        s = _solver(sp)
        s.set_ports([[700], [1800]], freqs)
        s.step(12000)
        X.append(s.port_spectra())
    Xv, Xs = X
    weff = plasma_omega(n)              # Drude weight of the velocity grid is 1 to 1e-12
    d = (k2 - k1 + 1) * dz
    worst = 0.0
    for i, f in enumerate(freqs):
        w = 2 * np.pi * f
        R, T = slab_rt(w, drude_eps(w, weff, nu), d)
        S11 = abs((Xs[0, i] - Xv[0, i]) / Xv[0, i])
        S21 = abs(Xs[1, i] / Xv[1, i])
        worst = max(worst, abs(S11 - abs(R)), abs(S21 - abs(T)))
    print(f"GPU slab |S11|, |S21| vs Airy: worst {worst:.2e}")
    assert worst < 2e-2


def test_ports_reject_bad_arguments():
    from paper_2211_05647_gb300 import FdtdError
    s = _solver(spec_1d_slab(nz=200, slab=(80, 120), precision="f32", steps=1, nv=16))
    for ports, freqs in (([[201]], [1e9]), ([[]], [1e9]), ([[5]], [np.nan]), ([[-1]], [1e9])):
        with pytest.raises(FdtdError):
            s.set_ports(ports, freqs)
    with pytest.raises(FdtdError):      # no ports set
        s.port_spectra()
