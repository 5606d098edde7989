"""Pins of the coupled oracle against wave physics (Sec. 5.3 S-parameter
experiment, made synthetic) and of the first-order Mur boundary.

* A uniform collisional plasma slab in 1-D: |R| and |T| from running spectra
  at two probes (normalised by a vacuum run) against the Airy formula for a
  Drude slab (the kinetic update with constant nu is exactly Drude); total
  reflection below the plasma frequency as in the paper's Fig. "f" discussion.
* The Mur end's measured reflection against the reflection coefficient of the
  discrete first-order Mur condition for a discrete plane wave.
"""
import numpy as np
import pytest

from tests.physics import C0, EPS0, ME, QE, drude_eps, mur1_reflection, plasma_omega, slab_rt

LAM0 = 0.03
F0 = C0 / LAM0
OMEGA0 = 2 * np.pi * F0
T0 = 1 / F0


def test_slab_reflection_transmission(oracle_lib):
    O = oracle_lib
    dz, nz = LAM0 / 40, 2400
    k1, k2 = 1200, 1279
    n = (0.8 ** 2) * EPS0 * ME * OMEGA0 ** 2 / QE ** 2
    nu = 0.02 * OMEGA0
    dens = np.zeros(nz + 1)
    dens[k1:k2 + 1] = n
    base = dict(ndim=1, nz=nz, dx=dz, courant=0.5, mur=1, src_kind="gauss_sine", src_amp=1.0, src_fc=F0,
                src_tau=0.5 * T0, src_t0=3 * T0, src_k=200, vgrid="signed1d", nv=64, te_ev=1.0, nu0=nu,
                nu_model="const")
    sv, ss = O.Sim(O.params(**base)), O.Sim(O.params(**base), dens)
    p1, p2 = 700, 1800
    M = 12000
    freqs = np.linspace(0.55, 1.55, 21) * F0
    Xv, Xs = O.port_spectra([sv, ss], [[p1], [p2]], freqs, M)
    dt = sv.dt
    t = O.vtables(ss.p, dt)
    weff = plasma_omega(n) * np.sqrt(-np.sum(t["w"] * t["f0p"]))
    d = (k2 - k1 + 1) * dz          # plasma nodes k1..k2 each own one cell
    worst = 0.0
    for i, f in enumerate(freqs):
        w = 2 * np.pi * f
        R, T = slab_rt(w, drude_eps(w, weff, nu), d)
        Rm = abs((Xs[0, i] - Xv[0, i]) / Xv[0, i])      # S11 from the port spectra
        Tm = abs(Xs[1, i] / Xv[1, i])                   # S21
        worst = max(worst, abs(Rm - abs(R)), abs(Tm - abs(T)))
        if f < 0.75 * F0:            # below f_p = 0.8 f0: (almost) total reflection
            assert Rm > 0.93 and Tm < 0.05
    assert worst < 2e-2, worst


def test_port_spectra_equal_fft_at_bin_frequencies(oracle_lib):
    """At the FFT's bin frequencies k / (M dt) the running DFT of a pulse that
    has passed the port is dt times the discrete Fourier transform (numpy's
    FFT) of the recorded series, with the phase of the t_n = n dt time origin;
    a port of several nodes averages their fields."""
    O = oracle_lib
    dz, nz = LAM0 / 40, 1200
    base = dict(ndim=1, nz=nz, dx=dz, courant=0.5, mur=1, src_kind="gauss_sine", src_amp=1.0, src_fc=F0,
                src_tau=0.5 * T0, src_t0=3 * T0, src_k=200)
    s1, s2 = O.Sim(O.params(**base)), O.Sim(O.params(**base))
    M = 2048
    dt = s1.dt
    cells = [400, 401, 405]
    rec = np.zeros(M)
    for m in range(M):
        s2.step(1)
        rec[m] = np.mean(s2.get("ex")[cells])
    fr = np.arange(1, 60) / (M * dt)
    (X,) = O.port_spectra([s1], [cells], fr, M)
    # t_n = (m + 1) dt for record m: shift the FFT's origin by one step
    want = dt * np.fft.fft(rec)[1:60] * np.exp(-2j * np.pi * fr * dt)
    assert np.abs(X[0] - want).max() <= 1e-10 * np.abs(want).max()


def test_mur_reflection_matches_discrete_theory(oracle_lib):
    O = oracle_lib
    dz, nz = LAM0 / 20, 4000
    base = dict(ndim=1, nz=nz, dx=dz, courant=0.5, mur=1, src_kind="gauss_sine", src_amp=1.0, src_fc=F0,
                src_tau=0.5 * T0, src_t0=3 * T0, src_k=600)
    s = O.Sim(O.params(**base))
    pr, M = 300, 4000
    rec = np.zeros(M)
    for m in range(M):
        rec[m] = s.get("ex")[pr]
        s.step(1)
    t = np.arange(M)
    assert abs(rec[1350:1550]).max() < 1e-12 * abs(rec).max()   # incident and reflected pulses are separated
    Fi = np.fft.rfft(rec * (t < 1450))
    Fr = np.fft.rfft(rec * (t >= 1450))
    fr = np.fft.rfftfreq(M, s.dt)
    for f in np.linspace(0.6, 1.4, 9) * F0:
        i = np.argmin(abs(fr - f))
        R = abs(mur1_reflection(2 * np.pi * fr[i], s.dt, dz))
        assert abs(Fr[i] / Fi[i]) == pytest.approx(R, rel=2e-3)
