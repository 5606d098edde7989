"""Pins of the oracle's soft-source waveform and of the time level at which
the step applies it (Sec. 4, Eq. 14; Sec. 5.3, Table 3).

The pulse of Table 3 is pinned by the numbers the table prints besides the
ones that define it: its 20 GHz bandwidth and its 146 ps time bandwidth are
the -20 dB (one tenth in amplitude) widths of a Gaussian-modulated carrier
whose envelope is exp(-((t - t0)/tau)^2) with tau = 48 ps; the spectrum of such
a pulse peaks at f_c, and a sine carrier makes the pulse odd about t0, so its
spectrum referred to t0 is purely imaginary.  The time level is pinned by
what a soft source radiates in a 1-D vacuum line at Courant number S: a
travelling copy of g of amplitude 1/(2S), which leads g by dt/2 when the
source value added to E^{n+1} is g(t^{n+1}) and lags it by dt/2 if it were
g(t^n).
"""
import json
import math
import os

import numpy as np
import pytest

from tests.physics import C0

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _table3_params(O):
    return O.params(ndim=1, nz=10, dx=1e-3, src_kind="gauss_sine", src_amp=1.0,
                    src_fc=GOLD["pulse_fc_hz"]["value"], src_tau=GOLD["pulse_tau_s"]["value"],
                    src_t0=GOLD["pulse_t0_s"]["value"])


def _sample(O, p, t):
    return np.array([O.source(p, float(x)) for x in t])


def _crossings(x, y, level):
    """First and last abscissa where y (one hump) crosses `level`, linearly interpolated."""
    above = np.nonzero(y >= level)[0]
    i0, i1 = above[0], above[-1]
    lo = x[i0 - 1] + (level - y[i0 - 1]) / (y[i0] - y[i0 - 1]) * (x[i0] - x[i0 - 1])
    hi = x[i1] + (level - y[i1]) / (y[i1 + 1] - y[i1]) * (x[i1 + 1] - x[i1])
    return lo, hi


def test_table3_pulse_spectrum(oracle_lib):
    """Spectrum of the oracle's Table 3 pulse: peak at f_c, -20 dB full width =
    the printed 20 GHz bandwidth, the sine carrier's -pi/2 phase about t0, and
    the peak magnitude A tau sqrt(pi) / 2 of the Gaussian's Fourier transform."""
    O = oracle_lib
    p = _table3_params(O)
    fc, tau, t0 = p.src_fc, p.src_tau, p.src_t0
    h = 0.05e-12
    t = np.arange(0, 2 * t0, h)
    g = _sample(O, p, t)
    nfft = 1 << 20
    G = np.fft.rfft(g, nfft) * h                       # continuous transform by the rectangle rule
    f = np.fft.rfftfreq(nfft, h)
    mag = np.abs(G)
    k = int(np.argmax(mag))
    # parabolic refinement of the peak frequency
    a, b, c = mag[k - 1], mag[k], mag[k + 1]
    fpk = f[k] + 0.5 * (a - c) / (a - 2 * b + c) * (f[1] - f[0])
    assert abs(fpk / fc - 1) < 2e-3, fpk
    lo, hi = _crossings(f, mag, 0.1 * mag.max())
    bw = GOLD["pulse_bandwidth_hz"]["value"]
    assert abs((hi - lo) / bw - 1) < 0.02, (hi - lo, bw)
    # a cosine carrier would give phase 0, a pulse centred elsewhere a phase ramp
    ph = np.angle(G[k] * np.exp(2j * np.pi * f[k] * t0))
    assert abs(ph + np.pi / 2) < 1e-3, ph
    assert abs(mag.max() / (tau * math.sqrt(math.pi) / 2) - 1) < 1e-4
    # odd about t0 (sine carrier), zero at t0
    assert abs(O.source(p, t0)) < 1e-15
    s = np.linspace(1e-12, 3 * tau, 50)
    np.testing.assert_allclose(_sample(O, p, t0 + s), -_sample(O, p, t0 - s), atol=1e-15)


def test_table3_pulse_time_bandwidth(oracle_lib):
    """Envelope of the Table 3 pulse (magnitude of its analytic signal): its
    -20 dB span equals the printed 146 ps time bandwidth and it peaks at t0."""
    signal = pytest.importorskip("scipy.signal")
    O = oracle_lib
    p = _table3_params(O)
    h = 0.05e-12
    t = np.arange(0, 2 * p.src_t0, h)
    env = np.abs(signal.hilbert(_sample(O, p, t)))
    lo, hi = _crossings(t, env, 0.1 * env.max())
    dt_tab = GOLD["pulse_time_bandwidth_s"]["value"]
    assert abs((hi - lo) / dt_tab - 1) < 0.01, (hi - lo, dt_tab)
    assert abs(0.5 * (lo + hi) - p.src_t0) < 0.5e-12
    assert abs(t[int(np.argmax(env))] - p.src_t0) < 1e-12
    assert abs(env.max() - p.src_amp) < 1e-3


def test_soft_source_radiates_eq14_pulse_half_step_early(oracle_lib):
    """1-D vacuum line, Courant 0.5, Mur ends, Gaussian soft source with the
    paper's validation pulse (tau = 0.5 ns, t0 = 2.25 ns): the field d cells
    away is the travelling pulse of Eq. 14 of amplitude 1/(2S) = 1, leading by
    dt/2 because the value added to E^{n+1} is g(t^{n+1})."""
    O = oracle_lib
    dx = 0.03 / 40
    tau, t0 = GOLD["validation_pulse_tau_s"]["value"], GOLD["validation_pulse_t0_s"]["value"]
    nz, src, d = 4000, 800, 400
    p = O.params(ndim=1, nz=nz, dx=dx, courant=0.5, mur=1, src_kind="gauss", src_amp=1.0, src_tau=tau,
                 src_t0=t0, src_k=src)
    s = O.Sim(p)
    dt = s.dt
    n_steps = int((t0 + 2.5 * tau + d * dx / C0) / dt)
    rec = np.zeros(n_steps)
    for n in range(n_steps):
        s.step(1)
        rec[n] = s.get("ex")[src + d]
    t = (np.arange(n_steps) + 1) * dt                 # E^{n+1} sits at t^{n+1}
    k = int(np.argmax(rec))
    a, b, c = rec[k - 1], rec[k], rec[k + 1]
    t_peak = t[k] + 0.5 * (a - c) / (a - 2 * b + c) * dt
    lead = (t0 + d * dx / C0 - t_peak) / dt
    assert abs(lead - 0.5) < 0.05, lead                # g(t^n) would give -0.5
    assert abs(rec.max() - 1.0 / (2 * 0.5)) < 1e-4
    shifted = np.exp(-(((t + 0.5 * dt) - t0 - d * dx / C0) / tau) ** 2)
    assert np.abs(rec - shifted).max() < 2e-4
