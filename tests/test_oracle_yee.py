"""Pins of the oracle's Yee / CPML field update (Sec. 2, Eq. 1-12; Sec. 4).

Each test checks the oracle against something other than itself: exact
discrete eigenmodes of a PEC cavity, the discrete energy invariant, the
paper's vacuum Gaussian-pulse convergence order and a brute-force
oversized-domain run for the CPML, and the closed-form reflection of a
PEC-backed graded PML for the CPML profiles.
"""
import json
import os

import numpy as np
import pytest

from tests.physics import C0, EPS0, MU0, ETA0, yee_omega

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ------------------------------------------------------------ eigenmodes (P-a)

def test_eigenmode_1d(oracle_lib):
    O = oracle_lib
    nz, dx = 90, 1e-3
    s = O.Sim(O.params(ndim=1, nz=nz, dx=dx, courant=0.5))
    dt = s.dt
    k = 4 * np.pi / (nz * dx)
    w = yee_omega(dt, dx, [k])
    z, zh = np.arange(nz + 1) * dx, (np.arange(nz) + 0.5) * dx
    # H^{-1/2} of the standing mode follows from the discrete Faraday law
    B = -(dt / (MU0 * dx)) * np.sin(k * dx / 2) / np.sin(w * dt / 2)
    s.set("ex", np.sin(k * z))
    s.set("hy", B * np.cos(k * zh) * np.sin(-w * dt / 2))
    N = 10000
    s.step(N)
    assert np.abs(s.get("ex") - np.sin(k * z) * np.cos(w * N * dt)).max() < 1e-10


def test_eigenmode_2d_tmz(oracle_lib):
    O = oracle_lib
    nx, ny, dx = 40, 30, 2e-3
    s = O.Sim(O.params(ndim=2, nx=nx, ny=ny, dx=dx, courant=0.5))
    dt = s.dt
    kx, ky = 3 * np.pi / (nx * dx), 2 * np.pi / (ny * dx)
    w = yee_omega(dt, dx, [kx, ky])
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ez0 = np.sin(kx * i * dx) * np.sin(ky * j * dx)
    sw = np.sin(w * dt / 2)
    # Hx(i, j+1/2) and Hy(i+1/2, j) at t = -dt/2 from the discrete Faraday law
    hx = -(dt / (MU0 * dx)) * np.sin(ky * dx / 2) / sw * np.sin(kx * i * dx) * np.cos(ky * (j + 0.5) * dx) * np.sin(-w * dt / 2)
    hy = (dt / (MU0 * dx)) * np.sin(kx * dx / 2) / sw * np.cos(kx * (i + 0.5) * dx) * np.sin(ky * j * dx) * np.sin(-w * dt / 2)
    s.set("ez", ez0.ravel()); s.set("hx", hx.ravel()); s.set("hy", hy.ravel())
    N = 3000
    s.step(N)
    ref = ez0 * np.cos(w * N * dt)
    assert np.abs(s.get("ez").reshape(ny, nx) - ref).max() < 1e-10


@pytest.mark.parametrize("pol", ["ex", "ey", "ez"])
def test_eigenmode_3d(oracle_lib, pol):
    """Cavity mode polarised along one axis and uniform along it; the three
    polarisations together exercise all twelve curl differences."""
    O = oracle_lib
    n = (14, 12, 10)
    dx = 2e-3
    s = O.Sim(O.params(ndim=3, nx=n[0], ny=n[1], nz=n[2], dx=dx, courant=0.5))
    dt = s.dt
    a = "xyz".index(pol[1])
    o1, o2 = [(a + 1) % 3, (a + 2) % 3]
    m = {o1: 2, o2: 1}
    k = {ax: m[ax] * np.pi / (n[ax] * dx) for ax in (o1, o2)}
    w = yee_omega(dt, dx, [k[o1], k[o2]])
    K, J, I = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = [I, J, K]
    # component positions: E_a at half-integer along a, integer along others
    E0 = np.sin(k[o1] * idx[o1] * dx) * np.sin(k[o2] * idx[o2] * dx)
    sw = np.sin(w * dt / 2)
    t_h = np.sin(-w * dt / 2)
    # H_{o2} = ... from mu0 dH/dt = -curl E with only E_a nonzero:
    #   (curl E)_{o1} = eps(a,o2,o1) dE_a/d o2 ... written per cyclic order
    # cyclic (a, o1, o2): (curl E)_{o1} = dE_a/d o2,  (curl E)_{o2} = -dE_a/d o1
    ch = dt / (MU0 * dx)
    H_o1 = -ch * (2 * np.sin(k[o2] * dx / 2)) / (2 * sw) * np.sin(k[o1] * idx[o1] * dx) * np.cos(k[o2] * (idx[o2] + 0.5) * dx) * t_h
    H_o2 = ch * (2 * np.sin(k[o1] * dx / 2)) / (2 * sw) * np.cos(k[o1] * (idx[o1] + 0.5) * dx) * np.sin(k[o2] * idx[o2] * dx) * t_h
    s.set(pol, E0.ravel())
    s.set("h" + "xyz"[o1], H_o1.ravel())
    s.set("h" + "xyz"[o2], H_o2.ravel())
    N = 2000
    s.step(N)
    assert np.abs(s.get(pol) - (E0 * np.cos(w * N * dt)).ravel()).max() < 1e-10
    for other in ("ex", "ey", "ez"):
        if other != pol:
            assert np.abs(s.get(other)).max() < 1e-12


# -------------------------------------------------------- energy invariant (P-b)

@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_energy_invariant_pec_cavity(oracle_lib, ndim):
    O = oracle_lib
    rng = np.random.default_rng(7)
    if ndim == 1:
        p = O.params(ndim=1, nz=200, dx=1e-3)
    elif ndim == 2:
        p = O.params(ndim=2, nx=37, ny=29, dx=1e-3)
    else:
        p = O.params(ndim=3, nx=11, ny=9, nz=8, dx=1e-3)
    s = O.Sim(p)
    names = {1: ["ex", "hy"], 2: ["ez", "hx", "hy"], 3: ["ex", "ey", "ez", "hx", "hy", "hz"]}[ndim]
    for nm in names:
        n = s.get(nm).size
        a = rng.standard_normal(n) * (1.0 if nm[0] == "e" else 1.0 / ETA0)
        s.set(nm, a)
    # PEC nodes must start at zero (they are never updated)
    if ndim == 1:
        ex = s.get("ex"); ex[0] = ex[-1] = 0; s.set("ex", ex)
    elif ndim == 2:
        ez = s.get("ez").reshape(29, 37); ez[0, :] = 0; ez[:, 0] = 0; s.set("ez", ez.ravel())
    else:
        sh = (8, 9, 11)
        ex = s.get("ex").reshape(sh); ex[:, 0, :] = 0; ex[0, :, :] = 0; s.set("ex", ex.ravel())
        ey = s.get("ey").reshape(sh); ey[:, :, 0] = 0; ey[0, :, :] = 0; s.set("ey", ey.ravel())
        ez = s.get("ez").reshape(sh); ez[:, :, 0] = 0; ez[:, 0, :] = 0; s.set("ez", ez.ravel())
    W0 = s.diag()["energy"]
    ws = []
    for _ in range(20):
        s.step(50)
        ws.append(s.diag()["energy"])
    assert max(abs(w - W0) for w in ws) / W0 < 1e-12
    # the plain energy is NOT invariant: the test would not pass vacuously
    assert abs(s.diag()["energy_plain"] - W0) / W0 > 1e-6


# --------------------------------------------- Gaussian pulse convergence (P-c)

def _pulse_error(O, ppw):
    """RMS error (Eq. 15) of the 1-D Yee solution of the Eq. 14 pulse."""
    tau = GOLD["validation_pulse_tau_s"]["value"]
    t0 = GOLD["validation_pulse_t0_s"]["value"]
    ctau = C0 * tau
    dz = ctau / ppw
    L = 3.0
    nz = int(round(L / dz))
    s = O.Sim(O.params(ndim=1, nz=nz, dx=dz, courant=0.5))
    dt = s.dt
    exact = lambda z, t: np.exp(-(((C0 * (t - t0)) - z) / ctau) ** 2)
    ts = t0 + 0.6 / C0          # pulse centred at z = 0.6 m
    z, zh = np.arange(nz + 1) * dz, (np.arange(nz) + 0.5) * dz
    e0 = exact(z, ts); e0[0] = e0[-1] = 0.0
    s.set("ex", e0)
    s.set("hy", exact(zh, ts - dt / 2) / ETA0)
    T = 5e-9
    N = int(round(T / dt))
    s.step(N)
    u = s.get("ex")
    return np.sqrt(np.mean((u - exact(z, ts + N * dt)) ** 2))


def test_gaussian_pulse_order(oracle_lib):
    errs = [_pulse_error(oracle_lib, ppw) for ppw in (10, 20, 40, 80)]
    hs = np.array([1 / 10, 1 / 20, 1 / 40, 1 / 80])
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    target = GOLD["convergence_order"]["value"]
    assert abs(order - target) < 0.1, (errs, order)


# ------------------------------------------------------- CPML vs big box (P-k)

def test_cpml_2d_against_oversized_domain(oracle_lib):
    O = oracle_lib
    n, L, dx = 80, 10, 1e-3
    fc = C0 / (20 * dx)
    src = dict(src_kind="gauss_sine", src_amp=1.0, src_fc=fc, src_tau=1.0 / fc, src_t0=4.0 / fc)
    p = O.params(ndim=2, nx=n, ny=n, dx=dx, cpml=L, src_i=n // 2, src_j=n // 2, **src)
    big = 3 * n
    pb = O.params(ndim=2, nx=big, ny=big, dx=dx, src_i=big // 2, src_j=big // 2, **src)
    s, sb = O.Sim(p), O.Sim(pb)
    steps = 260   # the wave crosses the small box; the big box's walls are not reached
    s.step(steps); sb.step(steps)
    ez = s.get("ez").reshape(n, n)[L:n - L, L:n - L]
    off = n
    ezb = sb.get("ez").reshape(big, big)[off + L:off + n - L, off + L:off + n - L]
    rel = np.linalg.norm(ez - ezb) / np.linalg.norm(ezb)
    assert rel < 1e-3, rel
    # without CPML the same box is dominated by wall reflections
    s2 = O.Sim(O.params(ndim=2, nx=n, ny=n, dx=dx, src_i=n // 2, src_j=n // 2, **src))
    s2.step(steps)
    ez2 = s2.get("ez").reshape(n, n)[L:n - L, L:n - L]
    assert np.linalg.norm(ez2 - ezb) / np.linalg.norm(ezb) > 10 * rel


def test_cpml_3d_against_oversized_domain(oracle_lib):
    O = oracle_lib
    n, L, dx = 28, 8, 1e-3
    fc = C0 / (12 * dx)
    src = dict(src_kind="gauss_sine", src_amp=1.0, src_fc=fc, src_tau=1.0 / fc, src_t0=3.5 / fc)
    p = O.params(ndim=3, nx=n, ny=n, nz=n, dx=dx, cpml=L, src_i=n // 2, src_j=n // 2, src_k=n // 2, **src)
    big = 3 * n
    pb = O.params(ndim=3, nx=big, ny=big, nz=big, dx=dx, src_i=big // 2, src_j=big // 2, src_k=big // 2, **src)
    s, sb = O.Sim(p), O.Sim(pb)
    steps = 110
    s.step(steps); sb.step(steps)
    sl = slice(L, n - L)
    slb = slice(n + L, 2 * n - L)
    errs, refs = 0.0, 0.0
    for nm in ("ex", "ey", "ez"):
        a = s.get(nm).reshape(n, n, n)[sl, sl, sl]
        b = sb.get(nm).reshape(big, big, big)[slb, slb, slb]
        errs += np.sum((a - b) ** 2)
        refs += np.sum(b ** 2)
    rel = np.sqrt(errs / refs)
    assert rel < 3e-2, rel


def test_cpml_profile_shape(oracle_lib):
    """Profile sanity from Eq. 9-12: zero outside the layers, kappa rises to
    kappa_max towards the wall, 0 < b < 1 and a < 0 inside."""
    O = oracle_lib
    p = O.params(ndim=2, nx=60, ny=60, dx=1e-3, cpml=10)
    dt = 0.5 * 1e-3 / C0
    for at_h in (False, True):
        pr = O.cpml_profile(p, dt, 60, at_h)
        inside = np.zeros(60, bool)
        x = np.arange(60) + (0.5 if at_h else 0.0)
        inside[(x < 10) | (x > 50)] = True
        assert np.all(pr["kappa"][~inside] == 1.0) and np.all(pr["a"][~inside] == 0.0)
        assert np.all((pr["b"][inside] > 0) & (pr["b"][inside] < 1))
        assert np.all(pr["a"][inside] < 0)
        assert pr["kappa"][0 if not at_h else 0] <= 7.0 + 1e-12
    e = O.cpml_profile(p, dt, 60, False)
    assert e["kappa"][0] == pytest.approx(7.0)     # rho = delta at the PEC wall
    # symmetry of the two layers
    h = O.cpml_profile(p, dt, 60, True)
    assert np.allclose(h["b"][:10], h["b"][::-1][:10])


# ------------------------------------------- CPML reflection (Eq. 9-12, P-k)

def _cpml_line(O, n, L, dx, sigma_factor, kappa_max, alpha_max, src, probe, steps, fc):
    """1-D line of the oracle's CPML profiles (or_cpml_profile at E and H
    positions, PEC behind both layers), stepped with the textbook CPML
    recursion psi <- b psi + a dF, curl term dF / (kappa dx) + psi; returns E
    at `probe` after each step.  Only the profile values come from the oracle."""
    p = O.params(ndim=2, nx=n, ny=n, dx=dx, cpml=L, cpml_sigma_factor=sigma_factor, cpml_kappa_max=kappa_max,
                 cpml_alpha_min=0.0, cpml_alpha_max=alpha_max)
    dt = 0.5 * dx / C0
    pe, ph = O.cpml_profile(p, dt, n, False), O.cpml_profile(p, dt, n, True)
    ez, hy = np.zeros(n + 1), np.zeros(n)
    pse, psh = np.zeros(n - 1), np.zeros(n)
    be, ae, ke = pe["b"][1:n], pe["a"][1:n], pe["kappa"][1:n]
    tau, t0 = 1.0 / fc, 4.0 / fc
    rec = np.zeros(steps)
    for s in range(steps):
        dE = ez[1:] - ez[:-1]
        psh = ph["b"] * psh + ph["a"] * dE
        hy += dt / (MU0 * dx) * dE / ph["kappa"] + dt / MU0 * psh
        dH = hy[1:] - hy[:-1]
        pse = be * pse + ae * dH
        ez[1:n] += dt / (EPS0 * dx) * dH / ke + dt / EPS0 * pse
        t = (s + 1) * dt
        ez[src] += np.sin(2 * np.pi * fc * (t - t0)) * np.exp(-((t - t0) / tau) ** 2)
        rec[s] = ez[probe]
    return rec, dt


def _cpml_reflection(O, sigma_factor, kappa_max, alpha_max):
    """Measured normal-incidence reflection R(f) of a PEC-backed L-cell layer,
    referred to the bare PEC at the same depth (sigma = 0, kappa = 1), with the
    incident wave removed by an unbounded reference line."""
    dx, L, lam = 5e-3, 40, 200
    fc = C0 / (lam * dx)
    n, steps = 1200, 4000
    src, probe = n - L - 200, n - L - 150
    big = 6000
    ref, dt = _cpml_line(O, big, 0, dx, 0.0, 1.0, 0.0, big // 2, big // 2 + probe - src, steps, fc)
    pec, _ = _cpml_line(O, n, L, dx, 0.0, 1.0, 0.0, src, probe, steps, fc)
    lay, _ = _cpml_line(O, n, L, dx, sigma_factor, kappa_max, alpha_max, src, probe, steps, fc)
    nfft = 16384
    f = np.fft.rfftfreq(nfft, dt)
    band = (f > 0.5 * fc) & (f < 1.6 * fc)
    R = np.fft.rfft(lay - ref, nfft)[band] / np.fft.rfft(pec - ref, nfft)[band]
    return f[band], R, L * dx, dx


def test_cpml_sigma_max_attenuation(oracle_lib):
    """Weak graded layer, kappa = 1, alpha = 0: a PEC-backed PML returns the
    wave attenuated by exp(-2 int_0^delta sigma(rho) d rho / (eps0 c)) =
    exp(-2 sigma_max delta / ((n+1) eps0 c)) at every frequency, with sigma_max
    of Eq. 11.  A wrong constant in Eq. 11 (120 pi for 150 pi, a missing n + 1,
    delta for the cell size) moves the exponent by 25 % or more."""
    O = oracle_lib
    sf, order = 0.0125, 3.0
    f, R, delta, dx = _cpml_reflection(O, sf, 1.0, 0.0)
    sigma_max = sf * (order + 1) / (150 * np.pi * dx)
    expo = -2 * sigma_max * delta / ((order + 1) * EPS0 * C0)
    ratio = np.log(np.abs(R)) / expo
    assert np.abs(ratio - 1).max() < 0.02, ratio
    assert np.abs(np.angle(R)).max() < 0.05


def test_cpml_cfs_reflection(oracle_lib):
    """Complex-frequency-shifted layer with the paper's kappa_max = 7 and
    alpha_max = 0.05 S/m: the reflection equals exp(-2i (w/c) int (s - 1) d rho)
    with s = kappa + sigma / (alpha + i w eps0) and the gradings of Eq. 12
    (alpha largest at the inner interface, kappa and sigma rising as
    (rho/delta)^n), by quadrature of the continuous profiles.  Reversing the
    alpha grading changes the attenuation by ~90 % in this band; kappa sets the
    phase."""
    O = oracle_lib
    sf, km, am, order = 0.0125, 7.0, 0.05, 3.0
    f, R, delta, dx = _cpml_reflection(O, sf, km, am)
    m = 20000
    rho = (np.arange(m) + 0.5) / m * delta
    r = rho / delta
    sigma = sf * (order + 1) / (150 * np.pi * dx) * r ** order
    kappa = 1 + (km - 1) * r ** order
    alpha = am * (1 - r)
    w = 2 * np.pi * f[:, None]
    s = kappa + sigma / (alpha + 1j * w * EPS0)
    Rth = np.exp(-2j * w[:, 0] / C0 * np.sum(s - 1, axis=1) * (delta / m))
    assert (np.abs(R - Rth) / np.abs(Rth)).max() < 0.05
    assert np.abs(np.log(np.abs(R)) / np.log(np.abs(Rth)) - 1).max() < 0.02
