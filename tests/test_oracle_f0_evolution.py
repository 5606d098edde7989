"""Pins of the oracle's isotropic-F0 evolution on the speed grid (the F0
equation of the two-term expansion, Sec. 5.2: Joule heating through the
anisotropic part F1 plus elastic collisions with gas atoms of mass M at
temperature Tg).  Checks against what the equation fixes, not against the
update itself:
  * particle number: both terms are divergences, the grid sum of 4 pi v^2 dv
    times the F0 change stays 0;
  * energy: without collisions the electron kinetic energy gained equals the
    time integral of J E (the end nodes' flux terms aside, ~1e-6 here);
  * collisional relaxation with constant nu: the mean energy obeys
    d<eps>/dt = -2 (m/M) nu (<eps> - 3/2 k Tg) exactly in the continuum; the
    grid reproduces the exponential to second order in the node spacing;
  * weak fields: the J of the evolving model approaches the fixed-F0 model's
    as E^2 (the F0 change is second order in E)."""
import math

import numpy as np
import pytest

from tests.physics import ME, QE

DT = 1.25e-12
N = 3e17


def _drive(O, E, **kw):
    p = O.params(vgrid="speed3d", te_ev=1.0, evolve_f0=1, **kw)
    J, df, g = O.kinetic_drive(p, DT, N, E, with_f0=True)
    return J, df, g, O.vtables(p, DT)


def _pulse(amp, steps=3000):
    t = np.arange(steps) * DT
    return amp * np.sin(2 * np.pi * 1e10 * t) * np.exp(-((t - 1.5e-9) / 0.8e-9) ** 2)


def test_number_conserved_and_heating_equals_work(oracle_lib):
    E = _pulse(3e4)
    J, _, g, t = _drive(oracle_lib, E, nv=64, vmax_vth=6.0, nu0=2e9, nu_model="nsv", mass_ratio=0.0)
    v = t["v"]
    shell = 4 * np.pi * v ** 2 * (2 * v[0])
    assert abs(np.sum(shell * g)) <= 1e-14 * np.sum(np.abs(shell * g))
    W = N * np.sum(0.5 * ME * v ** 2 * shell * g)
    Jprev = np.concatenate([[0.0], J[:-1]])
    work = np.sum(E * 0.5 * (J + Jprev) * DT)           # J centred at step n
    print(f"electron energy gain {W:.6e} J/m^3, work of E on J {work:.6e}")
    assert W > 0 and abs(W / work - 1) <= 1e-5


def test_collisional_relaxation_closed_form(oracle_lib):
    mr, nu, tg, steps = 1e-2, 2e9, 0.2, 40000
    want = 1.5 * tg + 1.5 * (1.0 - tg) * math.exp(-2 * mr * nu * steps * DT)
    errs = {}
    for nv in (128, 256):
        _, _, g, t = _drive(oracle_lib, np.zeros(steps), nv=nv, vmax_vth=8.0, nu0=nu, nu_model="const",
                            mass_ratio=mr, tg_ev=tg)
        v = t["v"]
        shell = 4 * np.pi * v ** 2 * (2 * v[0])
        F0 = t["f0"] + g
        eps = np.sum(0.5 * ME * v ** 2 * shell * F0) / np.sum(shell * F0) / QE
        errs[nv] = eps / want - 1
        print(f"nv={nv}: <eps> = {eps:.6f} eV, closed form {want:.6f} eV, rel {errs[nv]:.2e}")
    assert abs(errs[256]) <= 2e-3
    assert 3.5 <= errs[128] / errs[256] <= 4.5        # second order in the node spacing


def test_weak_field_limit_is_the_fixed_f0_model(oracle_lib):
    O = oracle_lib
    t = np.arange(3000) * DT
    pl = O.params(vgrid="speed3d", nv=64, te_ev=1.0, vmax_vth=6.0, nu0=2e9, nu_model="nsv")
    d = {}
    for amp in (1e3, 5e2):
        E = amp * np.sin(2 * np.pi * 1e10 * t)
        Jl, _ = O.kinetic_drive(pl, DT, N, E)
        Je, _, _, _ = _drive(O, E, nv=64, vmax_vth=6.0, nu0=2e9, nu_model="nsv", mass_ratio=0.0)
        d[amp] = np.abs(Je - Jl).max() / np.abs(Jl).max()
    print(f"relative J difference evolving vs fixed F0: {d}")
    assert d[1e3] <= 1e-5 and 3.8 <= d[1e3] / d[5e2] <= 4.2


def test_field_run_energy_balance_per_cell(oracle_lib):
    """Coupled collision-free 1-D run: in every plasma cell the electron
    energy gained equals the work sum_n E^n (J^{n-1/2} + J^{n+1/2}) / 2 dt done
    by the field that cell saw, and the particle number of the F0 correction
    stays zero."""
    from fdtd_inputs import spec_1d_slab
    from tests.adapters import oracle_sim
    spec = spec_1d_slab(nz=600, slab=(250, 330), src_k=60, precision="f64", steps=900, nv=48)
    spec["source"]["amp"] = 3e4
    spec["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=0.0)
    sim = oracle_sim(oracle_lib, spec)
    cells = sim.slot_cells()
    work = np.zeros(cells.size)
    jprev = np.zeros(cells.size)
    for _ in range(900):
        e = sim.get("ex")[cells]
        sim.step(1)
        j = sim.get("j")
        work += e * 0.5 * (j + jprev) * sim.dt
        jprev = j
    g = sim.get("f0")
    t = oracle_lib.vtables(sim.p, sim.dt)
    v = t["v"]
    shell = 4 * np.pi * v ** 2 * (2 * v[0])
    assert np.abs(g @ shell).max() <= 1e-14 * np.abs(g).max() * shell.max() * len(v)
    dens = spec["plasma"]["density"][cells]
    gain = dens * (g @ (0.5 * ME * v ** 2 * shell))
    assert work.max() > 0
    err = np.abs(gain - work).max() / np.abs(work).max()
    print(f"per-cell energy balance: max |gain - work| / max work = {err:.2e}")
    assert err <= 1e-5
