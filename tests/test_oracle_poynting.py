"""Pins of the oracle's Poynting flux through a box (the power diagnostic of
Sec. 2): E^n on the face planes, H time-centred at step n.

With that centring the Yee scheme has an exact discrete energy balance: the
power that crosses a closed surface, summed over steps times dt, equals the
change of the discrete field energy 1/2 eps0 E^n.E^n + 1/2 mu0 H^{n-1/2}.H^{n+1/2}
outside it.  The checks below therefore compare the time-integrated flux with
field energies summed directly from the oracle's fields (no Poynting code
involved), once the pulse has cleared the surface; a dropped time-centring, a
wrong face sign or a missing curl term breaks them by many orders of magnitude
more than the tolerance."""
import numpy as np
import pytest

from tests.physics import C0, EPS0

MU0 = 1.0 / (EPS0 * C0 ** 2)
DX = 1e-3


def _pulse(lam_cells):
    lam = lam_cells * DX
    tau = 0.96 * lam / C0
    return dict(src_kind="gauss_sine", src_fc=C0 / lam, src_tau=tau, src_t0=4.52 * tau)


def _energy(sim, ndim, sl):
    """Discrete field energy at the current step: (total, share on the nodes
    selected by sl).  Reads H^{n-1/2}, steps once for H^{n+1/2}."""
    ef = ["ex"] if ndim == 1 else ["ez"] if ndim == 2 else ["ex", "ey", "ez"]
    hf = ["hy"] if ndim == 1 else ["hx", "hy"] if ndim == 2 else ["hx", "hy", "hz"]
    E = {f: sim.get(f) for f in ef}
    H0 = {f: sim.get(f) for f in hf}
    sim.step(1)
    H1 = {f: sim.get(f) for f in hf}
    shp = {1: (-1,), 2: (sim.p.ny, sim.p.nx), 3: (sim.p.nz, sim.p.ny, sim.p.nx)}[ndim]
    dens = [EPS0 * E[f] ** 2 for f in ef] + [MU0 * H0[f] * H1[f] for f in hf]
    dV = 0.5 * DX ** ndim
    return (sum(np.sum(d) for d in dens) * dV, sum(np.sum(d.reshape(shp)[sl]) for d in dens) * dV)


def test_poynting_1d_plane_carries_pulse_energy(oracle_lib):
    """The energy that crossed the plane k0 equals the energy beyond it."""
    p = oracle_lib.params(ndim=1, nz=3000, dx=DX, mur=1, src_k=100, **_pulse(20))
    s = oracle_lib.Sim(p)
    k0 = 600
    acc = np.zeros(7)
    for _ in range(2600):
        acc += s.poynting([0, 0, 0, 0, k0, 2999]) * s.dt
        s.step(1)
    assert acc[4] > 0 and acc[5] == 0.0
    assert acc[6] == pytest.approx(-acc[4], rel=0, abs=0)
    ex = s.get("ex")
    assert np.abs(ex[k0 - 5:k0 + 5]).max() < 1e-9 * np.abs(ex).max()   # pulse has cleared the plane
    W = _energy(s, 1, slice(k0, None))[1]
    rel = abs(acc[4] / W - 1)
    print(f"1-D: flux x dt {acc[4]:.6e}, energy beyond {W:.6e}, rel {rel:.2e}")
    assert rel <= 1e-9


@pytest.mark.parametrize("ndim,n,half,T,lam", [(2, 300, 20, 100, 10), (3, 80, 10, 75, 8)])
def test_poynting_radiated_energy_leaves_box(oracle_lib, ndim, n, half, T, lam):
    """A point source at the centre of a box: the net outward energy equals
    the field energy outside the box after the pulse has left it."""
    c = n // 2
    kw = dict(ndim=ndim, nx=n, ny=n, nz=n if ndim == 3 else 1, dx=DX, src_i=c, src_j=c, src_k=c, **_pulse(lam))
    s = oracle_lib.Sim(oracle_lib.params(**kw))
    box = [c - half, c + half] * 2 + ([c - half, c + half] if ndim == 3 else [0, 0])
    steps = int(T * DX / C0 / s.dt)
    acc = np.zeros(7)
    for _ in range(steps):
        acc += s.poynting(box) * s.dt
        s.step(1)
    inner = tuple(slice(c - half + 1, c + half) for _ in range(ndim))
    Wall, Win = _energy(s, ndim, inner)
    rel = abs(acc[6] / (Wall - Win) - 1)
    print(f"{ndim}-D: net outward x dt {acc[6]:.6e}, energy outside {Wall - Win:.6e}, rel {rel:.2e}")
    assert Win < 1e-8 * Wall
    assert rel <= 1e-8
    # symmetry of the radiation about the source: equal and opposite face fluxes
    # along the axes normal to the source polarisation
    ax = (0, 1) if ndim == 2 else (1, 2)
    for a in ax:
        assert acc[2 * a + 1] > 0 and abs(acc[2 * a] + acc[2 * a + 1]) <= 1e-9 * acc[2 * a + 1]


def test_poynting_box_without_source_balances_energy_inside(oracle_lib):
    """A 2-D box beside the source, read while the cylindrical wave's wake is
    still crossing it: the net outward energy equals minus the field energy
    left inside (face nodes at half weight, corners at a quarter).  The
    balance is second order in dx while fields sit on the faces (H is averaged
    onto the face plane), hence the looser bound; the face towards the source
    sees the pulse enter (positive flux along +x)."""
    n = 300
    kw = dict(ndim=2, nx=n, ny=n, dx=DX, src_i=100, src_j=150, **_pulse(10))
    s = oracle_lib.Sim(oracle_lib.params(**kw))
    i0, i1, j0, j1 = 140, 180, 130, 170
    steps = int(130 * DX / C0 / s.dt)
    acc = np.zeros(7)
    for _ in range(steps):
        acc += s.poynting([i0, i1, j0, j1, 0, 0]) * s.dt
        s.step(1)
    assert acc[0] > 0 and acc[1] > 0
    I = np.arange(n)

    def node(a, lo, hi):
        return np.where((a > lo) & (a < hi), 1.0, np.where((a == lo) | (a == hi), 0.5, 0.0))

    def half(a, lo, hi):      # node at a + 1/2
        return ((a >= lo) & (a < hi)).astype(float)
    wE, wHx, wHy = (np.outer(node(I, j0, j1), node(I, i0, i1)), np.outer(half(I, j0, j1), node(I, i0, i1)),
                    np.outer(node(I, j0, j1), half(I, i0, i1)))
    ez, hx0, hy0 = (s.get(f).reshape(n, n) for f in ("ez", "hx", "hy"))
    s.step(1)
    hx1, hy1 = (s.get(f).reshape(n, n) for f in ("hx", "hy"))
    Win = 0.5 * DX ** 2 * (EPS0 * np.sum(wE * ez ** 2) + MU0 * np.sum(wHx * hx0 * hx1) + MU0 * np.sum(wHy * hy0 * hy1))
    rel = abs(acc[6] + Win) / acc[0]
    print(f"box beside the source: in {acc[0]:.4e}, net outward {acc[6]:.4e}, inside {Win:.4e}, rel {rel:.2e}")
    assert Win > 0.1 * acc[0]        # the wake is still there: the balance is not trivially 0 = 0
    assert rel <= 2e-3
