"""Workload recipes (see the package docstring for the spec format).

Scales: free-space wavelength lam0 = 3 cm (f0 = c/lam0 ~ 9.99 GHz).  The
source pulse keeps the ratios of the paper's Table 3 pulse (f_c tau = 0.96,
t0 / tau = 4.52) at f_c = f0.  Densities are given through w_p / w0, i.e.
n = (w_p / w0)^2 n_c(w0) with n_c = eps0 m w0^2 / e^2.
"""
from __future__ import annotations

import numpy as np

C0 = 299792458.0
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12
LAM0 = 0.03
F0 = C0 / LAM0
OMEGA0 = 2 * np.pi * F0


def critical_density(omega: float = OMEGA0) -> float:
    """n such that the plasma frequency equals omega (input scaling only)."""
    return EPS0 * ME * omega * omega / (QE * QE)


def pulse_params(fc: float = F0, paper_absolute: bool = False) -> dict:
    """Gaussian-modulated sine with Table 3's shape: tau = 0.96 / f_c,
    t0 = 4.52 tau (or the paper's absolute 20 GHz / 48 ps / 217 ps)."""
    if paper_absolute:
        return dict(kind="gauss_sine", fc=20e9, tau=48e-12, t0=217e-12, amp=1.0)
    tau = 0.96 / fc
    return dict(kind="gauss_sine", fc=fc, tau=tau, t0=4.52 * tau, amp=1.0)


def gaussian_random_field(shape, corr_cells: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance Gaussian random field: white noise filtered (FFT,
    periodic) by a Gaussian kernel of ``corr_cells`` correlation length."""
    noise = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n) for n in shape]
    K2 = sum(np.meshgrid(*[k ** 2 for k in ks], indexing="ij"))
    filt = np.exp(-0.5 * (2 * np.pi * corr_cells) ** 2 * K2)
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    return f / f.std()


def cylinder_density(nx: int, ny: int, cx: float, cy: float, R: float, n_peak: float, seed: int,
                     corr: float = 16.0, ripple: float = 0.2) -> np.ndarray:
    """Seeded Gaussian density in a cylinder (2-D TMz, on Ez nodes, x fastest):
    n = n_pk exp(-r^2 / 2 s^2) (1 + ripple xi), s = R/2, clipped at 0,
    rescaled to max n_pk, zero for r > R; xi a unit Gaussian random field of
    ``corr``-cell correlation length drawn from numpy's PCG64(seed)."""
    rng = np.random.default_rng(seed)
    x0, x1 = max(int(np.floor(cx - R)) - 1, 0), min(int(np.ceil(cx + R)) + 2, nx)
    y0, y1 = max(int(np.floor(cy - R)) - 1, 0), min(int(np.ceil(cy + R)) + 2, ny)
    j, i = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    r2 = (i - cx) ** 2 + (j - cy) ** 2
    pad = int(4 * corr)
    xi = gaussian_random_field((y1 - y0 + 2 * pad, x1 - x0 + 2 * pad), corr, rng)[pad:-pad, pad:-pad]
    s = R / 2.0
    box = np.exp(-r2 / (2 * s * s)) * (1.0 + ripple * xi)
    box = np.clip(box, 0.0, None)
    box[r2 > R * R] = 0.0
    box *= n_peak / box.max()
    out = np.zeros((ny, nx))
    out[y0:y1, x0:x1] = box
    return out.ravel()


def random_state(sizes: dict, seed: int, e_scale: float = 1.0) -> dict:
    """Seeded random fields (E ~ N(0, e_scale), H ~ N(0, e_scale / eta0)) for
    state-parity checks; ``sizes`` maps field name -> length."""
    rng = np.random.default_rng(seed)
    eta0 = 376.730313668
    return {k: rng.standard_normal(n) * (e_scale if k.startswith("e") else e_scale / eta0)
            for k, n in sizes.items()}


def cross_section_table(te_ev: float = 1.0, n: int = 24, vmax_vth: float = 8.0, seed: int = 7):
    """Synthetic elastic cross-section s(v) for the tabulated collision law: a
    smooth positive curve with a deep minimum near 0.6 v_th (the shape of a
    Ramsauer-Townsend minimum) rising to a broad maximum, sampled at n
    ascending speeds from 0 to vmax_vth v_th, with seeded +-5 % jitter of the
    sample values.  Returns (speeds in m/s, s in arbitrary units): only the
    shape enters nu = N s(v) v, whose mean is fixed separately."""
    rng = np.random.default_rng(seed)
    vth = np.sqrt(QE * te_ev / ME)
    u = np.linspace(0.0, vmax_vth, n)
    s = 0.05 + (u - 0.6) ** 2 * np.exp(-u / 2.5)
    s *= 1.0 + 0.05 * rng.uniform(-1.0, 1.0, n)
    return u * vth, s


def spec_1d_slab(nz=2000, ppw=40, slab=(1000, 1500), wp_w0=0.5, nu_w0=0.01, nv=64, src_k=100, steps=2000,
                 precision="f64", f_dtype=None, te_ev=1.0, nu_model="nsv", seed=1) -> dict:
    """1-D FDTD + kinetic: uniform slab on E nodes slab[0]..slab[1]-1, Mur ends,
    soft source at node src_k, signed 1-D velocity grid +-6 v_th."""
    dens = np.zeros(nz + 1)
    dens[slab[0]:slab[1]] = wp_w0 ** 2 * critical_density()
    if f_dtype is None:
        f_dtype = "f64" if precision == "f64" else "f32"
    return dict(
        name=f"1d_slab_nz{nz}",
        grid=dict(ndim=1, nx=1, ny=1, nz=nz, dx=LAM0 / ppw, courant=0.5, cpml_cells=0, mur=1, precision=precision),
        source=dict(location="point", i=0, j=0, k=src_k, **pulse_params()),
        plasma=dict(density=dens, vgrid="signed1d", nv=nv, nv_perp=1, te_ev=te_ev, vmax_vth=6.0,
                    nu0=nu_w0 * OMEGA0, nu_model=nu_model, f_dtype=f_dtype, seed=seed),
        steps=steps)


def spec_2d_cylinder(n=4096, ny=None, ppw=20, cpml=10, R=512, center=None, src=None, wp_w0=0.8, nu_w0=0.01,
                     nv=32, nv_perp=32, steps=2000, precision="f32", f_dtype="f32", seed=20221112,
                     density_seed=None) -> dict:
    """2-D TMz FDTD + kinetic: seeded Gaussian-density cylinder, line source
    (one Ez node), Cartesian (v_par, v_perp) velocity grid."""
    nx = n
    ny = n if ny is None else ny
    if center is None:
        center = (nx / 2, ny / 2)
    if src is None:
        src = (nx // 4, ny // 2)
    dseed = seed if density_seed is None else density_seed
    dens = cylinder_density(nx, ny, center[0], center[1], R, wp_w0 ** 2 * critical_density(), dseed)
    return dict(
        name=f"2d_tmz_{nx}x{ny}",
        grid=dict(ndim=2, nx=nx, ny=ny, nz=1, dx=LAM0 / ppw, courant=0.5, cpml_cells=cpml, mur=0,
                  precision=precision),
        source=dict(location="point", i=int(src[0]), j=int(src[1]), k=0, **pulse_params()),
        plasma=dict(density=dens, vgrid="cart2d", nv=nv, nv_perp=nv_perp, te_ev=1.0, vmax_vth=6.0,
                    nu0=nu_w0 * OMEGA0, nu_model="nsv", f_dtype=f_dtype, seed=seed),
        steps=steps)


def spec_3d_slab(n=512, ny=None, nz=None, ppw=20, cpml=8, slab=(192, 320), src_k=24, wp_w0_max=1.2, nu_w0=0.005,
                 nv=32, steps=1000, precision="f32", f_dtype="bf16", seed=20221113) -> dict:
    """3-D Yee FDTD + kinetic: soft Ex sheet on plane src_k over the interior
    (non-CPML) x-y region, slab of planes slab[0] <= k < slab[1] with density
    rising linearly in z to (wp_w0_max)^2 n_c, signed 1-D velocity grid along x."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    nmax = wp_w0_max ** 2 * critical_density()
    prof = np.zeros(nz)
    k0, k1 = slab
    prof[k0:k1] = nmax * (np.arange(k0, k1) - k0 + 1) / (k1 - k0)
    dens = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).ravel()
    return dict(
        name=f"3d_slab_{nx}x{ny}x{nz}",
        grid=dict(ndim=3, nx=nx, ny=ny, nz=nz, dx=LAM0 / ppw, courant=0.5, cpml_cells=cpml, mur=0,
                  precision=precision),
        source=dict(location="sheet", i=0, j=0, k=src_k, i0=cpml, i1=nx - cpml, j0=cpml, j1=ny - cpml,
                    **pulse_params()),
        plasma=dict(density=dens, vgrid="signed1d", nv=nv, nv_perp=1, te_ev=1.0, vmax_vth=6.0,
                    nu0=nu_w0 * OMEGA0, nu_model="nsv", f_dtype=f_dtype, seed=seed),
        steps=steps)


def batch_runs_1d(nruns=256, seed=20221114, nz_range=(1024, 65536), slab_frac=(0.2, 0.6), wp_w0=(0.1, 1.5),
                  log_nu_w0=(-3.0, -1.0), nv=64, ppw=40, f_dtype="f32", precision="f32", src_k=100, steps=5000):
    """Independent 1-D slab runs of uneven size: nz uniform on nz_range, a
    centred slab of uniform density covering a uniform fraction of the grid,
    w_p/w0 uniform, nu/w0 log-uniform, Mur ends, source at node src_k."""
    rng = np.random.default_rng(seed)
    specs = []
    for r in range(nruns):
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        frac = rng.uniform(*slab_frac)
        w = rng.uniform(*wp_w0)
        nu = 10.0 ** rng.uniform(*log_nu_w0)
        half = int(frac * nz / 2)
        s = spec_1d_slab(nz=nz, ppw=ppw, slab=(nz // 2 - half, nz // 2 + half), wp_w0=w, nu_w0=nu, nv=nv,
                         src_k=min(src_k, nz // 4), steps=steps, precision=precision, f_dtype=f_dtype, seed=seed + r)
        specs.append(s)
    return specs


def spec_closure_8192(steps=4000, seed=20221115):
    """Learned-closure comparison grid: 2-D TMz 8192^2, dx = lam0/20, the
    4096^2 cylinder recipe scaled x2 (radius 1024, centre 4096^2, source at
    (2048, 4096)) with peak w_p/w0 = 0.9, above the 0.8 of the training runs,
    so the densest core keeps the kinetic update."""
    return spec_2d_cylinder(n=8192, R=1024, wp_w0=0.9, steps=steps, seed=seed)


def closure_training_specs(k=3, steps=2000, seed0=20221200):
    """Kinetic training runs: the 4096^2 cylinder recipe with k density seeds."""
    return [spec_2d_cylinder(steps=steps, seed=seed0 + i) for i in range(k)]


# The benchmark workloads (full sizes) by name, plus reduced profiling cases
def _evolving(spec: dict) -> dict:
    spec["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=1.37e-5, tg_ev=0.026)
    return spec


WORKLOADS = {
    "1d_slab_fp64": lambda: spec_1d_slab(),
    "1d_slab_fp32": lambda: spec_1d_slab(precision="f32"),
    "2d_tmz_4096_kinetic": lambda: spec_2d_cylinder(),
    "2d_tmz_4096_kinetic_bf16": lambda: spec_2d_cylinder(f_dtype="bf16"),
    "3d_512_kinetic_bf16": lambda: spec_3d_slab(),
    "3d_512_kinetic_f32": lambda: spec_3d_slab(f_dtype="f32"),
    # profiling cases: same recipes at half the lengths (inputs still larger than L2)
    "2d_tmz_2048_kinetic": lambda: spec_2d_cylinder(n=2048, R=256),
    "3d_256_kinetic_bf16": lambda: spec_3d_slab(n=256, slab=(96, 160), src_k=12),
    # evolving isotropic F0 on the speed grid (Joule heating + elastic collisions with argon, m/M = 1.37e-5,
    # gas at 0.026 eV), FP32 delta f
    "3d_256_f0evolve_f32": lambda: _evolving(spec_3d_slab(n=256, slab=(96, 160), src_k=12, f_dtype="f32")),
    "2d_tmz_8192_closure": lambda: spec_closure_8192(),
    # inference cost of the closure on every plasma cell of the 2048^2 cylinder (seeded random weights)
    "2d_tmz_2048_closure_cost": lambda: spec_2d_cylinder(n=2048, R=512),
    "batch1d_256_f32": lambda: batch_runs_1d(),
    "batch1d_256_bf16": lambda: batch_runs_1d(f_dtype="bf16"),
}
