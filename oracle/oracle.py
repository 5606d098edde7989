"""ctypes front end of the FP64 CPU oracle (``fdtd_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` import this module.  The product
library never loads it, and it imports nothing from the product package.

The oracle is a plain FP64 transcription of the coupled Yee-FDTD + two-term
kinetic electron step of arXiv 2211.05647 (Sec. 2 Eq. 1-12 for the fields and
CPML, Sec. 5.2 Eq. 20-24 and the printed f_1x / Jx update for the plasma).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

FIELDS = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5, "j": 6, "df": 7, "f0": 8}
VGRID = {"signed1d": 0, "cart2d": 1, "speed3d": 2}
SRC = {"none": 0, "gauss_sine": 1, "gauss": 2}
NU = {"nsv": 0, "const": 1, "table": 2}
F0 = {"maxwell": 0, "druyvesteyn": 1}


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction);
    omp=True builds the all-core variant of the same source (-fopenmp: the
    per-cell and per-slot loops shared among threads, results identical)."""
    os.makedirs(_BUILD, exist_ok=True)
    lib = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11"] +
                              (["-fopenmp"] if omp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class Params(ctypes.Structure):
    """Mirror of ``or_params`` (every member is 8 bytes)."""
    _fields_ = [
        ("ndim", ctypes.c_int64), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
        ("dx", ctypes.c_double), ("courant", ctypes.c_double),
        ("cpml", ctypes.c_int64),
        ("cpml_order", ctypes.c_double), ("cpml_sigma_factor", ctypes.c_double),
        ("cpml_kappa_max", ctypes.c_double), ("cpml_alpha_min", ctypes.c_double),
        ("cpml_alpha_max", ctypes.c_double),
        ("mur", ctypes.c_int64),
        ("src_kind", ctypes.c_int64),
        ("src_amp", ctypes.c_double), ("src_fc", ctypes.c_double), ("src_tau", ctypes.c_double),
        ("src_t0", ctypes.c_double),
        ("src_i", ctypes.c_int64), ("src_j", ctypes.c_int64), ("src_k", ctypes.c_int64),
        ("src_sheet", ctypes.c_int64),
        ("sheet_i0", ctypes.c_int64), ("sheet_i1", ctypes.c_int64),
        ("sheet_j0", ctypes.c_int64), ("sheet_j1", ctypes.c_int64),
        ("vgrid", ctypes.c_int64), ("nv", ctypes.c_int64), ("nv_perp", ctypes.c_int64),
        ("te_ev", ctypes.c_double), ("vmax_vth", ctypes.c_double), ("nu0", ctypes.c_double),
        ("nu_model", ctypes.c_int64), ("nonlinear", ctypes.c_int64),
        ("f0_model", ctypes.c_int64), ("s_n", ctypes.c_int64),
        ("s_speed", ctypes.POINTER(ctypes.c_double)), ("s_sigma", ctypes.POINTER(ctypes.c_double)),
        ("evolve_f0", ctypes.c_int64), ("mass_ratio", ctypes.c_double), ("tg_ev", ctypes.c_double),
    ]


def _load(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is not None:
            return _lib_omp if omp else _lib
        lib = ctypes.CDLL(build(omp=omp))
        P = ctypes.POINTER(Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.or_create.restype = vp
        lib.or_create.argtypes = [P, dp]
        lib.or_destroy.argtypes = [vp]
        lib.or_dt.restype = ctypes.c_double
        lib.or_dt.argtypes = [vp]
        for fn in ("or_nslots", "or_nnode", "or_steps_done"):
            getattr(lib, fn).restype = ctypes.c_int64
            getattr(lib, fn).argtypes = [vp]
        lib.or_field_len.restype = ctypes.c_int64
        lib.or_field_len.argtypes = [vp, ctypes.c_int]
        lib.or_slot_cells.argtypes = [vp, ip]
        lib.or_get.restype = ctypes.c_int
        lib.or_get.argtypes = [vp, ctypes.c_int, dp]
        lib.or_set.restype = ctypes.c_int
        lib.or_set.argtypes = [vp, ctypes.c_int, dp]
        lib.or_step.argtypes = [vp, ctypes.c_int64]
        lib.or_diag.argtypes = [vp, dp]
        lib.or_vtables.argtypes = [P, ctypes.c_double] + [dp] * 8
        lib.or_nnode_of.restype = ctypes.c_int64
        lib.or_nnode_of.argtypes = [P]
        lib.or_cpml_profile.argtypes = [P, ctypes.c_double, ctypes.c_int64, ctypes.c_int, dp, dp, dp]
        lib.or_source.restype = ctypes.c_double
        lib.or_source.argtypes = [P, ctypes.c_double]
        lib.or_kinetic_drive.argtypes = [P, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int64, dp, dp, dp]
        lib.or_poynting.argtypes = [vp, ip, dp]
        lib.or_threads.restype = ctypes.c_int64
        lib.or_threads.argtypes = []
        if omp:
            _lib_omp = lib
        else:
            _lib = lib
        return lib


def threads(omp: bool = False) -> int:
    """Threads the step loops of the (all-core) build use."""
    return int(_load(omp).or_threads())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


DEFAULTS = dict(
    ndim=1, nx=1, ny=1, nz=1, dx=1e-3, courant=0.5,
    cpml=0, cpml_order=3.0, cpml_sigma_factor=1.3, cpml_kappa_max=7.0, cpml_alpha_min=0.0,
    cpml_alpha_max=0.05,
    mur=0, src_kind=0, src_amp=1.0, src_fc=0.0, src_tau=1.0, src_t0=0.0,
    src_i=0, src_j=0, src_k=0, src_sheet=0, sheet_i0=0, sheet_i1=0, sheet_j0=0, sheet_j1=0,
    vgrid=0, nv=64, nv_perp=1, te_ev=1.0, vmax_vth=6.0, nu0=0.0, nu_model=0, nonlinear=0,
    f0_model=0, s_table=None, evolve_f0=0, mass_ratio=0.0, tg_ev=0.0,
)


def params(**kw) -> Params:
    """Build an ``or_params`` from keyword arguments (names of the C struct);
    string values are accepted for ``vgrid``, ``src_kind`` and ``nu_model``."""
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(f"unknown oracle parameter {k!r}")
        if k == "vgrid" and isinstance(v, str):
            v = VGRID[v]
        if k == "src_kind" and isinstance(v, str):
            v = SRC[v]
        if k == "nu_model" and isinstance(v, str):
            v = NU[v]
        if k == "f0_model" and isinstance(v, str):
            v = F0[v]
        d[k] = v
    if d["evolve_f0"] and d["vgrid"] != 2:
        raise ValueError("evolve_f0 needs the speed grid (vgrid 'speed3d')")
    p = Params()
    table = d.pop("s_table")
    for k, v in d.items():
        setattr(p, k, v)
    if table is not None:
        sp = np.ascontiguousarray(table[0], dtype=np.float64)
        sg = np.ascontiguousarray(table[1], dtype=np.float64)
        if sp.size != sg.size or sp.size < 2 or np.any(np.diff(sp) <= 0):
            raise ValueError("s_table: two arrays of equal length >= 2, speeds strictly ascending")
        p._keep = (sp, sg)          # the C side holds raw pointers into these
        p.s_n = sp.size
        p.s_speed = sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.s_sigma = sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    elif d["nu_model"] == 2:
        raise ValueError("nu_model 'table' needs s_table=(speeds, sigma)")
    return p


class Sim:
    """One oracle simulation.  ``density`` lives on the polarisation E nodes:
    length nz+1 (1-D Ex), nx*ny (2-D Ez) or nx*ny*nz (3-D Ex), x fastest."""

    def __init__(self, p: Params, density: np.ndarray | None = None, omp: bool = False):
        self._lib = _load(omp)
        self.p = p
        self._dens = None if density is None else np.ascontiguousarray(density, dtype=np.float64).ravel()
        self._h = self._lib.or_create(ctypes.byref(p), None if self._dens is None else _dp(self._dens))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def dt(self) -> float:
        return self._lib.or_dt(self._h)

    @property
    def nslots(self) -> int:
        return self._lib.or_nslots(self._h)

    @property
    def nnode(self) -> int:
        return self._lib.or_nnode(self._h)

    @property
    def steps_done(self) -> int:
        return self._lib.or_steps_done(self._h)

    def slot_cells(self) -> np.ndarray:
        out = np.zeros(max(self.nslots, 1), np.int64)
        self._lib.or_slot_cells(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return out[: self.nslots]

    def _len(self, which: int) -> int:
        if which == 6:
            return self.nslots
        if which in (7, 8):
            return self.nslots * self.nnode
        return self._lib.or_field_len(self._h, which)

    def get(self, name: str) -> np.ndarray:
        w = FIELDS[name]
        n = self._len(w)
        out = np.zeros(max(n, 1), np.float64)
        if n and self._lib.or_get(self._h, w, _dp(out)) != 0:
            raise ValueError(name)
        out = out[:n]
        return out.reshape(self.nslots, self.nnode) if name in ("df", "f0") else out

    def set(self, name: str, arr: np.ndarray):
        w = FIELDS[name]
        a = np.ascontiguousarray(arr, dtype=np.float64).ravel()
        if a.size != self._len(w):
            raise ValueError(f"{name}: expected {self._len(w)} values, got {a.size}")
        if self._lib.or_set(self._h, w, _dp(a)) != 0:
            raise ValueError(name)

    def step(self, n: int = 1):
        self._lib.or_step(self._h, int(n))

    def poynting(self, box) -> np.ndarray:
        """Power through the faces of box (i0, i1, j0, j1, k0, k1): [x0, x1, y0, y1, z0, z1, net outward]."""
        b = np.ascontiguousarray(box, dtype=np.int64)
        out = np.zeros(7)
        self._lib.or_poynting(self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
        return out

    def diag(self) -> dict:
        out = np.zeros(6)
        self._lib.or_diag(self._h, _dp(out))
        return dict(energy=out[0], number=out[1], number_max_cell=out[2], number_abs=out[3],
                    finite=bool(out[4]), energy_plain=out[5])


def vtables(p: Params, dt: float) -> dict:
    lib = _load()
    n = lib.or_nnode_of(ctypes.byref(p))
    arrs = [np.zeros(n) for _ in range(8)]
    lib.or_vtables(ctypes.byref(p), dt, *[_dp(a) for a in arrs])
    return dict(zip(["v", "w", "f0", "f0p", "nu", "dV", "alpha", "beta"], arrs))


def cpml_profile(p: Params, dt: float, n: int, at_h: bool) -> dict:
    lib = _load()
    b, a, k = np.zeros(n), np.zeros(n), np.zeros(n)
    lib.or_cpml_profile(ctypes.byref(p), dt, n, int(at_h), _dp(b), _dp(a), _dp(k))
    return dict(b=b, a=a, kappa=k)


def source(p: Params, t: float) -> float:
    return _load().or_source(ctypes.byref(p), float(t))


def kinetic_drive(p: Params, dt: float, density: float, E: np.ndarray, with_f0: bool = False):
    """0-D plasma cell driven by E^m; returns (J^{m+1/2} series, final delta f
    row), and the final F0 correction row when with_f0."""
    lib = _load()
    E = np.ascontiguousarray(E, dtype=np.float64)
    n = lib.or_nnode_of(ctypes.byref(p))
    J = np.zeros(E.size)
    df = np.zeros(n)
    g = np.zeros(n)
    lib.or_kinetic_drive(ctypes.byref(p), dt, density, _dp(E), E.size, _dp(J), _dp(df), _dp(g))
    return (J, df, g) if with_f0 else (J, df)


def port_spectra(sims, ports, freqs, steps: int) -> list:
    """Running DFT at ports (Sec. 5.3: the slab's S-parameters come from port
    spectra).  Steps every simulation in sims `steps` times; after step n the
    polarisation field E^n at t_n = n dt, averaged over each port's node
    indices, is accumulated into X[p, f] = sum_n E_p(t_n) exp(-i 2 pi f t_n) dt.
    Returns one complex array [nports, nfreq] per simulation."""
    freqs = np.asarray(freqs, dtype=np.float64)
    comp = {1: "ex", 2: "ez", 3: "ex"}
    out = []
    for sim in sims:
        X = np.zeros((len(ports), freqs.size), dtype=np.complex128)
        name = comp[int(sim.p.ndim)]
        dt = sim.dt
        for _ in range(steps):
            sim.step(1)
            t = sim.steps_done * dt
            e = sim.get(name)
            phase = np.exp(-2j * np.pi * freqs * t) * dt
            for q, cells in enumerate(ports):
                X[q] += np.mean(e[np.asarray(cells, dtype=np.int64)]) * phase
        out.append(X)
    return out

