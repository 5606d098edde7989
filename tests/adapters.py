"""Spec -> oracle adapter and comparison helpers for the parity tests.

A spec (see ``fdtd_inputs``) drives both sides: the oracle gets it through
``oracle_sim`` below, the CUDA path through ``Solver.from_spec``.
"""
from __future__ import annotations

import numpy as np

POL = {1: "ex", 2: "ez", 3: "ex"}
FIELDS = {1: ["ex", "hy"], 2: ["ez", "hx", "hy"], 3: ["ex", "ey", "ez", "hx", "hy", "hz"]}


def oracle_params(O, spec):
    g, s, p = spec["grid"], spec.get("source"), spec.get("plasma")
    kw = dict(ndim=g["ndim"], nx=g.get("nx", 1), ny=g.get("ny", 1), nz=g.get("nz", 1), dx=g["dx"],
              courant=g.get("courant", 0.5), cpml=g.get("cpml_cells", 0), mur=g.get("mur", 0))
    for k in ("cpml_order", "cpml_sigma_factor", "cpml_kappa_max", "cpml_alpha_min", "cpml_alpha_max"):
        if k in g:
            kw[k] = g[k]
    if s:
        kw.update(src_kind=s["kind"], src_amp=s.get("amp", 1.0), src_fc=s.get("fc", 0.0), src_tau=s["tau"],
                  src_t0=s.get("t0", 0.0), src_i=s.get("i", 0), src_j=s.get("j", 0), src_k=s.get("k", 0))
        if s.get("location") == "sheet":
            kw.update(src_sheet=1, sheet_i0=s["i0"], sheet_i1=s["i1"], sheet_j0=s["j0"], sheet_j1=s["j1"])
    if p is not None:
        kw.update(vgrid=p["vgrid"], nv=p["nv"], nv_perp=p.get("nv_perp", 1), te_ev=p.get("te_ev", 1.0),
                  vmax_vth=p.get("vmax_vth", 6.0), nu0=p.get("nu0", 0.0), nu_model=p.get("nu_model", "nsv"),
                  nonlinear=p.get("nonlinear", 0), f0_model=p.get("f0_model", "maxwell"),
                  s_table=p.get("s_table"), evolve_f0=p.get("evolve_f0", 0), mass_ratio=p.get("mass_ratio", 0.0),
                  tg_ev=p.get("tg_ev", 0.0))
    return O.params(**kw)


def oracle_sim(O, spec, omp: bool = False):
    p = spec.get("plasma")
    return O.Sim(oracle_params(O, spec), None if p is None else p["density"], omp=omp)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def compare(solver, sim, ndim, quantities=None):
    """Relative L2 error of every field component (and J) of the CUDA run
    against the oracle.  A component's error is normalised by the oracle norm
    of its whole field vector (all E components, or all H components): a
    component that is identically zero in exact arithmetic (Hx of an
    x-directed current, say) then reports rounding noise relative to the
    field, not relative to zero."""
    names = quantities or FIELDS[ndim] + (["j"] if sim.nslots else [])
    ref = {n: sim.get(n) for n in names}
    got = {n: np.asarray(solver.read(n, device=False), dtype=np.float64) for n in names}
    norm = {}
    for grp in ("e", "h"):
        members = [n for n in FIELDS[ndim] if n[0] == grp]
        norm[grp] = np.sqrt(sum(np.sum(sim.get(n) ** 2) for n in members))
    out = {}
    for n in names:
        den = norm[n[0]] if n[0] in ("e", "h") else np.linalg.norm(ref[n])
        out[n] = float(np.linalg.norm(got[n] - ref[n]) / den) if den > 0 else float(np.linalg.norm(got[n]))
    return out
