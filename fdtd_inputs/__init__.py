"""Seeded synthetic workloads: grid sizes, source placement and density
fields shaped like the paper's problems (Sec. 5.3 plasma slab, Table 3
pulse) at the sizes of the benchmark configurations.

This module holds no part of the method's arithmetic (no field update,
CPML profile, velocity table or collision model): it only describes inputs,
as plain dicts, so that the oracle, the CUDA path, the tests and the
benchmark all consume the same arrays.

Spec format (consumed by ``paper_2211_05647_gb300.Solver.from_spec`` and by
the tests' oracle adapter):
    {"grid":   {ndim, nx, ny, nz, dx, courant, cpml_cells, mur, precision},
     "source": {kind, location, amp, fc, tau, t0, i, j, k, i0, i1, j0, j1},
     "plasma": {density (float64 array on the polarisation nodes), vgrid, nv,
                nv_perp, te_ev, vmax_vth, nu0, nu_model, f_dtype, seed}
               or None,
     "steps":  int, "name": str}
"""
from .workloads import (C0, LAM0, F0, OMEGA0, QE, ME, EPS0, critical_density, pulse_params,
                        cylinder_density, gaussian_random_field, spec_1d_slab, spec_2d_cylinder,
                        spec_3d_slab, random_state, batch_runs_1d, spec_closure_8192, closure_training_specs,
                        cross_section_table, WORKLOADS)

__all__ = ["C0", "LAM0", "F0", "OMEGA0", "QE", "ME", "EPS0", "critical_density", "pulse_params",
           "cylinder_density", "gaussian_random_field", "spec_1d_slab", "spec_2d_cylinder", "spec_3d_slab",
           "random_state", "batch_runs_1d", "spec_closure_8192",
           "closure_training_specs", "cross_section_table", "WORKLOADS"]
