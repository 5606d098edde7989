"""The all-core build of the oracle (the same source compiled with -fopenmp,
its per-cell and per-slot loops shared among threads) gives the single-thread
build's results bit for bit: each cell and slot is computed by the same
expressions in the same order, only by another thread."""
import numpy as np
import pytest

from fdtd_inputs import spec_1d_slab, spec_2d_cylinder, spec_3d_slab
from tests.adapters import oracle_sim


def _cases():
    f0 = spec_3d_slab(n=20, cpml=4, slab=(8, 12), src_k=5, f_dtype="f32", precision="f64")
    f0["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=1.37e-5, tg_ev=0.026)
    nl = spec_2d_cylinder(n=64, ny=48, R=12, center=(36, 24), src=(12, 24), precision="f64", f_dtype="f64")
    nl["plasma"]["nonlinear"] = 1
    return {
        "1d_slab": (spec_1d_slab(nz=600, slab=(300, 420), src_k=50), 400),
        "2d_cylinder_cpml": (spec_2d_cylinder(n=96, ny=80, R=18, center=(50, 40), src=(22, 40), precision="f64",
                                              f_dtype="f64"), 120),
        "2d_nonlinear": (nl, 120),
        "3d_slab_cpml": (spec_3d_slab(n=24, cpml=4, slab=(10, 16), src_k=6, precision="f64", f_dtype="f64"), 40),
        "3d_f0_evolution": (f0, 30),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_all_core_build_equals_single_thread(oracle_lib, name):
    O = oracle_lib
    O.build(omp=True)
    spec, steps = _cases()[name]
    a, b = oracle_sim(O, spec), oracle_sim(O, spec, omp=True)
    a.step(steps)
    b.step(steps)
    names = {1: ["ex", "hy"], 2: ["ez", "hx", "hy"], 3: ["ex", "ey", "ez", "hx", "hy", "hz"]}[spec["grid"]["ndim"]]
    names += ["j", "df"] + (["f0"] if spec["plasma"].get("evolve_f0") else [])
    assert np.abs(a.get("j")).max() > 0
    for n in names:
        assert np.array_equal(a.get(n), b.get(n)), n
    assert O.threads(omp=True) >= 1 and O.threads() == 1
