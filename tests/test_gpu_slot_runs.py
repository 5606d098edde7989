"""Slot runs (FDTD_OPT_SLOT_RUNS): where the plasma is piecewise uniform
(consecutive cells of one stored density), the register kinetic kernel takes
each row's cell and density from its run instead of the per-slot arrays.
The update (Sec. 5.2, Eq. 22 and 24) is the same arithmetic on the same
values, so every row, J and field is identical bit for bit with runs on and
off; the run count follows from the density layout (one run per plasma plane
of the 3-D slab whose density rises plane by plane, one per row of a uniform
2-D rectangle, none for a smooth profile)."""
import copy

import numpy as np
import pytest

from fdtd_inputs import critical_density, spec_1d_slab, spec_2d_cylinder, spec_3d_slab
from tests.adapters import FIELDS

pytestmark = pytest.mark.gpu


def _rect_2d(nx=300, ny=220, x=(40, 150), y=(30, 200), f_dtype="f32"):
    """2-D TMz grid with a uniform rectangle of plasma: one run per grid row."""
    spec = spec_2d_cylinder(n=nx, ny=ny, R=10, center=(nx / 2, ny / 2), src=(20, ny // 2), nv=8, nv_perp=8,
                            steps=1, f_dtype=f_dtype, seed=21)
    d = np.zeros((ny, nx))
    d[y[0]:y[1], x[0]:x[1]] = 0.5 * critical_density()
    spec["plasma"]["density"] = d.ravel()
    return spec


def _run(spec, runs, steps, shape=None):
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("slot_runs", runs)
    if shape is not None:
        s.set_option("kinetic_shape", shape[0] * 10**6 + shape[1] * 1000)
    nr = s.launch_shapes()["slot_runs"]
    s.step(steps)
    out = {n: s.read(n, device=False).copy() for n in FIELDS[spec["grid"]["ndim"]] + ["j", "df"]}
    s.close()
    return nr, out


CASES = {
    # density rising plane by plane over 40 planes: 40 runs of 62 x 46 cells
    "3d_slab_bf16": (lambda: spec_3d_slab(n=62, ny=47, nz=80, cpml=6, slab=(20, 60), src_k=8, nv=32, steps=1),
                     40, [(2, 2), (4, 1), (1, 4)]),
    "3d_slab_f32": (lambda: spec_3d_slab(n=62, ny=47, nz=80, cpml=6, slab=(20, 60), src_k=8, nv=32, steps=1,
                                         f_dtype="f32"), 40, [(4, 2), (2, 4)]),
    # one uniform slab: a single run
    "1d_slab": (lambda: spec_1d_slab(nz=900, slab=(300, 620), src_k=60, nv=64, precision="f32", steps=1, seed=5),
                1, [(4, 4), (16, 1)]),
    # 170 rows of 110 cells: many short runs, rows of a warp straddle their ends
    "2d_rect": (lambda: _rect_2d(), 170, [(4, 4), (2, 8), (16, 1)]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_slot_runs_equal_per_slot_arrays(case):
    make, want_runs, shapes = CASES[case]
    spec = make()
    for shape in shapes:
        try:
            n_on, on = _run(spec, 1, 25, shape)
        except Exception as e:      # not a candidate shape of this row length
            if "candidate" in str(e):
                continue
            raise
        n_off, off = _run(spec, 0, 25, shape)
        assert n_on == want_runs and n_off == 0, (case, n_on, n_off)
        for k, v in off.items():
            assert np.array_equal(on[k], v), (case, shape, k)
        assert np.count_nonzero(on["j"]) > 0


def test_smooth_profile_has_no_runs():
    spec = spec_2d_cylinder(n=160, ny=120, R=30, center=(95, 60), src=(50, 60), steps=1, seed=2)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    assert s.launch_shapes()["slot_runs"] == 0        # the seeded Gaussian density differs cell to cell
    s.close()
    spec3 = copy.deepcopy(CASES["3d_slab_bf16"][0]())
    s3 = Solver.from_spec(spec3)
    assert s3.launch_shapes()["slot_runs"] == 40
    s3.set_option("slot_runs", 0)
    assert s3.launch_shapes()["slot_runs"] == 0
    s3.set_option("slot_runs", 1)
    assert s3.launch_shapes()["slot_runs"] == 40
    s3.close()
