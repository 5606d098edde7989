"""Evolving isotropic F0 (speed grid) on the GPU, through the C ABI, against
the FP64 oracle: fields, J, delta f and the F0 correction rows."""
import numpy as np
import pytest

from fdtd_inputs import spec_1d_slab, spec_3d_slab
from tests.adapters import compare, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _spec_1d(prec, nv=48, steps=900):
    spec = spec_1d_slab(nz=600, slab=(250, 330), src_k=60, precision=prec, steps=steps, nv=nv)
    spec["source"]["amp"] = 3e4
    spec["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=1e-3, tg_ev=0.05)
    return spec


def _run_pair(oracle_lib, spec, steps):
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    sim = oracle_sim(oracle_lib, spec)
    s.step(steps)
    sim.step(steps)
    return s, sim


@pytest.mark.parametrize("prec,nv,tol,tol_f0", [("f64", 48, 1e-12, 1e-11), ("f32", 48, 1e-4, 2e-3),
                                                 ("f64", 160, 1e-12, 1e-11), ("f32", 31, 1e-4, 2e-3)])
def test_evolving_f0_1d_matches_oracle(oracle_lib, prec, nv, tol, tol_f0):
    """Rows of 48 and 31 nodes (padded to 64 / 32) run the vector kernel with
    16 / 8 / 32 lanes per row; 160 FP64 nodes (128 vectors) the one-warp-per-row
    kernel."""
    spec = _spec_1d(prec, nv=nv)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 1)
    g_ref = sim.get("f0")
    errs["f0"] = rel_l2(s.read("f0", device=False), g_ref)
    errs["df"] = rel_l2(s.read("df", device=False), sim.get("df"))
    print(f"evolving F0 1-D {prec} nv={nv}: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert np.abs(g_ref).max() > 0 and np.abs(sim.get("j")).max() > 0
    assert max(errs["ex"], errs["hy"], errs["j"]) <= tol, errs
    assert errs["df"] <= tol_f0 and errs["f0"] <= tol_f0, errs


def test_evolving_f0_3d_fp32(oracle_lib):
    spec = spec_3d_slab(n=36, ny=32, nz=56, cpml=6, slab=(26, 40), src_k=10, nv=24, steps=260, precision="f32",
                        f_dtype="f32", seed=23)
    spec["source"]["amp"] = 2e4
    spec["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=1e-3, tg_ev=0.05)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 3)
    errs["f0"] = rel_l2(s.read("f0", device=False), sim.get("f0"))
    print("evolving F0 3-D f32: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(v for k, v in errs.items() if k != "f0") <= 1e-4, errs
    assert errs["f0"] <= 2e-3


def test_evolving_f0_checkpoint_resume():
    from paper_2211_05647_gb300 import Solver
    spec = _spec_1d("f32", steps=600)
    a = Solver.from_spec(spec)
    a.step(300)
    blob = a.save_state(device=False)
    a.step(300)
    b = Solver.from_spec(spec)
    b.load_state(blob)
    b.step(300)
    for q in ("ex", "hy", "j", "df", "f0"):
        assert np.array_equal(a.read(q, device=False), b.read(q, device=False)), q


def test_evolving_f0_rejected_off_the_speed_grid():
    from paper_2211_05647_gb300 import FdtdError, Solver
    spec = _spec_1d("f32", steps=1)
    for bad in (dict(vgrid="signed1d"), dict(f_dtype="bf16"), dict(mass_ratio=-1.0)):
        sp = _spec_1d("f32", steps=1)
        sp["plasma"].update(bad)
        with pytest.raises(FdtdError):
            Solver.from_spec(sp)
    del spec
