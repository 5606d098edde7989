"""Degenerate cases of the method against the FP64 oracle: a collisionless
plasma (nu = 0: undamped rows), the smallest signed velocity grid (2 nodes), a
single plasma cell, plasma on the first and last updated nodes, the smallest
grid (3 nodes), a batch of one run and a batch of vacuum runs."""
import numpy as np
import pytest

from fdtd_inputs import spec_1d_slab
from fdtd_inputs.workloads import critical_density
from tests.adapters import compare, oracle_sim

pytestmark = pytest.mark.gpu


def _dens(nz, nodes, wp_w0=0.5):
    d = np.zeros(nz + 1)
    d[list(nodes)] = wp_w0 ** 2 * critical_density()
    return d


def _cases():
    out = {}
    s = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, steps=700, nv=32)
    s["plasma"].update(nu_model="const", nu0=0.0)
    out["collisionless"] = s
    s = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, steps=700, nv=2)
    out["nv2"] = s
    s = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, steps=700, nv=32)
    s["plasma"]["density"] = _dens(400, [200])
    out["one_cell"] = s
    s = spec_1d_slab(nz=120, slab=(1, 119), src_k=60, steps=500, nv=16)
    s["plasma"]["density"] = _dens(120, [1, 119])
    out["end_nodes"] = s
    s = spec_1d_slab(nz=3, slab=(1, 3), src_k=1, steps=200, nv=16)
    s["plasma"]["density"] = _dens(3, [1, 2])
    out["nz3"] = s
    return out


@pytest.mark.parametrize("case", ["collisionless", "nv2", "one_cell", "end_nodes", "nz3"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-4)])
def test_degenerate_1d_matches_oracle(oracle_lib, case, prec, tol):
    from paper_2211_05647_gb300 import Solver
    spec = _cases()[case]
    spec["grid"]["precision"] = prec
    spec["plasma"]["f_dtype"] = prec
    s = Solver.from_spec(spec)
    s.step(spec["steps"])
    sim = oracle_sim(oracle_lib, spec)
    sim.step(spec["steps"])
    errs = compare(s, sim, 1)
    print(f"{case} {prec}: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert np.abs(sim.get("j")).max() > 0
    assert max(errs.values()) <= tol, errs


def test_batch_of_one_run_and_of_vacuum_runs(oracle_lib):
    from paper_2211_05647_gb300 import Batch
    one = spec_1d_slab(nz=600, slab=(250, 330), src_k=60, steps=800, nv=32)
    vac = [spec_1d_slab(nz=n, slab=(10, 20), src_k=30, steps=800, nv=32) for n in (300, 517)]
    for v in vac:
        v["plasma"]["density"] = np.zeros(v["grid"]["nz"] + 1)
    for specs in ([one], vac):
        b = Batch(specs)
        b.step(800)
        for r, sp in enumerate(specs):
            sim = oracle_sim(oracle_lib, sp)
            sim.step(800)
            e = np.linalg.norm(b.read(r, "ex") - sim.get("ex")) / np.linalg.norm(sim.get("ex"))
            assert e <= 1e-12, (r, e)
