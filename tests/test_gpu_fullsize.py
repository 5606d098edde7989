"""Full-size parity: the benchmark's own workloads in the launch configuration
bench.py times (the autotuner runs first, as in the bench: on the 3-D grids it
selects the TMA column stencils), from a seeded random initial E/H state, a
few steps, against the FP64 oracle run at the same full size.  Every field
value and every J is compared (relative L2, field-vector normalisation)."""
import os

import numpy as np
import pytest

from fdtd_inputs import WORKLOADS, random_state
from tests.adapters import FIELDS, compare, oracle_sim

pytestmark = pytest.mark.gpu


def _mem_available_gb():
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable"):
                return int(ln.split()[1]) / 1e6
    except Exception:
        pass
    return 0.0


def _zero_pec(ndim, sizes, st):
    nx, ny, nz = sizes
    if ndim == 2:
        st["ez"].reshape(ny, nx)[0, :] = 0
        st["ez"].reshape(ny, nx)[:, 0] = 0
    else:
        ex, ey, ez = (st[n].reshape(nz, ny, nx) for n in ("ex", "ey", "ez"))
        ex[:, 0, :] = 0; ex[0] = 0
        ey[:, :, 0] = 0; ey[0] = 0
        ez[:, :, 0] = 0; ez[:, 0, :] = 0


@pytest.mark.parametrize("name,steps,tol,min_gb", [("2d_tmz_4096_kinetic", 4, 1e-5, 24),
                                                    ("3d_512_kinetic_bf16", 3, 5e-3, 80),
                                                    ("3d_256_kinetic_bf16", 3, 5e-3, 12),
                                                    ("3d_256_f0evolve_f32", 3, 1e-4, 14)])
def test_full_size_random_state(oracle_lib, name, steps, tol, min_gb, monkeypatch, tmp_path):
    if _mem_available_gb() < min_gb:
        pytest.skip(f"needs {min_gb} GB of host memory for the FP64 oracle at full size")
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    from paper_2211_05647_gb300 import Solver
    spec = WORKLOADS[name]()
    g = spec["grid"]
    nd = g["ndim"]
    n = g["nx"] * g["ny"] * (g["nz"] if nd == 3 else 1)
    st = random_state({f: n for f in FIELDS[nd]}, seed=99)
    _zero_pec(nd, (g["nx"], g["ny"], g["nz"]), st)
    s = Solver.from_spec(spec)
    s.autotune()
    shapes = s.launch_shapes()
    for f, v in st.items():
        s.write(f, v.astype(np.float32))
    sim = oracle_sim(oracle_lib, spec)
    for f, v in st.items():
        sim.set(f, v.astype(np.float32).astype(np.float64))   # same rounded start on both sides
    del st
    s.step(steps)
    sim.step(steps)
    errs = compare(s, sim, nd)
    if spec["plasma"].get("evolve_f0"):
        from tests.adapters import rel_l2
        errs["f0"] = rel_l2(s.read("f0", device=False), sim.get("f0"))
    print(f"{name} {shapes}: " + " ".join(f"{k}={v:.3e}" for k, v in errs.items()))
    assert sim.nslots == s.plasma_shape()[0] > 0
    assert max(v for k, v in errs.items() if k != "f0") <= tol, errs
    assert errs.get("f0", 0.0) <= 2e-3, errs


@pytest.mark.parametrize("name,tol", [("batch1d_256_f32", 1e-5), ("batch1d_256_bf16", 5e-3)])
def test_batch_full_size_random_state(oracle_lib, name, tol):
    """The 256-run batched workload as bench.py builds and launches it (same
    Batch construction, so the same cluster packing and row shapes), every run
    from a seeded random E/H state, 4 steps, against each run's FP64 oracle:
    fields of every run and J of every plasma slot."""
    if _mem_available_gb() < 8:
        pytest.skip("needs 8 GB of host memory for the FP64 oracle of 256 runs")
    from paper_2211_05647_gb300 import Batch
    specs = WORKLOADS[name]()
    b = Batch(specs)
    sims = []
    for r, sp in enumerate(specs):
        nz = sp["grid"]["nz"]
        st = random_state({"ex": nz + 1, "hy": nz}, seed=1000 + r)
        sim = oracle_sim(oracle_lib, sp)
        for f, v in st.items():
            v32 = v.astype(np.float32)
            b.write(r, f, v32)
            sim.set(f, v32.astype(np.float64))
        sims.append(sim)
    b.step(4)
    worst = {"ex": 0.0, "hy": 0.0, "j": 0.0}
    nslots = 0
    for r, sim in enumerate(sims):
        sim.step(4)
        for f in ("ex", "hy"):
            ref = sim.get(f)
            worst[f] = max(worst[f], float(np.linalg.norm(b.read(r, f) - ref) / np.linalg.norm(ref)))
        if sim.nslots:
            nslots += sim.nslots
            jr = sim.get("j")
            worst["j"] = max(worst["j"], float(np.linalg.norm(b.read(r, "j") - jr) / np.linalg.norm(jr)))
    info = b.info()
    print(f"{name}: {len(specs)} runs, {info['clusters']} clusters x {info['cluster_ctas']} CTAs, {nslots} slots: "
          + " ".join(f"{k}={v:.3e}" for k, v in worst.items()))
    assert nslots > 0 and max(worst.values()) <= tol, worst
