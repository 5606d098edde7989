"""TMA stencils (FP32): 3-D column kernels (blocks of 32 x 8 threads walking tz
planes along z) and 2-D strip kernels (walking rows in 8-row chunks), planes /
chunks staged in shared memory by tensor copies.  They compute the
same cell formulas as the grid-of-cells kernels, so the fields must agree bit
for bit on grids with ragged tiles on every axis (partial 32-cell rows, partial
8-row tiles, a last block with fewer than tz planes), with and without CPML,
with the sheet source and a kinetic slab; and within the FP32 tolerance of the
FP64 oracle."""
import numpy as np
import pytest

from fdtd_inputs import spec_3d_slab
from tests.adapters import FIELDS, compare, oracle_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _no_tune_cache(monkeypatch, tmp_path):
    # default launch shapes (one cell per thread) for the grid-of-cells side
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "none.txt"))


def _spec(steps, n=(44, 36, 70), cpml=6, slab=(34, 52), src_k=12):
    nx, ny, nz = n
    return spec_3d_slab(n=nx, ny=ny, nz=nz, cpml=cpml, slab=slab, src_k=src_k, nv=16, steps=steps,
                        precision="f32", f_dtype="f32", seed=37)


def _pair(spec, tz, calls):
    from paper_2211_05647_gb300 import Solver
    tma, cells = Solver.from_spec(spec), Solver.from_spec(spec)
    tma.set_option("stencil_tz", tz)
    assert tma.launch_shapes()["stencil_tz"] == tz and cells.launch_shapes()["stencil_tz"] == 0
    for n in calls:
        tma.step(n)
        cells.step(n)
    return tma, cells


@pytest.mark.parametrize("tz", [1, 3, 16, 64])
def test_tma_equals_cells_bitwise(tz):
    tma, cells = _pair(_spec(45), tz, (7, 38))
    for q in FIELDS[3] + ["j", "df"]:
        a, b = tma.read(q, device=False), cells.read(q, device=False)
        assert np.abs(b).max() > 0, q
        assert np.array_equal(a, b), (q, np.abs(a - b).max())


@pytest.mark.parametrize("n,tz", [((64, 40, 33), 8), ((36, 9, 5), 2), ((96, 17, 3), 4)])
def test_tma_no_cpml_ragged(n, tz):
    """PEC walls only: x a multiple of 4 but not of 32, y not a multiple of 8,
    nz not a multiple of tz (and the smallest nz, 3)."""
    nx, ny, nz = n
    spec = _spec(30, n=n, cpml=0, slab=(0, nz) if nz < 4 else (nz // 3, 2 * nz // 3), src_k=min(2, nz - 1))
    spec["source"].update(i0=0, i1=nx, j0=1, j1=ny)
    tma, cells = _pair(spec, tz, (30,))
    for q in FIELDS[3]:
        assert np.array_equal(tma.read(q, device=False), cells.read(q, device=False)), q


def test_tma_matches_oracle(oracle_lib):
    spec = _spec(260)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("stencil_tz", 16)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 3)
    print("TMA column stencils 3-D f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


def test_tma_with_fused_option_and_checkpoint():
    """The opt-in fused pass runs its own kernel on the second field set; the
    unfused transitions and the last E update of each sequence use the TMA
    kernels on set 0.  A checkpoint resumes bit for bit."""
    from paper_2211_05647_gb300 import Solver
    spec = _spec(40)
    a = Solver.from_spec(spec)
    a.set_option("stencil_tz", 8)
    a.set_option("fused_stencils", 1)
    a.step(21)
    blob = a.save_state(device=False)
    a.step(19)
    b = Solver.from_spec(spec)
    b.set_option("stencil_tz", 8)
    b.set_option("fused_stencils", 1)
    b.load_state(blob)
    b.step(19)
    for q in FIELDS[3] + ["j"]:
        assert np.array_equal(a.read(q, device=False), b.read(q, device=False)), q


def test_tma_option_errors():
    from fdtd_inputs import spec_2d_cylinder
    from paper_2211_05647_gb300 import FdtdError, Solver
    pec = _spec(1, n=(38, 16, 20), cpml=0, slab=(8, 12), src_k=3)   # nx not a multiple of 4
    pec["source"].update(i0=0, i1=38, j0=1, j1=16)
    s = Solver.from_spec(pec)
    s3 = Solver.from_spec(_spec(1))
    s2 = Solver.from_spec(spec_2d_cylinder(n=64, ny=32, R=8, nv=4, nv_perp=4, steps=1, precision="f32",
                                           f_dtype="f32"))
    for solver, v in ((s, 8), (s3, -1), (s3, 2000)):
        with pytest.raises(FdtdError):
            solver.set_option("stencil_tz", v)
    s2.set_option("stencil_tz", 16)          # 2-D FP32 with nx a multiple of 4: the TMA strips
    s3.set_option("stencil_tz", 8)
    s3.set_option("stencil_tz", 0)
    assert s3.launch_shapes()["stencil_tz"] == 0


# ------------------------------------------- fused E + H pass on TMA-staged planes
# With both options set, every fused transition of the step sequence runs
# k_eh3d_tma (reading one field set, writing the other); the first transition of
# an odd count and the last E update run the separate TMA kernels.  The cell
# formulas are the separate kernels', so the fields agree with the grid-of-cells
# sequence bit for bit.

def _fused_tma(spec, tz, calls):
    from paper_2211_05647_gb300 import Solver
    f, cells = Solver.from_spec(spec), Solver.from_spec(spec)
    f.set_option("stencil_tz", tz)
    f.set_option("fused_stencils", 1)
    for n in calls:
        f.step(n)
        cells.step(n)
    return f, cells


@pytest.mark.parametrize("tz,calls", [(12, (1,)), (12, (2,)), (12, (3,)), (12, (33,)), (3, (64, 5)), (1, (7, 1, 40)),
                                      (70, (36,))])
def test_fused_tma_equals_cells_bitwise(tz, calls):
    f, cells = _fused_tma(_spec(sum(calls)), tz, calls)
    assert np.abs(cells.read("ex", device=False)).max() > 0
    for q in FIELDS[3] + ["j", "df"]:
        a, b = f.read(q, device=False), cells.read(q, device=False)
        assert np.array_equal(a, b), (q, np.abs(a - b).max())


@pytest.mark.parametrize("n,tz", [((64, 40, 33), 8), ((36, 9, 5), 2), ((96, 17, 3), 4)])
def test_fused_tma_no_cpml_ragged(n, tz):
    nx, ny, nz = n
    spec = _spec(30, n=n, cpml=0, slab=(0, nz) if nz < 4 else (nz // 3, 2 * nz // 3), src_k=min(2, nz - 1))
    spec["source"].update(i0=0, i1=nx, j0=1, j1=ny)
    f, cells = _fused_tma(spec, tz, (30,))
    for q in FIELDS[3]:
        assert np.array_equal(f.read(q, device=False), cells.read(q, device=False)), q


def test_fused_tma_matches_oracle(oracle_lib):
    spec = _spec(260)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("stencil_tz", 12)
    s.set_option("fused_stencils", 1)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 3)
    print("fused TMA pass 3-D f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


# ------------------------------------------------------------ 2-D TMz strips
# 148 x 70 cells: x a multiple of 4 but not of 32 (a partial strip), y not a multiple of 8 (a partial chunk).

def _spec2(steps, n=(148, 70), cpml=8, src=(40, 35)):
    from fdtd_inputs import spec_2d_cylinder
    nx, ny = n
    return spec_2d_cylinder(n=nx, ny=ny, cpml=cpml, R=min(nx, ny) // 4, center=(0.6 * nx, 0.5 * ny), src=src,
                            nv=8, nv_perp=8, steps=steps, precision="f32", f_dtype="f32", seed=33)


@pytest.mark.parametrize("rows,src", [(8, (40, 35)), (24, (64, 48)), (64, (147, 69))])
def test_tma_2d_equals_cells(rows, src):
    spec = _spec2(45, cpml=0 if src == (147, 69) else 8, src=src)
    tma, cells = _pair(spec, rows, (7, 38))
    worst = 0.0
    for q in FIELDS[2] + ["j", "df"]:
        a, b = tma.read(q, device=False), cells.read(q, device=False)
        d = np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)
        worst = max(worst, d)
    print(f"2-D TMA rows={rows} vs grid-of-cells: max |diff| / max |value| = {worst:.2e}")
    assert worst <= 1e-6


def test_tma_2d_matches_oracle(oracle_lib):
    spec = _spec2(260)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("stencil_tz", 32)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 2)
    print("TMA strips 2-D f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs
