"""Fused E^{n+1} + H^{n+3/2} stencil pass (2-D TMz and 3-D, FP32, opt-in): the
same physics as the unfused sequence (FP32 rounding order only), for step
counts that exercise the parity rule (an odd number of fused transitions runs
the first one unfused), the 32-step graph chunks and the 1-step graph, with
CPML, the source (a 3-D sheet; a 2-D point, also on a tile's halo node) and a
kinetic region; and against the FP64 oracle."""
import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder, spec_3d_slab
from tests.adapters import FIELDS, compare, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _spec(steps, n=(44, 36, 70), cpml=6, slab=(34, 52)):
    nx, ny, nz = n
    return spec_3d_slab(n=nx, ny=ny, nz=nz, cpml=cpml, slab=slab, src_k=12, nv=16, steps=steps,
                        precision="f32", f_dtype="f32", seed=31)


def _pair(spec, calls):
    from paper_2211_05647_gb300 import Solver
    fused, plain = Solver.from_spec(spec), Solver.from_spec(spec)
    fused.set_option("fused_stencils", 1)
    for n in calls:
        fused.step(n)
        plain.step(n)
    return fused, plain


@pytest.mark.parametrize("calls", [(1,), (2,), (3,), (33,), (64, 5), (7, 1, 40)])
def test_fused_equals_unfused(calls):
    fused, plain = _pair(_spec(sum(calls)), calls)
    worst = 0.0
    for q in FIELDS[3] + ["j", "df"]:
        a, b = fused.read(q, device=False), plain.read(q, device=False)
        if np.abs(b).max() == 0:
            assert np.abs(a).max() == 0, q
            continue
        worst = max(worst, rel_l2(a, b))
    print(f"calls {calls}: fused vs unfused max rel L2 {worst:.2e}")
    assert worst <= 1e-6


def test_fused_matches_oracle(oracle_lib):
    spec = _spec(260)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("fused_stencils", 1)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 3)
    print("fused 3-D f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


def test_fused_no_cpml_and_ragged_tiles():
    """Grid sizes that leave partial 32 x 8 x 32 tiles on every axis, PEC walls."""
    spec = _spec(50, n=(37, 13, 45), cpml=0, slab=(24, 36))
    spec["source"].update(i0=0, i1=37, j0=1, j1=13)   # the whole updated Ex plane (no CPML frame)
    fused, plain = _pair(spec, (50,))
    for q in FIELDS[3]:
        assert rel_l2(fused.read(q, device=False), plain.read(q, device=False)) <= 1e-6, q


def test_fused_option_errors_and_checkpoint():
    from paper_2211_05647_gb300 import FdtdError, Solver
    spec = _spec(40)
    s = Solver.from_spec(spec)
    with pytest.raises(FdtdError):
        s.set_option("fused_stencils", 2)
    s.set_option("fused_stencils", 1)
    s.step(21)
    blob = s.save_state(device=False)
    s.step(19)
    r = Solver.from_spec(spec)
    r.set_option("fused_stencils", 1)
    r.load_state(blob)
    r.step(19)
    for q in FIELDS[3] + ["j"]:
        assert np.array_equal(s.read(q, device=False), r.read(q, device=False)), q


# ---------------------------------------------------------------- 2-D TMz
# 150 x 70 cells leave ragged 64 x 16 tiles on both axes; with an 8-cell CPML
# frame the tiles at x0 = 64, y0 = 16 / 32 are the CPML-free ones.

def _spec2(steps, n=(150, 70), cpml=8, src=(40, 35)):
    nx, ny = n
    return spec_2d_cylinder(n=nx, ny=ny, cpml=cpml, R=min(nx, ny) // 4, center=(0.6 * nx, 0.5 * ny), src=src,
                            nv=8, nv_perp=8, steps=steps, precision="f32", f_dtype="f32", seed=32)


def _worst(fused, plain, quantities):
    worst = 0.0
    for q in quantities:
        a, b = fused.read(q, device=False), plain.read(q, device=False)
        if np.abs(b).max() == 0:
            assert np.abs(a).max() == 0, q
            continue
        worst = max(worst, rel_l2(a, b))
    return worst


@pytest.mark.parametrize("calls", [(1,), (2,), (3,), (33,), (64, 5), (7, 1, 40)])
def test_fused_2d_equals_unfused(calls):
    fused, plain = _pair(_spec2(sum(calls)), calls)
    worst = _worst(fused, plain, FIELDS[2] + ["j", "df"])
    print(f"2-D calls {calls}: fused vs unfused max rel L2 {worst:.2e}")
    assert worst <= 1e-6


@pytest.mark.parametrize("src", [(64, 48), (63, 47), (149, 69)])
def test_fused_2d_source_on_tile_edges(src):
    """The point source on a node that one tile computes as halo and another
    owns, on the last node of a tile, and on the grid's last node."""
    spec = _spec2(70, cpml=0 if src == (149, 69) else 8, src=src)
    fused, plain = _pair(spec, (70,))
    assert _worst(fused, plain, FIELDS[2] + ["j"]) <= 1e-6


def test_fused_2d_matches_oracle(oracle_lib):
    spec = _spec2(260)
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("fused_stencils", 1)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 2)
    print("fused 2-D f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


def test_fused_2d_no_cpml_small_grid():
    """A grid smaller than one tile (PEC walls only) and one a tile wide."""
    for n, src in (((37, 13), (20, 6)), ((64, 16), (30, 8))):
        fused, plain = _pair(_spec2(45, n=n, cpml=0, src=src), (45,))
        assert _worst(fused, plain, FIELDS[2]) <= 1e-6, n


def test_fused_2d_checkpoint():
    from paper_2211_05647_gb300 import Solver
    spec = _spec2(40)
    s = Solver.from_spec(spec)
    s.set_option("fused_stencils", 1)
    s.step(21)
    blob = s.save_state(device=False)
    s.step(19)
    r = Solver.from_spec(spec)
    r.set_option("fused_stencils", 1)
    r.load_state(blob)
    r.step(19)
    for q in FIELDS[2] + ["j", "df"]:
        assert np.array_equal(s.read(q, device=False), r.read(q, device=False)), q


# ---------------------------------------------- 2-D column march (nx % 4 == 0)
# 296 x 70 cells: two full 128-column strips and a partial one (dead lanes),
# segments of 1, 5 and 32 rows (ragged at the top) and one segment for all.

@pytest.mark.parametrize("rows", [1, 5, 32, 4096])
@pytest.mark.parametrize("src", [(40, 35), (128, 32), (127, 31), (136, 30), (135, 29), (8, 20), (7, 21), (288, 40),
                                 (295, 69)])
def test_fused_2d_march_equals_unfused(rows, src):
    """The source in the interior; on the first column of a strip (formed as
    halo by the strip to its left) and on a strip's last column, both for
    strips cut at multiples of 128 (no CPML) and at the CPML's x slabs (8
    cells: strips [0, 8), [8, 136), [136, 264), [264, 288), [288, 296)); and
    on the grid's last node; fields bit for bit."""
    from paper_2211_05647_gb300 import Solver
    spec = _spec2(70, n=(296, 70), cpml=0 if src in ((295, 69), (128, 32), (127, 31)) else 8, src=src)
    fused, plain = Solver.from_spec(spec), Solver.from_spec(spec)
    fused.set_option("fused_stencils", 1)
    fused.set_option("fused_rows", rows)
    for n in (33, 37):
        fused.step(n)
        plain.step(n)
    for q in FIELDS[2] + ["j"]:
        assert np.array_equal(fused.read(q, device=False), plain.read(q, device=False)), q


def test_fused_2d_march_matches_oracle(oracle_lib):
    spec = _spec2(260, n=(152, 70))
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    s.set_option("fused_stencils", 1)
    s.set_option("fused_rows", 16)
    s.step(100)
    s.step(160)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(260)
    errs = compare(s, sim, 2)
    print("fused 2-D column march f32 vs oracle: " + " ".join(f"{k}={v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) <= 1e-4, errs


def test_fused_rows_option():
    from paper_2211_05647_gb300 import FdtdError, Solver
    s = Solver.from_spec(_spec2(10, n=(152, 70)))
    for bad in (-1, 4097):
        with pytest.raises(FdtdError):
            s.set_option("fused_rows", bad)
    s.set_option("fused_rows", 0)
    s.set_option("fused_rows", 4096)


def test_every_2d_stencil_path_bit_identical(tmp_path, monkeypatch):
    """The 2-D kernels share one fixed-rounding form of the cell updates: the
    default grid-of-cells kernels, the TMA column kernels, the fused column
    march and the fused 64 x 16 tiles give the same fields, J and delta f bit
    for bit (CPML, point source, kinetic region)."""
    from paper_2211_05647_gb300 import Solver
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "none.txt"))
    spec = _spec2(75, n=(296, 70), src=(130, 33))
    variants = {"default": {}, "tma": {"stencil_tz": 32}, "march": {"fused_stencils": 1, "fused_rows": 8},
                "tiles": {"fused_stencils": 1, "fused_rows": 0}}
    out = {}
    for name, opts in variants.items():
        s = Solver.from_spec(spec)
        for k, v in opts.items():
            s.set_option(k, v)
        s.step(40)
        s.step(35)
        out[name] = {q: s.read(q, device=False) for q in FIELDS[2] + ["j", "df"]}
    for name in variants:
        for q, v in out[name].items():
            assert np.array_equal(v, out["default"][q]), (name, q)


def test_autotuned_fused_choice(tmp_path, monkeypatch):
    """The autotuner's 2-D choice (fused column march or separate passes) is
    reported, cached for later handles, and steps bit for bit like a handle
    on the default kernels; half steps stay allowed."""
    from paper_2211_05647_gb300 import Solver
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    spec = _spec2(64, n=(1024, 512), src=(300, 256))
    s = Solver.from_spec(spec)
    res = s.autotune()
    assert res["fused_rows"] in (0, 4, 8, 16, 32)
    assert s.launch_shapes()["fused_rows"] == res["fused_rows"]
    assert Solver.from_spec(spec).launch_shapes()["fused_rows"] == res["fused_rows"]
    s.step(64)
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "none.txt"))
    plain = Solver.from_spec(spec)
    assert plain.launch_shapes()["fused_rows"] == 0
    # the same kinetic shape (its J reduction order is the one thing shapes may change)
    plain.set_option("kinetic_shape", res["kin_stages"] * 10**9 + res["kin_vpl"] * 10**6 + res["kin_l"] * 1000
                     + res["kin_blocks_per_sm"])
    plain.step(64)
    for q in FIELDS[2] + ["j"]:
        assert np.array_equal(s.read(q, device=False), plain.read(q, device=False)), q
    s.step_half(0)
    s.step_half(1)


def test_step_counts_split_into_graphs_bit_identical():
    """A call's steps run as 32-step chunks plus one 16/8/4/2/1-step graph per
    set bit of the remainder, each with its own fused transitions: any split
    of the same steps into calls gives the same state bit for bit (2-D)."""
    from paper_2211_05647_gb300 import Solver
    spec = _spec2(100, n=(152, 70))
    a, b = Solver.from_spec(spec), Solver.from_spec(spec)
    a.set_option("fused_stencils", 1)
    b.set_option("fused_stencils", 1)
    for n in (23, 45, 1, 31):
        a.step(n)
    for _ in range(100):
        b.step(1)
    for q in FIELDS[2] + ["j", "df"]:
        assert np.array_equal(a.read(q, device=False), b.read(q, device=False)), q
