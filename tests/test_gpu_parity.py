"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 per field over the whole grid, and for J over all
plasma cells, after the full run):
  * FP64 instantiation: 1e-12 (rounding-order differences only)
  * FP32 fields + FP32 delta f: 1e-4
  * FP32 fields + BF16 delta f with stochastic rounding: 5e-3 on the fields;
    J, a moment of 8-bit-mantissa nodes whose rounding noise random-walks
    over the run, is held to what that noise explains: a second run with
    another rounding seed gives the noise level sigma = |J1 - J2| / sqrt(2)
    (two independent draws of zero-mean noise), and the error against the
    FP64 oracle must stay within 1.5 sigma (plus the FP32 arithmetic's 1e-4),
    so anything beyond the rounding noise -- a bias, a dropped term -- fails;
    1e-1 remains as an outer cap (the noise is shown to be unbiased by
    test_bf16_stochastic_rounding_is_unbiased)
Sizes span several stencil tiles (32 x 8 / 32 x 4 x 2) with ragged tails.
"""
import numpy as np
import pytest

from fdtd_inputs import (OMEGA0, critical_density, cross_section_table, pulse_params, spec_1d_slab, spec_2d_cylinder,
                         spec_3d_slab)
from tests.adapters import FIELDS, compare, oracle_sim

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-4, "bf16": 5e-3}
TOL_J_BF16 = 1e-1


def _check(errs, prec, fdt):
    tol = TOL["bf16" if fdt == "bf16" else prec]
    for k, v in errs.items():
        assert v <= (TOL_J_BF16 if (k == "j" and fdt == "bf16") else tol), errs


def _solver(spec):
    from paper_2211_05647_gb300 import Solver
    return Solver.from_spec(spec)


def _report(name, errs):
    print(f"{name}: " + " ".join(f"{k}={v:.3e}" for k, v in errs.items()))


def _check_bf16_j_noise(spec, s, sim, steps):
    """BF16 delta f: J's error against the FP64 oracle is the stochastic-rounding noise and nothing else."""
    import copy
    from tests.adapters import rel_l2
    sp = copy.deepcopy(spec)
    sp["plasma"]["seed"] = int(sp["plasma"]["seed"]) + 7919
    s2 = _solver(sp)
    s2.step(steps)
    ref = sim.get("j")
    j1 = np.asarray(s.read("j", device=False), dtype=np.float64)
    j2 = np.asarray(s2.read("j", device=False), dtype=np.float64)
    err = rel_l2(j1, ref)
    sigma = np.linalg.norm(j1 - j2) / np.sqrt(2.0) / np.linalg.norm(ref)
    print(f"bf16 J: error vs FP64 {err:.3e}, seed-to-seed noise {sigma:.3e}")
    assert sigma > 0
    assert err <= 1.5 * sigma + 1e-4, (err, sigma)


def _run_pair(oracle_lib, spec, steps):
    sim = oracle_sim(oracle_lib, spec)
    s = _solver(spec)
    sim.step(steps)
    s.step(steps)
    return s, sim


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_1d_slab_full_run(oracle_lib, prec):
    """The 1-D slab workload (Nz = 2000, Nv = 64, Mur, source at node 100),
    run long enough for the pulse to cross the slab."""
    spec = spec_1d_slab(precision=prec, steps=2600)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 1)
    _report(f"1d {prec}", errs)
    assert np.abs(sim.get("j")).max() > 0
    assert max(errs.values()) <= TOL[prec], errs


def _small_2d(prec="f32", f_dtype="f32", nx=200, ny=150, R=40, steps=500, nv=32, nv_perp=32):
    spec = spec_2d_cylinder(n=nx, ny=ny, R=R, center=(nx * 0.55, ny * 0.5), src=(int(nx * 0.55) - R - 12, ny // 2),
                            nv=nv, nv_perp=nv_perp, steps=steps, precision=prec, f_dtype=f_dtype, seed=11)
    return spec


@pytest.mark.parametrize("prec,fdt", [("f64", "f64"), ("f32", "f32"), ("f32", "bf16")])
def test_2d_tmz_cylinder(oracle_lib, prec, fdt):
    spec = _small_2d(prec, fdt)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 2)
    _report(f"2d {prec} {fdt}", errs)
    assert np.abs(sim.get("j")).max() > 0
    _check(errs, prec, fdt)
    if fdt == "bf16":
        _check_bf16_j_noise(spec, s, sim, spec["steps"])


def _small_3d(prec="f32", f_dtype="f32", n=(40, 36, 64), steps=220, nv=32, slab=(28, 44), src_k=12, cpml=8):
    nx, ny, nz = n
    return spec_3d_slab(n=nx, ny=ny, nz=nz, cpml=cpml, slab=slab, src_k=src_k, nv=nv, steps=steps,
                        precision=prec, f_dtype=f_dtype, seed=13)


@pytest.mark.parametrize("prec,fdt", [("f64", "f64"), ("f32", "f32"), ("f32", "bf16")])
def test_3d_slab(oracle_lib, prec, fdt):
    spec = _small_3d(prec, fdt)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 3)
    _report(f"3d {prec} {fdt}", errs)
    assert np.abs(sim.get("j")).max() > 0
    _check(errs, prec, fdt)
    if fdt == "bf16":
        _check_bf16_j_noise(spec, s, sim, spec["steps"])


@pytest.mark.parametrize("ndim,nx,cpml", [(2, 201, 10), (2, 196, 6), (3, 38, 8), (3, 44, 6)])
def test_fp32_stencil_paths(oracle_lib, ndim, nx, cpml):
    """FP32 stencils on both code paths: rows that are not a multiple of 4
    cells run one cell per thread (nx = 201, 38); rows that are run four cells
    per thread with shuffled x neighbours, here with CPML slabs of 6 cells that
    end inside a quad (nx = 196, 44)."""
    if ndim == 2:
        spec = spec_2d_cylinder(n=nx, ny=131, R=30, cpml=cpml, center=(nx * 0.55, 65), src=(int(nx * 0.55) - 42, 65),
                                nv=16, nv_perp=8, steps=500, precision="f32", f_dtype="f32", seed=17)
    else:
        spec = spec_3d_slab(n=nx, ny=34, nz=60, cpml=cpml, slab=(26, 42), src_k=12, nv=16, steps=400,
                            precision="f32", f_dtype="f32", seed=19)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, ndim)
    _report(f"{ndim}d f32 nx={nx} cpml={cpml}", errs)
    assert np.abs(sim.get("j")).max() > 0
    _check(errs, "f32", "f32")


@pytest.mark.parametrize("vgrid,nv,nvp", [("speed3d", 31, 1), ("signed1d", 48, 1), ("cart2d", 8, 6),
                                         ("signed1d", 2, 1), ("signed1d", 512, 1)])
def test_velocity_grids_and_ragged_rows(oracle_lib, vgrid, nv, nvp):
    """Non-power-of-two and tiny / large node counts (padded rows) on every grid kind."""
    spec = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, precision="f64", steps=700, nv=nv)
    spec["plasma"].update(vgrid=vgrid, nv=nv, nv_perp=nvp)
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 1)
    assert np.abs(sim.get("j")).max() > 0
    assert max(errs.values()) <= 1e-12, errs
    df = s.read("df", device=False)
    assert np.allclose(df, sim.get("df"), rtol=1e-11, atol=1e-12 * np.abs(sim.get("df")).max())


@pytest.mark.parametrize("vgrid,nv,nvp", [("signed1d", 48, 1), ("speed3d", 31, 1), ("cart2d", 14, 10)])
@pytest.mark.parametrize("nu_model", ["nsv", "table"])
def test_druyvesteyn_and_cross_section_table(oracle_lib, vgrid, nv, nvp, nu_model):
    """Druyvesteyn F0 (Sec. 5.2) with the N s v collision law, s constant or
    tabulated (Eq. 23), FP64 on every grid kind against the oracle, whose
    tables come from its own formulas and quadrature."""
    spec = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, precision="f64", steps=700, nv=nv)
    spec["plasma"].update(vgrid=vgrid, nv=nv, nv_perp=nvp, f0_model="druyvesteyn", nu_model=nu_model)
    if nu_model == "table":
        spec["plasma"]["s_table"] = cross_section_table(te_ev=spec["plasma"]["te_ev"])
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 1)
    _report(f"druyvesteyn {vgrid} {nu_model}", errs)
    assert np.abs(sim.get("j")).max() > 0
    assert max(errs.values()) <= 1e-12, errs
    df = s.read("df", device=False)
    assert np.allclose(df, sim.get("df"), rtol=1e-11, atol=1e-12 * np.abs(sim.get("df")).max())


def test_cross_section_table_rejected_when_malformed():
    from paper_2211_05647_gb300 import FdtdError
    spec = spec_1d_slab(nz=200, slab=(80, 120), precision="f32", steps=1, nv=16)
    sp, sg = cross_section_table()
    for bad in ((sp[::-1].copy(), sg), (sp, -sg), (sp[:1], sg[:1])):
        spec["plasma"].update(nu_model="table", s_table=bad)
        with pytest.raises(FdtdError):
            _solver(spec)


def test_bf16_stochastic_rounding_is_unbiased(oracle_lib):
    """Averaging J over independently seeded BF16 runs converges to the FP64
    oracle like 1/sqrt(runs): the stochastic rounding adds zero-mean noise
    (round-to-nearest would freeze the slow collisional decay instead)."""
    from tests.adapters import rel_l2
    base = spec_1d_slab(nz=400, slab=(150, 260), src_k=40, precision="f32", f_dtype="bf16", steps=900)
    sim = oracle_sim(oracle_lib, base)
    sim.step(base["steps"])
    ref = sim.get("j")
    js = []
    for seed in range(8):
        base["plasma"]["seed"] = 1000 + seed
        s = _solver(base)
        s.step(base["steps"])
        js.append(s.read("j", device=False).astype(np.float64))
    e1 = np.mean([rel_l2(j, ref) for j in js])
    e8 = rel_l2(np.mean(js, axis=0), ref)
    print(f"bf16 J error: single run {e1:.3e}, mean of 8 seeds {e8:.3e}")
    assert e8 < 0.6 * e1
    assert not np.array_equal(js[0], js[1])


def test_const_nu_and_random_initial_state(oracle_lib):
    """Random E, H and delta f as the initial state (2-D, CPML, const nu)."""
    spec = _small_2d("f64", "f64", nx=130, ny=97, R=30, steps=150)
    spec["plasma"]["nu_model"] = "const"
    sim = oracle_sim(oracle_lib, spec)
    s = _solver(spec)
    rng = np.random.default_rng(5)
    for nm in FIELDS[2]:
        v = rng.standard_normal(sim.get(nm).size) * (1.0 if nm[0] == "e" else 1 / 377.0)
        if nm == "ez":
            v.reshape(97, 130)[0, :] = 0
            v.reshape(97, 130)[:, 0] = 0
        sim.set(nm, v)
        s.write(nm, v)
    df0 = rng.standard_normal((sim.nslots, sim.nnode)) * 1e-2
    sim.set("df", df0)
    s.write("df", df0)
    sim.step(150)
    s.step(150)
    errs = compare(s, sim, 2)
    assert max(errs.values()) <= 1e-12, errs


def test_vacuum_and_no_plasma_cells(oracle_lib):
    """No plasma at all, and a density that is nonzero only on PEC nodes (no slots)."""
    spec = _small_2d("f64", "f64", nx=64, ny=64, R=10, steps=120)
    dens = np.zeros(64 * 64)
    dens.reshape(64, 64)[0, :] = 1e17   # PEC row j = 0: excluded
    spec["plasma"]["density"] = dens
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    assert sim.nslots == 0 and s.plasma_shape()[0] == 0
    errs = compare(s, sim, 2)
    assert max(errs.values()) <= 1e-12, errs
    spec["plasma"] = None
    s2, sim2 = _run_pair(oracle_lib, spec, spec["steps"])
    assert max(compare(s2, sim2, 2).values()) <= 1e-12


def test_step_chunking_is_invisible(oracle_lib):
    """step(1) x N and step(N) (graph chunk of 32 + singles) give identical state."""
    spec = _small_2d("f32", "f32", nx=96, ny=80, R=20, steps=70)
    a, b = _solver(spec), _solver(spec)
    for _ in range(70):
        a.step(1)
    b.step(70)
    for nm in FIELDS[2] + ["j", "df"]:
        assert np.array_equal(a.read(nm, device=False), b.read(nm, device=False)), nm


def test_checkpoint_resume_bit_identical(oracle_lib):
    spec = _small_3d("f32", "bf16", n=(24, 20, 40), steps=60, slab=(20, 30), src_k=9, cpml=6)
    a = _solver(spec)
    a.step(60)
    b = _solver(spec)
    b.step(30)
    blob = b.save_state(device=False)
    c = _solver(spec)
    c.load_state(blob)
    assert c.info()[1] == 30
    c.step(30)
    for nm in FIELDS[3] + ["j", "df"]:
        assert np.array_equal(a.read(nm, device=False), c.read(nm, device=False)), nm


def test_diagnostics_match_oracle(oracle_lib):
    spec = _small_2d("f64", "f64", nx=100, ny=90, R=25, steps=400)
    spec["plasma"]["density"] = spec["plasma"]["density"]
    s, sim = _run_pair(oracle_lib, spec, 400)
    dg, do = s.diagnostics(), sim.diag()
    for k in ("energy", "energy_plain", "number_abs"):
        assert dg[k] == pytest.approx(do[k], rel=1e-11), k
    assert abs(dg["number"]) <= 1e-12 * do["number_abs"]
    assert dg["finite"] and dg["step"] == 400


@pytest.mark.parametrize("ndim,prec", [(1, "f64"), (2, "f64"), (3, "f64"), (1, "f32"), (2, "f32"), (3, "f32")])
def test_poynting_matches_oracle(oracle_lib, ndim, prec):
    """Random fields written to both sides (FP32-representable values for the
    FP32 solver, so both start from the same numbers): the FP64 Poynting
    diagnostic agrees face by face to rounding order.  Boxes include faces on
    the grid edges, a box with coincident faces and a single plane."""
    from paper_2211_05647_gb300 import FdtdError, Solver
    shape = {1: dict(nz=300), 2: dict(nx=70, ny=53), 3: dict(nx=37, ny=29, nz=23)}[ndim]
    s = Solver(dict(ndim=ndim, dx=1e-3, courant=0.5, precision=prec, **shape))
    sim = oracle_lib.Sim(oracle_lib.params(ndim=ndim, dx=1e-3, courant=0.5, **shape))
    rng = np.random.default_rng(40 + ndim)
    for nm in FIELDS[ndim]:
        v = rng.standard_normal(sim.get(nm).size) * (1.0 if nm[0] == "e" else 1 / 377.0)
        if prec == "f32":
            v = v.astype(np.float32).astype(np.float64)
        s.write(nm, v)
        sim.set(nm, v)
    boxes = {1: [[0, 0, 0, 0, 0, 300], [0, 0, 0, 0, 17, 250], [0, 0, 0, 0, 5, 5]],
             2: [[0, 69, 0, 52, 0, 0], [10, 50, 7, 40, 0, 0], [3, 3, 5, 30, 0, 0]],
             3: [[0, 36, 0, 28, 0, 22], [5, 30, 4, 20, 3, 19], [10, 10, 2, 27, 4, 9]]}[ndim]
    for box in boxes:
        got, want = np.array(s.poynting(box)), sim.poynting(box)
        scale = np.abs(want[:6]).sum()
        assert scale > 0
        err = np.abs(got - want).max() / scale
        print(f"poynting {ndim}-D {prec} box {box}: max face error / scale {err:.2e}")
        assert err <= 1e-12, (got, want)
    bad = {1: [0, 0, 0, 0, 3, 301], 2: [0, 70, 0, 10, 0, 0], 3: [5, 4, 0, 1, 0, 1]}[ndim]
    with pytest.raises(FdtdError):
        s.poynting(bad)


def test_energy_invariant_gpu_fp32():
    """Lossless PEC cavity, random fields: the FP64 diagnostic of the FP32 run
    drifts by at most 1e-5 relative."""
    from paper_2211_05647_gb300 import Solver
    s = Solver(dict(ndim=3, nx=48, ny=40, nz=36, dx=1e-3, courant=0.5, precision="f32"))
    rng = np.random.default_rng(2)
    for nm in FIELDS[3]:
        v = rng.standard_normal(48 * 40 * 36).reshape(36, 40, 48) * (1.0 if nm[0] == "e" else 1 / 377.0)
        if nm == "ex":
            v[:, 0, :] = 0; v[0, :, :] = 0
        if nm == "ey":
            v[:, :, 0] = 0; v[0, :, :] = 0
        if nm == "ez":
            v[:, :, 0] = 0; v[:, 0, :] = 0
        s.write(nm, v.ravel())
    W0 = s.diagnostics()["energy"]
    for _ in range(10):
        s.step(100)
        assert abs(s.diagnostics()["energy"] - W0) <= 1e-5 * W0


def test_abi_errors():
    from paper_2211_05647_gb300 import FdtdError, Solver
    from paper_2211_05647_gb300 import fdtd_plasma as F
    with pytest.raises(FdtdError) as e:
        Solver(dict(ndim=3, nx=16, ny=16, nz=16, dx=1e-3, courant=0.6))
    assert e.value.code == F.FDTD_ERR_UNSTABLE
    with pytest.raises(FdtdError) as e:
        Solver(dict(ndim=2, nx=2, ny=16, dx=1e-3))
    assert e.value.code == F.FDTD_ERR_INVAL
    with pytest.raises(FdtdError):
        Solver(dict(ndim=2, nx=30, ny=30, dx=1e-3, cpml_cells=10))
    s = Solver(dict(ndim=1, nz=100, dx=1e-3, mur=1, precision="f32"))
    with pytest.raises(FdtdError) as e:
        s.set_plasma(np.full(101, np.nan), f_dtype="f32")
    assert e.value.code == F.FDTD_ERR_NONFINITE
    with pytest.raises(FdtdError):
        s.set_plasma(np.full(101, 1e17), f_dtype="f64")        # f64 storage on an f32 grid
    with pytest.raises(FdtdError) as e:
        s.set_plasma(np.full(101, 1e30), f_dtype="f32")        # w_p dt too large
    assert e.value.code == F.FDTD_ERR_UNSTABLE
    with pytest.raises(FdtdError):
        s.set_source(kind="gauss", k=0, tau=1e-10)            # Mur node is not a source node
    for bad in (dict(amp=float("nan")), dict(fc=float("inf")), dict(t0=float("nan")), dict(tau=0.0)):
        with pytest.raises(FdtdError):
            s.set_source(**dict(dict(kind="gauss_sine", k=10, tau=1e-10, fc=1e10, t0=4e-10), **bad))
    s.set_plasma(np.full(101, 1e17), f_dtype="f32")
    s.step(3)
    with pytest.raises(FdtdError) as e:
        s.set_plasma(np.full(101, 1e17), f_dtype="f32")
    assert e.value.code == F.FDTD_ERR_STATE
    with pytest.raises(FdtdError):
        s.step(-1)
    lib = F.load_library()
    assert lib.fdtd_plasma_step(None, 1) == F.FDTD_ERR_INVAL
    lib.fdtd_plasma_destroy(None)
    buf = np.zeros(7)
    assert lib.fdtd_plasma_read_fields(s.h, 0, buf.ctypes.data, 56, 0) == F.FDTD_ERR_INVAL
    s.reset()
    s.set_plasma(np.full(101, 1e17), f_dtype="bf16")
    assert s.info()[1] == 0


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_nonlinear_mode_1d(oracle_lib, prec):
    """Flux-form advection of delta f (strong field so it matters) vs the oracle;
    the particle-number perturbation stays at rounding level."""
    spec = spec_1d_slab(nz=500, slab=(200, 320), src_k=60, precision=prec, steps=900)
    spec["source"]["amp"] = 3e5
    spec["plasma"]["nonlinear"] = 1
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 1)
    _report(f"1d nonlinear {prec}", errs)
    # the advection term is really active: the even part of delta f is not small
    df = sim.get("df")
    assert np.abs(0.5 * (df + df[:, ::-1])).max() > 1e-6 * np.abs(df).max()
    assert max(errs.values()) <= TOL[prec], errs
    d = s.diagnostics()
    assert abs(d["number"]) <= (1e-13 if prec == "f64" else 1e-6) * d["number_abs"]


def test_nonlinear_mode_2d_cartesian(oracle_lib):
    spec = _small_2d("f64", "f64", nx=120, ny=100, R=25, steps=300, nv=16, nv_perp=8)
    spec["source"]["amp"] = 3e5
    spec["plasma"]["nonlinear"] = 1
    s, sim = _run_pair(oracle_lib, spec, spec["steps"])
    errs = compare(s, sim, 2)
    _report("2d nonlinear f64", errs)
    assert max(errs.values()) <= 1e-12, errs


def test_set_plasma_again_after_reset():
    """After reset, set_plasma with the same slot layout keeps the delta-f array (zeroed again) and one
    with another layout allocates a new one; either way the run equals a fresh solver's bit for bit."""
    import copy
    spec = _small_2d("f32", "f32", steps=60)
    other = copy.deepcopy(spec)
    d = np.array(other["plasma"]["density"], dtype=np.float64)
    d[np.flatnonzero(d)[::7]] = 0.0                       # fewer plasma cells: another layout
    other["plasma"]["density"] = d
    s = _solver(spec)
    s.step(60)                                            # leaves delta f, J and the fields non-zero
    for sp in (spec, other, spec):
        s.reset()
        s.set_plasma(**dict(sp["plasma"]))
        s.set_source(**dict(sp["source"]))
        s.step(60)
        fresh = _solver(sp)
        fresh.step(60)
        for n in FIELDS[2] + ["j", "df"]:
            assert np.array_equal(s.read(n, device=False), fresh.read(n, device=False)), n
        fresh.close()
