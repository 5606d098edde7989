"""Batched persistent 1-D driver: every run of a batch against the FP64
oracle run alone, and (FP32) bit-identical to the same run on the
single-run path (same reduction order)."""
import numpy as np
import pytest

from fdtd_inputs import batch_runs_1d, spec_1d_slab
from tests.adapters import compare, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _mixed_runs(precision, f_dtype):
    specs = batch_runs_1d(nruns=7, seed=5, nz_range=(40, 3000), nv=64, f_dtype=f_dtype, precision=precision,
                          src_k=30, steps=900)
    specs[1]["grid"]["mur"] = 0                       # one run with PEC ends
    specs[2]["plasma"]["density"] = np.zeros_like(specs[2]["plasma"]["density"])   # a vacuum run
    specs[3]["source"]["kind"] = "gauss"              # another source shape
    specs[4]["plasma"]["nu_model"] = "nsv"
    return specs


@pytest.mark.parametrize("precision,f_dtype,tol", [("f64", "f64", 1e-12), ("f32", "f32", 1e-4)])
def test_batch_runs_match_oracle(oracle_lib, precision, f_dtype, tol):
    from paper_2211_05647_gb300 import Batch
    specs = _mixed_runs(precision, f_dtype)
    for s in specs:
        s["plasma"]["nu_model"] = specs[0]["plasma"]["nu_model"]
    b = Batch(specs)
    b.step(900)
    info = b.info()
    assert info["steps"] == 900 and info["clusters"] >= 1
    for r, sp in enumerate(specs):
        sim = oracle_sim(oracle_lib, sp)
        sim.step(900)
        norm_e = np.linalg.norm(sim.get("ex"))
        e = np.linalg.norm(b.read(r, "ex") - sim.get("ex")) / norm_e
        h = np.linalg.norm(b.read(r, "hy") - sim.get("hy")) / np.linalg.norm(sim.get("hy"))
        print(f"run {r} nz={sp['grid']['nz']} slots={sim.nslots}: ex {e:.2e} hy {h:.2e}")
        assert e <= tol and h <= tol, (r, e, h)
        if sim.nslots:
            # J normalised by its norm, floored at 1e-6 A/m^2 per cell: runs whose slab the pulse
            # tail reaches only at ~1e-40 amplitude (below FP32's range) do not count as mismatches
            jr = sim.get("j")
            den = max(np.linalg.norm(jr), 1e-6 * np.sqrt(jr.size))
            assert np.linalg.norm(b.read(r, "j") - jr) / den <= tol


def test_batch_druyvesteyn_table_matches_oracle(oracle_lib):
    """Batched runs with the Druyvesteyn F0 and a tabulated s(v), FP64."""
    from fdtd_inputs import cross_section_table
    from paper_2211_05647_gb300 import Batch
    specs = _mixed_runs("f64", "f64")
    tab = cross_section_table()
    for s in specs:
        s["plasma"].update(f0_model="druyvesteyn", nu_model="table", s_table=tab)
    b = Batch(specs)
    b.step(specs[0]["steps"])
    for r, sp in enumerate(specs):
        sim = oracle_sim(oracle_lib, sp)
        sim.step(sp["steps"])
        for f in ("ex", "hy"):
            assert rel_l2(b.read(r, f), sim.get(f)) <= 1e-12, (r, f)
        if sim.nslots:
            jr = sim.get("j")
            den = max(np.linalg.norm(jr), 1e-6 * np.sqrt(jr.size))
            assert np.linalg.norm(b.read(r, "j") - jr) / den <= 1e-12, r


def test_batch_fp32_bit_identical_to_single_runs():
    from paper_2211_05647_gb300 import Batch, Solver
    specs = _mixed_runs("f32", "f32")
    b = Batch(specs)
    b.step(600)
    for r, sp in enumerate(specs):
        s = Solver.from_spec(sp)
        s.step(600)
        for q in ("ex", "hy", "j", "df"):
            if q in ("j", "df") and s.plasma_shape()[0] == 0:
                continue
            assert np.array_equal(b.read(r, q).ravel(), s.read(q, device=False).ravel()), (r, q)


def test_batch_bf16_fields_close_to_fp32():
    from paper_2211_05647_gb300 import Batch
    a = Batch(_mixed_runs("f32", "f32"))
    c = Batch(_mixed_runs("f32", "bf16"))
    a.step(700)
    c.step(700)
    for r in range(a.nruns):
        assert rel_l2(c.read(r, "ex"), a.read(r, "ex")) <= 5e-3


def test_batch_rejects_mixed_grids():
    from paper_2211_05647_gb300 import Batch, FdtdError
    specs = _mixed_runs("f32", "f32")
    specs[1]["grid"]["dx"] *= 1.5
    with pytest.raises(FdtdError):
        Batch(specs)


def test_batch_autotune_restores_state_and_keeps_results(oracle_lib):
    """The row-shape tuner times its candidates on the batch's buffers and
    restores the state bit for bit; stepping on with the shape it kept still
    matches the FP64 oracle."""
    from paper_2211_05647_gb300 import Batch
    specs = _mixed_runs("f32", "f32")
    for s in specs:
        s["plasma"]["nu_model"] = specs[0]["plasma"]["nu_model"]
    b = Batch(specs)
    b.step(300)
    before = [(b.read(r, "ex"), b.read(r, "hy"), b.read(r, "j"), b.read(r, "df")) for r in range(len(specs))]
    t = b.autotune()
    print(f"batch row shape kept: {t}")
    assert t["vpl"] * t["lanes"] >= 1 and t["ms_per_step"] > 0
    for r in range(len(specs)):
        after = (b.read(r, "ex"), b.read(r, "hy"), b.read(r, "j"), b.read(r, "df"))
        for x, y in zip(before[r], after):
            assert np.array_equal(x, y), r
    assert b.info()["steps"] == 300
    b.step(600)
    for r, sp in enumerate(specs):
        sim = oracle_sim(oracle_lib, sp)
        sim.step(900)
        e = np.linalg.norm(b.read(r, "ex") - sim.get("ex")) / np.linalg.norm(sim.get("ex"))
        assert e <= 1e-4, (r, e)
