"""BF16 delta-f storage rounds on the GPU exactly as the oracle's
stochastic-rounding reference prescribes (oracle/sr_bf16.py: Philox4x32-7
draws keyed by the seed and counted by (row, 16-byte vector, step), added
below the kept half of the FP32 bit pattern).

With delta f = 0 and every E component = 1 before a step, the step's kinetic
update forms alpha_j * 0 + beta_j * n_i * 1 in FP32 -- the value an FP32-storage
run of the same problem stores -- so every BF16 code the GPU writes is
predicted bit for bit from that FP32 run and the draws.  Checked at step 0
and after k steps of a driven run (the counter carries the absolute step
index), on the 1-D signed, 2-D Cartesian and 3-D grids and in the batched
driver (global row = the run's row offset + its local row, key = run 0's seed)."""
import copy

import numpy as np
import pytest

from fdtd_inputs import batch_runs_1d, spec_1d_slab, spec_2d_cylinder, spec_3d_slab
from oracle.sr_bf16 import bf16_sr, row_draws
from tests.adapters import FIELDS

pytestmark = pytest.mark.gpu


def _update_after(spec, f_dtype, k):
    from paper_2211_05647_gb300 import Solver
    sp = copy.deepcopy(spec)
    sp["plasma"]["f_dtype"] = f_dtype
    s = Solver.from_spec(sp)
    if k:
        s.step(k)
    ns, nn = s.plasma_shape()
    s.write("df", np.zeros((ns, nn)))
    for q in FIELDS[sp["grid"]["ndim"]]:
        if q.startswith("e"):
            s.write(q, np.ones(s.quantity_bytes(q) // 4))
    s.step(1)
    return s.read("df", device=False)


def _codes(df_bf16_as_f32):
    return (np.ascontiguousarray(df_bf16_as_f32, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _check(spec, k):
    f32 = _update_after(spec, "f32", k)
    got = _codes(_update_after(spec, "bf16", k))
    ns, nn = f32.shape
    assert nn % 8 == 0 and np.count_nonzero(f32) > 0.5 * f32.size
    want = bf16_sr(f32, row_draws(np.arange(ns), nn, step=k, seed=spec["plasma"]["seed"]))
    bad = np.argwhere(got != want)
    assert bad.size == 0, (bad[:5], got[tuple(bad[0])], want[tuple(bad[0])])
    truncated = (f32.view(np.uint32) >> 16).astype(np.uint16)
    frac_up = np.mean(got != truncated)
    print(f"{spec['name']} step {k}: {ns} rows x {nn} nodes, all codes equal; rounded up {frac_up:.3f}")
    assert 0.2 < frac_up < 0.8


def _specs():
    s1 = spec_1d_slab(nz=600, slab=(200, 330), src_k=60, nv=64, precision="f32", steps=1, seed=77)
    s2 = spec_2d_cylinder(n=96, ny=80, R=20, nv=16, nv_perp=16, steps=1, seed=78)
    s3 = spec_3d_slab(n=40, ny=24, nz=48, cpml=6, slab=(20, 34), src_k=8, nv=32, steps=1, seed=(5 << 32) + 79)
    return {"1d": s1, "2d": s2, "3d": s3}


@pytest.mark.parametrize("grid", ["1d", "2d", "3d"])
@pytest.mark.parametrize("k", [0, 37])
def test_bf16_codes_equal_philox_rounding(grid, k):
    _check(_specs()[grid], k)


def test_batched_bf16_codes_equal_philox_rounding():
    from paper_2211_05647_gb300 import Batch
    out = {}
    for fd in ("f32", "bf16"):
        specs = batch_runs_1d(nruns=5, nz_range=(300, 900), nv=64, f_dtype=fd, seed=404)
        b = Batch(specs)
        for r, sp in enumerate(specs):
            b.write(r, "ex", np.ones(sp["grid"]["nz"] + 1))
        b.step(1)
        out[fd] = [b.read(r, "df").reshape(-1, 64) for r in range(len(specs))]
        seed = specs[0]["plasma"]["seed"]
        b.close()
    off = 0
    for r, (f32, bf) in enumerate(zip(out["f32"], out["bf16"])):
        ns = f32.shape[0]
        want = bf16_sr(f32, row_draws(np.arange(off, off + ns), 64, step=0, seed=seed))
        assert np.array_equal(_codes(bf), want), r
        off += ns
    assert off > 0
