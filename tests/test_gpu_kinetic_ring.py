"""The bulk-copy ring kernel of the kinetic update (FDTD_OPT_KINETIC_SHAPE
with ring stages > 0) stores the same delta-f rows, J and fields as the
register kernel of the same (vectors per lane, lanes per row) shape, bit for
bit: the row arithmetic (Sec. 5.2, Eq. 22), the J sum (Eq. 24) and the BF16
stochastic-rounding counters are the same.  Cases: FP32 and BF16 rows on 2-D
and 3-D grids whose plasma-cell count leaves a ragged last chunk, with one
CTA per SM so that each CTA walks more chunks than the ring has stages (the
ring wraps), and stage counts from 2 up."""
import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder, spec_3d_slab
from tests.adapters import FIELDS

pytestmark = pytest.mark.gpu


def _run(spec, shape, steps):
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    vpl, l, bps, stages = shape
    s.set_option("kinetic_shape", stages * 10**9 + vpl * 10**6 + l * 1000 + bps)
    got = s.launch_shapes()
    assert (got["kin_vpl"], got["kin_l"], got["kin_blocks_per_sm"], got["kin_stages"]) == shape
    s.step(steps)
    # a ring wait that gave up would set the error word, which the reads report (FDTD_ERR_TIMEOUT)
    out = {n: s.read(n, device=False).copy() for n in FIELDS[spec["grid"]["ndim"]] + ["j", "df"]}
    s.close()
    return out


def _cases():
    # 3-D: 62 x 46 x 40 = 114 080 plasma rows (ragged for 64 / 128 / 256-row chunks), 32 nodes
    s3 = spec_3d_slab(n=62, ny=47, nz=80, cpml=6, slab=(20, 60), src_k=8, nv=32, steps=1)
    # 2-D: a radius-90 cylinder, 16 x 16 nodes (a row of 256 nodes: 1 KB FP32, 512 B BF16)
    s2 = spec_2d_cylinder(n=280, ny=250, R=90, center=(150, 125), src=(40, 125), nv=16, nv_perp=16, steps=1,
                          seed=9)
    return {"3d": s3, "2d": s2}


@pytest.mark.parametrize("grid", ["3d", "2d"])
@pytest.mark.parametrize("f_dtype", ["bf16", "f32"])
def test_ring_equals_register_kernel(grid, f_dtype):
    import copy
    spec = copy.deepcopy(_cases()[grid])
    spec["plasma"]["f_dtype"] = f_dtype
    vec = {"bf16": 8, "f32": 4}[f_dtype]
    nn = {"3d": 32, "2d": 256}[grid]
    nvec = nn // vec
    shapes = [(v, nvec // v) for v in (1, 2, 4, 8, 16) if nvec % v == 0 and nvec // v <= 32 and v * (nvec // v) == nvec]
    steps = 30
    checked = 0
    for vpl, l in shapes:
        try:
            ref = _run(spec, (vpl, l, 0, 0), steps)
        except Exception as e:   # not a candidate shape of this row length
            if "candidate" in str(e):
                continue
            raise
        for bps, stages in ((1, 2), (1, 3), (0, 4)):
            from paper_2211_05647_gb300 import FdtdError
            try:
                got = _run(spec, (vpl, l, bps, stages), steps)
            except FdtdError as e:
                assert "ring stages" in str(e)   # these stages do not fit in shared memory
                continue
            for n, v in ref.items():
                assert np.array_equal(got[n], v), (grid, f_dtype, vpl, l, stages, n)
            checked += 1
    print(f"{grid} {f_dtype}: {checked} ring launches equal to the register kernel")
    assert checked >= 3


def test_ring_stage_bounds():
    """Stage counts that do not fit, FP64 rows and the nonlinear update are refused."""
    import copy
    from paper_2211_05647_gb300 import FdtdError, Solver
    spec = copy.deepcopy(_cases()["2d"])
    s = Solver.from_spec(spec)
    with pytest.raises(FdtdError):
        s.set_option("kinetic_shape", 1 * 10**9 + 4 * 10**6 + 16 * 1000)      # one stage
    with pytest.raises(FdtdError):
        s.set_option("kinetic_shape", 64 * 10**9 + 4 * 10**6 + 16 * 1000)     # 64 stages of 16 KB
    s.set_option("kinetic_shape", 4 * 10**9 + 4 * 10**6 + 16 * 1000)
    assert s.launch_shapes()["kin_stages"] == 4
    spec["grid"]["precision"] = "f64"
    spec["plasma"]["f_dtype"] = "f64"
    s64 = Solver.from_spec(spec)
    with pytest.raises(FdtdError):
        s64.set_option("kinetic_shape", 4 * 10**9 + 8 * 10**6 + 16 * 1000)
