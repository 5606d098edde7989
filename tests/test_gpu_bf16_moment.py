"""The J moment of BF16 delta-f rows (Eq. 24, the Jx sum of Sec. 5.2) where
its terms nearly cancel.

BF16 rows update in FP32 and sum J = -e sum_j w_j df_j per lane in two plain
FP32 partial sums (even and odd nodes), then across the lanes of a row by a
TwoSum tree.  Rows are written with random-sign values whose moment is
projected to ~0 before rounding to BF16, so |J| is far below the sum of the
magnitudes of its terms.  One step with zero fields gives
J = -e sum_j w_j alpha_j df_j from exactly those values; per slot it is
compared with the FP64 oracle run on the same BF16 values, relative to
S = e sum_j |w_j alpha_j df_j|, the scale FP32 products and sums can reach.
The bound, 1e-6 S, holds however small J is; the measured error and the
cancellation S / |J| are printed."""
import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder, spec_3d_slab
from tests.adapters import oracle_params, oracle_sim

pytestmark = pytest.mark.gpu
QE = 1.602176634e-19


def _specs():
    return [spec_2d_cylinder(n=64, ny=48, R=12, center=(36, 24), src=(12, 24), steps=1, seed=5, f_dtype="bf16"),
            spec_3d_slab(n=16, ny=12, nz=24, cpml=2, slab=(10, 14), src_k=5, steps=1, f_dtype="bf16")]


@pytest.mark.parametrize("k", [0, 1])
def test_bf16_j_moment_under_cancellation(oracle_lib, k):
    import torch
    from paper_2211_05647_gb300 import Solver
    O = oracle_lib
    spec = _specs()[k]
    s = Solver.from_spec(spec)
    ns, nn = s.plasma_shape()
    sim = oracle_sim(O, spec)
    tab = O.vtables(oracle_params(O, spec), sim.dt)
    wa = tab["w"] * tab["alpha"]
    rng = np.random.default_rng(20 + k)
    df = rng.standard_normal((ns, nn)) * np.exp(rng.uniform(-3, 3, (ns, 1)))
    df -= (df @ wa / (wa @ wa))[:, None] * wa[None, :]          # moment ~0 before rounding
    dfb = torch.from_numpy(df).to(torch.bfloat16).to(torch.float64).numpy()
    s.write("df", dfb)
    s.step(1)
    J = s.read("j", device=False).astype(np.float64)
    sim.set("df", dfb)
    sim.step(1)
    Jo = sim.get("j")
    S = QE * np.abs(dfb * wa[None, :]).sum(axis=1)
    err = np.abs(J - Jo) / S
    cancel = S / np.maximum(np.abs(Jo), 1e-300)
    print(f"{spec['name']}: {ns} rows x {nn} BF16 nodes; cancellation S/|J| median {np.median(cancel):.1e} "
          f"max {cancel.max():.1e}; |J - J_FP64| / S max {err.max():.2e}, "
          f"relative to |J| median {np.median(np.abs(J - Jo) / np.abs(Jo)):.2e}")
    assert np.median(cancel) > 30
    assert err.max() <= 1e-6
