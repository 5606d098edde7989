"""Maximum grid size: the solver accepts up to 2^31 - 1 nodes, so its index
arithmetic must hold right below that limit.  A point source 10 cells from the
high corner of a PEC grid of 1290^3 (3-D) or 46340^2 (2-D) nodes, and the same
source 10 cells from the corner of a small grid: until a disturbance can reach
a wall the two grids do not share (the influence spreads by at most two cells a
step), the fields around the source agree bit for bit.  Compared on the device."""
import numpy as np
import pytest

from fdtd_inputs.workloads import C0, LAM0

pytestmark = pytest.mark.gpu

DX = LAM0 / 20


def _spec(ndim, n, src):
    dt = 0.5 * DX / C0
    grid = dict(ndim=ndim, nx=n, ny=n, nz=n if ndim == 3 else 1, dx=DX, courant=0.5, cpml_cells=0, mur=0,
                precision="f32")
    source = dict(kind="gauss", location="point", i=src, j=src, k=src if ndim == 3 else 0, amp=1.0, fc=0.0,
                  tau=8 * dt, t0=24 * dt)
    return dict(name=f"max{ndim}d", grid=grid, source=source, plasma=None, steps=12)


def _free_gb():
    import torch
    return torch.cuda.mem_get_info()[0] / 1e9


@pytest.mark.parametrize("ndim,n_big,need_gb,tz", [(2, 46340, 30, 0), (3, 1290, 60, 0), (2, 46340, 30, 64),
                                                    (3, 1288, 60, 12)])
def test_fields_near_the_high_corner_of_a_maximum_grid(ndim, n_big, need_gb, tz):
    """tz > 0: the TMA stencils (32-bit tensor coordinates, 64-bit offsets) on both grids."""
    import torch
    from paper_2211_05647_gb300 import Solver
    assert n_big ** ndim < 2 ** 31 - 1
    if _free_gb() < need_gb:
        pytest.skip(f"needs {need_gb} GB of free device memory")
    n_small, steps, w = 48, 12, 30
    fields = ["ez", "hx", "hy"] if ndim == 2 else ["ex", "ey", "ez", "hx", "hy", "hz"]
    out = {}
    for n in (n_small, n_big):
        s = Solver.from_spec(_spec(ndim, n, n - 10))
        if tz:
            s.set_option("stencil_tz", tz)
        s.step(steps)
        shape = (n, n) if ndim == 2 else (n, n, n)
        out[n] = {f: s.read(f, device=True).reshape(shape)[(slice(n - w, n),) * ndim].clone() for f in fields}
        s.close()
        del s
        torch.cuda.empty_cache()
    worst = 0.0
    for f in fields:
        a, b = out[n_big][f], out[n_small][f]
        assert torch.count_nonzero(b) > 0, f
        assert torch.equal(a, b), (f, float((a - b).abs().max()))
        worst = max(worst, float(b.abs().max()))
    print(f"{ndim}-D {n_big}^{ndim} = {n_big ** ndim} nodes, stencil_tz {tz}: the {w}^{ndim} corner equals the "
          f"{n_small}^{ndim} run "
          f"(max |field| {worst:.3e})")
