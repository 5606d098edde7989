"""Domain decomposition on one GPU: a grid split along its slowest axis into
sub-domains (fdtd_plasma_create_subdomain) that exchange one plane of
tangential E and H per step (fdtd_plasma_halo_pack / _unpack between the two
half steps) computes every field, J and delta-f value bit for bit as the whole
grid does -- with CPML on the split axis, a slab thinner than the CPML layer,
plasma and the source on slab boundaries' either side, FP32 and BF16 delta f
(stochastic rounding keyed by the global slot index) -- and the FP64
decomposed run matches the FP64 oracle."""
import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder, spec_3d_slab
from tests.adapters import FIELDS, oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _default_shapes(tmp_path, monkeypatch):
    # whole grid and sub-domains run the same (built-in) launch shapes
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "none.txt"))


def _equal(dec, whole, names):
    for n in names:
        a, b = dec.read(n), whole.read(n, device=False)
        assert np.array_equal(a, b.reshape(a.shape)), n


def _spec2d(f_dtype="f32", precision="f32"):
    return spec_2d_cylinder(n=160, ny=140, R=30, center=(90, 70), src=(40, 60), steps=150, seed=6,
                            f_dtype=f_dtype, precision=precision)


@pytest.mark.parametrize("f_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("bounds", [[(0, 6), (6, 60), (66, 74)], [(0, 70), (70, 70)]])
def test_2d_decomposed_equals_whole_grid(f_dtype, bounds):
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300.decomposed import DecomposedSolver
    spec = _spec2d(f_dtype)
    whole = Solver.from_spec(spec)
    whole.step(150)
    dec = DecomposedSolver(spec, bounds=bounds)
    dec.step(150)
    assert sum(s.plasma_shape()[0] for s in dec.subs) == whole.plasma_shape()[0]
    assert np.abs(whole.read("j", device=False)).max() > 0
    _equal(dec, whole, FIELDS[2] + ["j", "df"])


@pytest.mark.parametrize("f_dtype,shape", [("f32", (16, 16)), ("bf16", (8, 16))])
def test_2d_decomposed_ring_kernel_equals_whole_grid(f_dtype, shape):
    """The same with the bulk-copy ring kernel (three stages) on the whole grid and on every sub-domain:
    its per-slot stochastic-rounding counters are the global slot index, as in the register kernel."""
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300.decomposed import DecomposedSolver
    value = 3 * 10**9 + shape[0] * 10**6 + shape[1] * 1000
    spec = _spec2d(f_dtype)
    whole = Solver.from_spec(spec)
    whole.set_option("kinetic_shape", value)
    whole.step(150)
    dec = DecomposedSolver(spec, bounds=[(0, 6), (6, 60), (66, 74)])
    for sub in dec.subs:
        if sub.plasma_shape()[0]:
            sub.set_option("kinetic_shape", value)
    dec.step(150)
    assert np.abs(whole.read("j", device=False)).max() > 0
    _equal(dec, whole, FIELDS[2] + ["j", "df"])


@pytest.mark.parametrize("bounds", [[(0, 3), (3, 30), (33, 31)], [(0, 22), (22, 21), (43, 21)]])
def test_3d_decomposed_equals_whole_grid(bounds):
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300.decomposed import DecomposedSolver
    spec = spec_3d_slab(n=40, ny=36, nz=64, cpml=4, slab=(28, 44), src_k=10, steps=90, f_dtype="bf16")
    whole = Solver.from_spec(spec)
    whole.step(90)
    dec = DecomposedSolver(spec, bounds=bounds)
    dec.step(90)
    assert np.abs(whole.read("j", device=False)).max() > 0
    _equal(dec, whole, FIELDS[3] + ["j", "df"])


def test_decomposed_fp64_matches_oracle(oracle_lib):
    from paper_2211_05647_gb300.decomposed import DecomposedSolver
    spec = _spec2d("f64", "f64")
    dec = DecomposedSolver(spec, parts=4)
    dec.step(150)
    sim = oracle_sim(oracle_lib, spec)
    sim.step(150)
    for n in FIELDS[2] + ["j"]:
        e = rel_l2(dec.read(n), sim.get(n))
        print(f"decomposed FP64 {n}: rel L2 vs oracle {e:.2e}")
        assert e <= 1e-12, n


def test_subdomain_rules():
    import torch
    from paper_2211_05647_gb300 import FdtdError, Solver
    spec = _spec2d()
    mid = Solver.from_spec(spec, subdomain=(40, 50))
    with pytest.raises(FdtdError):          # neighbours on both sides: halves with halos only
        mid.step(1)
    with pytest.raises(FdtdError):          # half 1 before half 0
        mid.step_half(1)
    mid.step_half(0)
    with pytest.raises(FdtdError):          # half 0 again while half 1 is pending
        mid.step_half(0)
    mid.step_half(1)
    first = Solver.from_spec(spec, subdomain=(0, 40))
    buf = torch.empty(first.halo_bytes("e"), dtype=torch.uint8, device="cuda")
    assert buf.numel() == 160 * 4
    with pytest.raises(FdtdError):          # the first slab has no neighbour below
        first.halo_pack("e", buf)
    with pytest.raises(FdtdError):
        first.set_option("fused_stencils", 1)
    whole_axis = Solver.from_spec(spec, subdomain=(0, 140))   # no neighbours: plain steps allowed
    whole_axis.step(3)
