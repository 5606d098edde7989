"""Launch-shape autotuner: it leaves the simulation state bit-for-bit as it
found it, writes its choices to the cache, later handles of the same class
start from them, and the tuned shapes give the same physics (FP32 rounding
order only)."""
import os

import numpy as np
import pytest

from fdtd_inputs import spec_2d_cylinder, spec_3d_slab
from tests.adapters import FIELDS, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_autotune_restores_state_and_caches(tmp_path, monkeypatch, kind):
    from paper_2211_05647_gb300 import Solver
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(cache))
    if kind == "2d":
        spec = spec_2d_cylinder(n=300, ny=260, R=60, center=(170, 130), src=(80, 130), steps=120, seed=4)
        names = FIELDS[2]
    else:
        spec = spec_3d_slab(n=48, ny=40, nz=64, cpml=8, slab=(28, 44), src_k=12, steps=120, f_dtype="f32")
        names = FIELDS[3]
    s = Solver.from_spec(spec)
    s.step(60)
    before = {n: s.read(n, device=False).copy() for n in names + ["j", "df"]}
    res = s.autotune()
    print(f"autotune {kind}: {res}")
    for n, v in before.items():
        assert np.array_equal(s.read(n, device=False), v), n
    assert res["kin_vpl"] > 0 and res["kin_l"] > 0 and res["block_x"] > 0
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 2 and any("|kinetic|" in ln for ln in lines) and any("|stencil" in ln for ln in lines)
    s.step(60)
    ref = Solver.from_spec(spec)      # picks the cached shapes up at create / set_plasma
    tuned = {k: v for k, v in res.items() if not k.endswith("_ms") and k != "reserved"}
    assert ref.launch_shapes() == tuned
    ref.step(120)
    again = Solver.from_spec(spec)    # same shapes throughout: bit-identical
    again.step(120)
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "empty.txt"))
    dflt = Solver.from_spec(spec)     # default shapes
    assert dflt.launch_shapes()["block_x"] > 0 or kind == "1d"
    dflt.step(120)
    for n in names:
        assert np.array_equal(again.read(n, device=False), ref.read(n, device=False)), n
        # other shapes (one or four cells per thread) differ only in rounding order
        assert rel_l2(s.read(n, device=False), ref.read(n, device=False)) <= 1e-5, n
        assert rel_l2(s.read(n, device=False), dflt.read(n, device=False)) <= 1e-5, n


def test_forced_kinetic_shape(tmp_path, monkeypatch):
    """FDTD_OPT_KINETIC_SHAPE: every candidate shape of the row length runs
    and gives the default shape's fields to FP32 rounding order; a shape that
    is not a candidate is refused."""
    from paper_2211_05647_gb300 import FdtdError, Solver
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "none.txt"))
    spec = spec_2d_cylinder(n=160, ny=120, R=30, center=(95, 60), src=(50, 60), steps=150, seed=2)
    ref = Solver.from_spec(spec)
    ref.step(150)
    for vpl, l in ((8, 32), (16, 16)):
        s = Solver.from_spec(spec)
        s.set_option("kinetic_shape", vpl * 1000000 + l * 1000)
        assert (s.launch_shapes()["kin_vpl"], s.launch_shapes()["kin_l"]) == (vpl, l)
        s.step(150)
        for n in FIELDS[2] + ["j"]:
            assert rel_l2(s.read(n, device=False), ref.read(n, device=False)) <= 1e-5, (vpl, l, n)
    with pytest.raises(FdtdError):
        Solver.from_spec(spec).set_option("kinetic_shape", 3 * 1000000 + 5 * 1000)


def test_autotune_leaves_ports_and_recording_untouched(tmp_path, monkeypatch):
    """The autotuner times kinetic candidates inside whole steps: those steps must add nothing to the port
    spectra or to the training-sample recorder (neither is part of the saved state it restores)."""
    import torch
    from paper_2211_05647_gb300 import Solver
    monkeypatch.setenv("FDTD_PLASMA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    spec = spec_2d_cylinder(n=200, ny=160, R=40, center=(110, 80), src=(50, 80), steps=40, seed=8)
    s = Solver.from_spec(spec)
    s.set_ports([[80 * 200 + 150], [80 * 200 + 60]], np.linspace(5e9, 15e9, 6))
    samples = torch.zeros(4096 * 19, dtype=torch.float32, device=s.device)
    count = torch.zeros(1, dtype=torch.int64, device=s.device)
    s.set_recording(samples, count, rate=0.01, seed=3)
    s.step(20)
    ports0 = s.port_spectra().copy()
    s.stream.synchronize()
    n0 = int(count.item())
    s.autotune()
    s.stream.synchronize()
    assert int(count.item()) == n0
    assert np.array_equal(s.port_spectra(), ports0)
    assert n0 > 0 and np.abs(ports0).max() > 0
