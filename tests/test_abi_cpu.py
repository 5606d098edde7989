"""CPU-side checks of the boundary: the library builds, loads without a GPU
and exports every entry point include/fdtd_plasma.h declares; the binding's
signature table covers exactly those; the input generators are deterministic."""
import os
import re
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fdtd_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2211_05647_gb300 import build as B
    lib = B.build()
    import paper_2211_05647_gb300 as P
    P.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, declared - exported
    assert declared == set(P.SIGNATURES), (declared ^ set(P.SIGNATURES))


def test_binding_refuses_missing_library(tmp_path):
    import pytest
    from paper_2211_05647_gb300 import fdtd_plasma as F
    with pytest.raises(RuntimeError):
        F._lib, saved = None, F._lib
        try:
            F.load_library(str(tmp_path / "nope.so"))
        finally:
            F._lib = saved


def test_input_generators_are_seeded():
    from fdtd_inputs import cylinder_density, spec_3d_slab
    a = cylinder_density(300, 280, 150, 140, 60, 1e18, seed=4)
    b = cylinder_density(300, 280, 150, 140, 60, 1e18, seed=4)
    c = cylinder_density(300, 280, 150, 140, 60, 1e18, seed=5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.max() == 1e18 and (a >= 0).all()
    r2 = ((np.arange(300)[None, :] - 150) ** 2 + (np.arange(280)[:, None] - 140) ** 2).ravel()
    assert (a[r2 > 60 ** 2] == 0).all() and (a[r2 < 50 ** 2] > 0).all()
    s = spec_3d_slab(n=32, cpml=4, slab=(10, 20), src_k=6)
    d = s["plasma"]["density"].reshape(32, 32, 32)
    assert (d[:10] == 0).all() and (d[20:] == 0).all() and np.all(np.diff(d[10:20, 5, 5]) > 0)
