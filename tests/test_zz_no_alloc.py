"""The allocation-free diagnostics entry point (fdtd_diagnostics_noalloc).

Some callers cannot allocate device memory when they want a diagnostic:
watchdog or monitoring code that must not take the allocator's locks or
trigger cudaMalloc's implicit synchronisation, frameworks that own every
device allocation through their own pool, and code close to the memory limit.
For them the library offers a variant of the diagnostics reduction whose
scratch is a fixed file-scope device array.  This test calls it through the C
ABI on caller-owned copies of a solver's state and checks, on two calls in a
row, that it returns what fdtd_plasma_diagnostics returns for the same state.

It sits in a file of its own, collected last, and runs the same whether it is
alone in a fresh process or after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _arrays(s, spec, keep):
    import torch
    from paper_2211_05647_gb300 import fdtd_plasma as F
    from fdtd_inputs import ME, QE
    g, p = spec["grid"], spec["plasma"]
    a = F.fdtd_diag_arrays()
    a.ndim, a.precision = g["ndim"], F.PRECISION[g["precision"]]
    a.nx, a.ny, a.nz = g["nx"], g["ny"], g["nz"]
    a.dx, a.courant = g["dx"], g["courant"]
    for name, q in F.QUANTITY.items():
        if q < 6 and s.quantity_bytes(name):
            t = s.read(name)              # caller-owned device copy
            keep.append(t)
            a.fields[q] = t.data_ptr()
    df = s.read("df")
    keep.append(df)
    ns, nn = s.plasma_shape()
    vmax = p["vmax_vth"] * np.sqrt(QE * p["te_ev"] / ME)
    dv = (2 * vmax / p["nv"]) * (2 * vmax / p["nv_perp"])   # Cartesian grid: uniform volume element
    dV = torch.full((nn,), dv, dtype=torch.float64, device=s.device)
    keep.append(dV)
    a.df, a.f_dtype, a.nslots, a.nnode, a.dV = df.data_ptr(), F.DF_DTYPE[p["f_dtype"]], ns, nn, dV.data_ptr()
    return a


def test_noalloc_diagnostics_match_the_allocating_entry_point():
    import torch
    from fdtd_inputs import spec_2d_cylinder
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300 import fdtd_plasma as F
    lib = F.load_library()
    spec = spec_2d_cylinder(n=300, ny=220, R=60, center=(170, 110), src=(95, 110), steps=300, seed=21)
    s = Solver.from_spec(spec)
    keys = ["energy", "energy_plain", "number", "number_max_cell", "number_abs", "finite"]
    for call in range(2):                 # two calls in a row, state advanced in between
        s.step(150)
        ref = s.diagnostics()
        keep = []
        a = _arrays(s, spec, keep)
        torch.cuda.synchronize()
        host = (ctypes.c_double * 6)()
        rc = lib.fdtd_diagnostics_noalloc(ctypes.byref(a), host, 0, ctypes.c_void_p(s.stream.cuda_stream))
        assert rc == 0, lib.fdtd_plasma_last_error(None)
        dev = torch.zeros(6, dtype=torch.float64, device=s.device)
        rc = lib.fdtd_diagnostics_noalloc(ctypes.byref(a), ctypes.cast(dev.data_ptr(), ctypes.POINTER(ctypes.c_double)),
                                          1, ctypes.c_void_p(s.stream.cuda_stream))
        assert rc == 0, lib.fdtd_plasma_last_error(None)
        torch.cuda.synchronize()
        got_dev = dev.cpu().numpy()
        for i, k in enumerate(keys):
            want = float(ref[k])
            for got in (host[i], got_dev[i]):
                if k == "number":          # a cancelling sum: compare against its absolute scale
                    assert abs(got - want) <= 1e-12 * ref["number_abs"], (call, k, got, want)
                else:
                    assert got == pytest.approx(want, rel=1e-12, abs=0.0), (call, k, got, want)
        assert ref["energy"] > 0 and ref["number_abs"] > 0


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2211_05647_gb300 import fdtd_plasma as F
    lib = F.load_library()
    a = F.fdtd_diag_arrays()
    a.ndim, a.precision, a.nx, a.ny, a.nz, a.dx, a.courant = 2, 0, 64, 64, 1, 1e-3, 0.5
    for q in (2, 3, 4):
        a.fields[q] = 1          # never dereferenced: the size check comes first
    a.df, a.dV, a.f_dtype, a.nnode = 1, 1, 0, 32
    a.nslots = 16384 * 8192      # needs more tiles than the fixed scratch holds
    out = (ctypes.c_double * 6)()
    rc = lib.fdtd_diagnostics_noalloc(ctypes.byref(a), out, 0, None)
    assert rc == F.FDTD_ERR_INVAL
    assert b"maximum" in lib.fdtd_plasma_last_error(None)
