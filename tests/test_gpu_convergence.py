"""The paper's vacuum validation (Sec. 4, Eq. 14-15) on the GPU path: the 1-D
Yee solution of the Gaussian pulse, started from the exact fields, converges at
order 2.0 (the paper's value, golden fixture) in RMS error; in FP64 its error
at every resolution equals the FP64 oracle's, and the FP32 instantiation
follows while truncation dominates its rounding."""
import json
import os

import numpy as np
import pytest

from tests.physics import C0, ETA0
from tests.test_oracle_yee import _pulse_error

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
PPW = (10, 20, 40, 80)


def _gpu_pulse_error(ppw, prec):
    """Same construction as the oracle's: a 3 m PEC line, pulse centred at
    0.6 m, 5 ns of travel, RMS error (Eq. 15) against the exact pulse."""
    from paper_2211_05647_gb300 import Solver
    tau = GOLD["validation_pulse_tau_s"]["value"]
    t0 = GOLD["validation_pulse_t0_s"]["value"]
    ctau = C0 * tau
    dz = ctau / ppw
    nz = int(round(3.0 / dz))
    s = Solver(dict(ndim=1, nx=1, ny=1, nz=nz, dx=dz, courant=0.5, precision=prec))
    dt = s.dt
    exact = lambda z, t: np.exp(-(((C0 * (t - t0)) - z) / ctau) ** 2)
    ts = t0 + 0.6 / C0
    z, zh = np.arange(nz + 1) * dz, (np.arange(nz) + 0.5) * dz
    e0 = exact(z, ts)
    e0[0] = e0[-1] = 0.0
    s.write("ex", e0)
    s.write("hy", exact(zh, ts - dt / 2) / ETA0)
    n = int(round(5e-9 / dt))
    s.step(n)
    u = s.read("ex", device=False).astype(np.float64)
    return np.sqrt(np.mean((u - exact(z, ts + n * dt)) ** 2))


def _order(errs):
    hs = 1.0 / np.array(PPW, dtype=np.float64)
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


def test_gaussian_pulse_order_fp64_equals_oracle(oracle_lib):
    gpu = np.array([_gpu_pulse_error(p, "f64") for p in PPW])
    ora = np.array([_pulse_error(oracle_lib, p) for p in PPW])
    order = _order(gpu)
    print("FP64 RMS errors", gpu, "order", order)
    assert abs(order - GOLD["convergence_order"]["value"]) < 0.1
    assert np.allclose(gpu, ora, rtol=1e-9, atol=0), (gpu, ora)


def test_gaussian_pulse_order_fp32():
    f64 = np.array([_gpu_pulse_error(p, "f64") for p in PPW])
    f32 = np.array([_gpu_pulse_error(p, "f32") for p in PPW])
    print("FP32 RMS errors", f32, "order", _order(f32))
    assert abs(_order(f32) - GOLD["convergence_order"]["value"]) < 0.15
    assert np.allclose(f32[:3], f64[:3], rtol=1e-2)
