"""The training-sample recorder keeps a (slot, step) pair when word 0 of
Philox4x32-7 at counter (slot, step) under the key (seed) is below
rate * 2^32.  The oracle's generator (oracle/sr_bf16.py, written from the
published definition) predicts, slot by slot, which steps a subsampled run
records; those samples must be, bit for bit, the ones a record-everything run
of the same problem takes at exactly those steps."""
import numpy as np
import pytest

from fdtd_inputs import spec_1d_slab
from oracle.sr_bf16 import philox4x32

pytestmark = pytest.mark.gpu

NCELL, NSTEP = 24, 150


def _spec():
    spec = spec_1d_slab(nz=300, slab=(140, 140 + NCELL), src_k=40, precision="f32", steps=NSTEP, wp_w0=0.9)
    dens = spec["plasma"]["density"].copy()
    dens[140:140 + NCELL] = dens[150] * (1.0 + 0.01 * np.arange(NCELL))   # a distinct density per slot
    spec["plasma"]["density"] = dens
    return spec


def _record(spec, rate, seed):
    import torch
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec)
    cap = NCELL * NSTEP
    buf = torch.zeros(cap * 19, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.set_recording(buf, cnt, rate, seed)
    s.step(NSTEP)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert n <= cap
    return buf.view(cap, 19)[:n].cpu().numpy()


def _by_slot(rec, d32):
    slot_of = {float(v): i for i, v in enumerate(d32)}
    out = [[] for _ in range(NCELL)]
    for row in rec:
        out[slot_of[float(row[16])]].append(row)   # samples of one slot arrive in step order
    return out


def _selected(seed, rate):
    thr = np.uint64(int(rate * 4294967296.0)) if rate < 1.0 else np.uint64(0xFFFFFFFF)
    slot, step = np.meshgrid(np.arange(NCELL, dtype=np.uint64), np.arange(NSTEP, dtype=np.uint64), indexing="ij")
    ctr = np.stack([slot, np.zeros_like(slot), step, np.zeros_like(step)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)
    return philox4x32(ctr, key)[..., 0].astype(np.uint64) < thr            # [slot, step]


@pytest.mark.parametrize("rate,seed", [(0.3, (3 << 32) + 12345), (0.05, 7)])
def test_recorded_pairs_are_the_philox_selection(rate, seed):
    spec = _spec()
    d32 = spec["plasma"]["density"][140:140 + NCELL].astype(np.float32)
    assert np.unique(d32).size == NCELL
    full = _by_slot(_record(spec, 1.0, 0), d32)
    assert _selected(0, 1.0).all()                        # no draw equals 2^32 - 1: every pair recorded
    assert all(len(f) == NSTEP for f in full)
    sub = _by_slot(_record(spec, rate, seed), d32)
    sel = _selected(seed, rate)
    for s in range(NCELL):
        steps = np.nonzero(sel[s])[0]
        assert len(sub[s]) == steps.size, (s, len(sub[s]), steps.size)
        want = np.array([full[s][n] for n in steps]).reshape(-1, 19)
        assert np.array_equal(np.array(sub[s]).reshape(-1, 19), want), s
    total = int(sel.sum())
    print(f"rate {rate}: {total} of {NCELL * NSTEP} pairs recorded, each at its predicted step")
    assert abs(total / (NCELL * NSTEP) - rate) < 5 * np.sqrt(rate * (1 - rate) / (NCELL * NSTEP))
