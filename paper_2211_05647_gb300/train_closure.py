"""Train the learned J closure for the 2-D TMz cylinder workloads and write
its parameters and normalisation to ``data/closure_2d_tmz_cylinder.npz``.

Training data: kinetic runs of the 4096^2 cylinder recipe (three seeded
density fields, 2000 steps each, the in-kernel recorder keeping a 1e-3
fraction of the (cell, step) pairs); normalisation, targets and training
(8 epochs of Adam, batch 4096, cosine-decayed rate from 2e-3) are library
calls (see closure.py).  Needs a GPU.

    python -m paper_2211_05647_gb300.train_closure [--out PATH] [--device N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "closure_2d_tmz_cylinder.npz")


def train_cylinder_closure(device: int = 0, epochs: int = 8, batch: int = 4096, lr: float = 2e-3, seed: int = 5,
                           rate: float = 1e-3, log=None) -> dict:
    """Record, normalise and train; returns the closure desc fields
    (params as float32 numpy, e/j/n scales, rho, beta, n_train_max) and the
    training record."""
    import torch
    from fdtd_inputs import C0, OMEGA0, closure_training_specs
    from . import closure as C
    t0 = time.perf_counter()
    specs = closure_training_specs()
    samples = torch.cat([C.record_samples(sp, sp["steps"], rate, 77 + i, 2_500_000, device=device)
                         for i, sp in enumerate(specs)])
    t_rec = time.perf_counter() - t0
    g = specs[0]["grid"]
    dt = g["courant"] * g["dx"] / C0
    sc = C.scales(samples, OMEGA0, dt, specs[0]["plasma"]["nu0"])
    x, t = C.dataset(samples, sc)
    t1 = time.perf_counter()
    params, hist = C.train(x, t, epochs=epochs, batch=batch, lr=lr, seed=seed, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    nmax = float(max(np.max(sp["plasma"]["density"]) for sp in specs))
    n = int(samples.shape[0])
    return dict(params=params.cpu().numpy().astype(np.float32), n_train_max=nmax, **sc,
                record=dict(runs=len(specs), steps=specs[0]["steps"], samples=n, rate=rate, epochs=epochs, batch=batch,
                            lr=lr, seed=seed, mse=hist, record_s=t_rec, train_s=t_train,
                            train_samples_per_s=epochs * (n // batch) * batch / t_train))


def save(res: dict, path: str = DEFAULT_OUT):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    meta = {k: v for k, v in res.items() if k != "params"}
    np.savez(path, params=res["params"], meta=json.dumps(meta))


def load(path: str = DEFAULT_OUT) -> dict:
    """The trained closure: {"params": float32[18945], e_scale, j_scale,
    n_scale, rho, beta, n_train_max, record}."""
    z = np.load(path)
    out = json.loads(str(z["meta"]))
    out["params"] = z["params"].astype(np.float32)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--device", type=int, default=0)
    args = ap.parse_args()
    res = train_cylinder_closure(args.device, log=lambda s: print(s, flush=True))
    save(res, args.out)
    print(json.dumps({k: v for k, v in res.items() if k != "params"}), flush=True)
    return 0


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(HERE))
    sys.exit(main())
