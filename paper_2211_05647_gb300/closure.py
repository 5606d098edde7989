"""Learned J closure: training data from kinetic runs, normalisation, and
training with the library's own GPU kernels.

The closure replaces, for cells inside the training density range, the
velocity-space update of Sec. 5.2 (the f_1x update and the Jx moment) by a
17 -> 128 -> 128 -> 1 GELU network on top of the Crank-Nicolson Drude update
of a plasma with the mean collision frequency nu:
    x = [E^{n-15} .. E^n] / E_s ++ [n / n_s]
    J^{n+1/2} = rho J^{n-1/2} + beta n E^n + J_s y
    rho = (2 - dt nu)/(2 + dt nu),  beta = 2 dt (e^2/m) / (2 + dt nu)
so the network learns only the kinetic correction (what the velocity-
dependent collision frequency adds to the Drude response).  E_s is the RMS
of E over the training samples, n_s the critical density at w0, and J_s the
RMS of the correction itself (targets of unit variance).  Every
step of the pipeline runs on the GPU: the kinetic runs record their samples
in-kernel, and the loss, its gradient and the Adam update are library kernels.
"""
from __future__ import annotations

import math

import numpy as np

EPS0 = 8.8541878128e-12
QE = 1.602176634e-19
ME = 9.1093837015e-31
NIN, NHID, NPARAMS = 17, 128, 18945


def init_params(seed: int, device):
    """He-style initialisation of the packed FP32 parameters (seeded)."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = [torch.randn(NIN * NHID, generator=g) * math.sqrt(2.0 / NIN), torch.zeros(NHID),
             torch.randn(NHID * NHID, generator=g) * math.sqrt(2.0 / NHID), torch.zeros(NHID),
             torch.randn(NHID, generator=g) * math.sqrt(1.0 / NHID), torch.zeros(1)]
    return torch.cat(parts).to(device=device, dtype=torch.float32).contiguous()


def record_samples(spec, steps: int, rate: float, seed: int, capacity: int, device=0):
    """Run the kinetic solver on ``spec`` for ``steps`` steps with the
    in-kernel recorder on; returns the [N, 19] float32 device tensor of
    [E^{n-15..n}, n, J^{n+1/2}, J^{n-1/2}] samples."""
    import torch
    from .fdtd_plasma import Solver
    s = Solver.from_spec(spec, device=device)
    buf = torch.empty(capacity * 19, dtype=torch.float32, device=s.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=s.device)
    s.set_recording(buf, cnt, rate, seed)
    s.step(steps)
    torch.cuda.synchronize()
    n = min(int(cnt.item()), capacity)
    out = buf[: n * 19].view(n, 19).clone()
    s.close()
    return out


def _residual(samples, rho, beta):
    s = samples.double()
    return s[:, 17] - rho * s[:, 18] - beta * s[:, 16] * s[:, 15]


def scales(samples, omega0: float, dt: float, nu_mean: float, increment: bool = True) -> dict:
    """Normalisations and the Drude part for the closure desc (see module doc);
    increment=False gives the direct form (rho = beta = 0)."""
    e_s = float(samples[:, :16].double().pow(2).mean().sqrt().item())
    n_c = EPS0 * ME * omega0 ** 2 / QE ** 2
    if increment:
        rho = (2.0 - dt * nu_mean) / (2.0 + dt * nu_mean)
        beta = 2.0 * dt * (QE * QE / ME) / (2.0 + dt * nu_mean)
    else:
        rho = beta = 0.0
    r = _residual(samples, rho, beta)
    j_s = float(r.pow(2).mean().sqrt().item()) or EPS0 * omega0 * e_s
    return dict(e_scale=e_s, j_scale=j_s, n_scale=n_c, rho=rho, beta=beta)


def dataset(samples, sc: dict):
    """Network inputs and targets (float32 device tensors) from raw samples."""
    import torch
    x = torch.empty(samples.shape[0], NIN, dtype=torch.float32, device=samples.device)
    x[:, :16] = samples[:, :16] / sc["e_scale"]
    x[:, 16] = samples[:, 16] / sc["n_scale"]
    t = (_residual(samples, sc["rho"], sc["beta"]) / sc["j_scale"]).float()
    return x.contiguous(), t.contiguous()


def train(x, t, epochs: int = 10, batch: int = 4096, lr: float = 2e-3, seed: int = 0, log=None):
    """Adam on the mean-squared error, cosine-decayed learning rate, seeded
    shuffles; returns (params, per-epoch mean losses)."""
    import torch
    from .fdtd_plasma import MlpTrainer
    dev = x.device
    params = init_params(seed, dev)
    tr = MlpTrainer(params, batch, lr=lr)
    n = x.shape[0]
    nb = n // batch
    total = max(epochs * nb, 1)
    g = torch.Generator(device=dev).manual_seed(seed + 1)
    hist = []
    it = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device=dev)
        acc = torch.zeros((), dtype=torch.float64, device=dev)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / total))
            loss = tr.step(x[idx].contiguous(), t[idx].contiguous(), lr=lr_t)
            acc += loss.double()[0]
            it += 1
        hist.append(float(acc.item()) / max(nb, 1))
        if log:
            log(f"epoch {ep}: mse {hist[-1]:.3e}")
    return params, hist
