"""Learned J closure: training data from kinetic runs, normalisation, and
training, each step a call into the CUDA library.

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
RMS of the correction itself (targets of unit variance).  This module only
sequences library calls and allocates their buffers: the kinetic runs record
their samples in-kernel (fdtd_plasma_set_recording), the scales, inputs and
targets come from fdtd_closure_scales / fdtd_closure_dataset, and training
from fdtd_mlp_init and fdtd_mlp_train_epoch.
"""
from __future__ import annotations

import ctypes

from .fdtd_plasma import MLP_NPARAMS, MlpTrainer, _check, fdtd_closure_scales_t, load_library

NIN, NHID, NPARAMS = 17, 128, MLP_NPARAMS


def _stream(device):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


def init_params(seed: int, device):
    """Seeded He-style initial parameters (fdtd_mlp_init), FP32 device tensor."""
    import torch
    lib = load_library()
    p = torch.empty(NPARAMS, dtype=torch.float32, device=device)
    _check(lib, None, lib.fdtd_mlp_init(p.data_ptr(), int(seed), _stream(p.device)))
    return p


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


def scales(samples, omega0: float, dt: float, nu_mean: float, increment: bool = True) -> dict:
    """Normalisations and the Drude part for the closure desc (see module
    doc; fdtd_closure_scales); increment=False gives the direct form
    (rho = beta = 0)."""
    import torch
    lib = load_library()
    s = samples.contiguous()
    ws_bytes = lib.fdtd_closure_workspace_bytes()
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=s.device)
    out = fdtd_closure_scales_t()
    _check(lib, None, lib.fdtd_closure_scales(s.data_ptr(), s.shape[0], float(omega0), float(dt), float(nu_mean),
                                              int(bool(increment)), ctypes.byref(out), ws.data_ptr(), ws_bytes,
                                              _stream(s.device)))
    return dict(e_scale=out.e_scale, j_scale=out.j_scale, n_scale=out.n_scale, rho=out.rho, beta=out.beta)


def dataset(samples, sc: dict):
    """Network inputs [N, 17] and targets [N] (float32 device tensors) from
    raw samples (fdtd_closure_dataset)."""
    import torch
    lib = load_library()
    s = samples.contiguous()
    n = s.shape[0]
    x = torch.empty(n, NIN, dtype=torch.float32, device=s.device)
    t = torch.empty(n, dtype=torch.float32, device=s.device)
    d = fdtd_closure_scales_t(sc["e_scale"], sc["j_scale"], sc["n_scale"], sc["rho"], sc["beta"])
    _check(lib, None, lib.fdtd_closure_dataset(s.data_ptr(), n, ctypes.byref(d), x.data_ptr(), t.data_ptr(),
                                               _stream(s.device)))
    return x, t


def train(x, t, epochs: int = 10, batch: int = 4096, lr: float = 2e-3, seed: int = 0, log=None):
    """Adam on the mean-squared error, cosine-decayed learning rate, seeded
    shuffles (fdtd_mlp_train_epoch per epoch); returns (params, per-epoch
    mean losses)."""
    params = init_params(seed, x.device)
    tr = MlpTrainer(params, batch, lr=lr)
    nb = x.shape[0] // batch
    total = max(epochs * nb, 1)
    hist = []
    for ep in range(epochs):
        hist.append(float(tr.epoch(x, t, seed + 1, ep, ep * nb, total).item()))
        if log:
            log(f"epoch {ep}: mse {hist[-1]:.3e}")
    return params, hist
