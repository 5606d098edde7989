"""Learned J closure on the GPU, through the C ABI, against the FP64 oracle
(oracle/mlp.py) and against the kinetic solve it stands in for.

Tolerances: the network runs with BF16 tensor-core operands and FP32
accumulation, so forward values and gradients are compared with relative L2
bounds of 1e-2 / 3e-2; Adam (pure FP32) at 1e-5."""
import math

import numpy as np
import pytest

from fdtd_inputs import OMEGA0, spec_1d_slab, spec_2d_cylinder
from oracle import mlp as M
from tests.adapters import oracle_sim, rel_l2

pytestmark = pytest.mark.gpu


def _flat_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = M.init_params(rng)
    P["b1"] = rng.standard_normal(128) * 0.1
    P["b2"] = rng.standard_normal(128) * 0.1
    P["b3"] = rng.standard_normal(1) * 0.1
    flat = np.concatenate([P["W1"].ravel(), P["b1"], P["W2"].ravel(), P["b2"], P["W3"].ravel(), P["b3"]]) * scale
    return flat.astype(np.float32)


def _oracle_params(flat):
    f = flat.astype(np.float64)
    o = 0
    out = {}
    for k, shp in (("W1", (17, 128)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 1)),
                   ("b3", (1,))):
        n = int(np.prod(shp))
        out[k] = f[o:o + n].reshape(shp)
        o += n
    assert o == 18945
    return out


def test_mlp_forward_matches_oracle():
    import torch
    from paper_2211_05647_gb300 import mlp_forward
    flat = _flat_params(1)
    x = np.random.default_rng(2).standard_normal((1000, 17)).astype(np.float32)   # 7 full tiles + a ragged one
    y = mlp_forward(torch.from_numpy(flat).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    yo, _ = M.forward(_oracle_params(flat), x.astype(np.float64))
    err = rel_l2(y, yo)
    print(f"mlp forward rel L2 vs FP64: {err:.3e}")
    assert err <= 1e-2


def test_mlp_forward_tcgen05_matches_oracle_and_mma():
    """The tcgen05 (tensor-memory accumulator) forward against the FP64 oracle
    and against the mma.sync forward: same BF16 roundings of the operands,
    different accumulation order only."""
    import torch
    from paper_2211_05647_gb300 import mlp_forward, mlp_forward_tc
    flat = _flat_params(21)
    x = np.random.default_rng(22).standard_normal((5000, 17)).astype(np.float32)
    p, xt = torch.from_numpy(flat).cuda(), torch.from_numpy(x).cuda()
    y_tc, err = mlp_forward_tc(p, xt)
    y_mma = mlp_forward(p, xt)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    y_tc, y_mma = y_tc.cpu().numpy(), y_mma.cpu().numpy()
    yo, _ = M.forward(_oracle_params(flat), x.astype(np.float64))
    e_or, e_mma = rel_l2(y_tc, yo), rel_l2(y_tc, y_mma)
    print(f"tcgen05 forward: rel L2 vs FP64 {e_or:.3e}, vs mma.sync {e_mma:.3e}")
    assert e_or <= 1e-2 and e_mma <= 2e-3


def test_mlp_loss_grad_matches_oracle():
    import torch
    from paper_2211_05647_gb300 import MlpTrainer
    flat = _flat_params(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((777, 17)).astype(np.float32)
    t = rng.standard_normal(777).astype(np.float32)
    p = torch.from_numpy(flat).cuda()
    tr = MlpTrainer(p, 1024)
    loss, g = tr.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    L, go = M.loss_and_grads(_oracle_params(flat), x.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss.item()) - L) <= 2e-2 * L
    gg = _oracle_params(g.cpu().numpy())
    for k in go:
        e = rel_l2(gg[k], go[k])
        print(f"grad {k}: rel L2 {e:.3e}")
        assert e <= 3e-2, k


def test_mlp_adam_matches_oracle():
    import torch
    from paper_2211_05647_gb300 import fdtd_plasma as F
    lib = F.load_library()
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(18945).astype(np.float32)
    m0 = (rng.standard_normal(18945) * 0.1).astype(np.float32)
    v0 = (rng.random(18945) * 0.01).astype(np.float32)
    g = rng.standard_normal(18945).astype(np.float32)
    tp, tm, tv, tg = (torch.from_numpy(a.copy()).cuda() for a in (p0, m0, v0, g))
    assert lib.fdtd_mlp_adam(tp.data_ptr(), tg.data_ptr(), tm.data_ptr(), tv.data_ptr(), 18945, 7, 1e-3, 0.9, 0.999,
                             1e-8, None) == 0
    torch.cuda.synchronize()
    P = {"w": p0.astype(np.float64)}
    st = {"t": 6, "m": {"w": m0.astype(np.float64)}, "v": {"w": v0.astype(np.float64)}}
    M.adam_step(P, {"w": g.astype(np.float64)}, st, lr=1e-3)
    assert np.allclose(tp.cpu().numpy(), P["w"], rtol=1e-5, atol=1e-6)


def test_recorder_matches_oracle_history(oracle_lib):
    """One plasma cell, every step recorded: sample n is [E^{n-15..n}, n, J^{n+1/2}, J^{n-1/2}]."""
    import torch
    from paper_2211_05647_gb300 import Solver
    spec = spec_1d_slab(nz=300, slab=(150, 151), src_k=40, precision="f32", steps=400, wp_w0=0.9)
    s = Solver.from_spec(spec)
    buf = torch.zeros(400 * 19, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.set_recording(buf, cnt, 1.0, 7)
    s.step(400)
    torch.cuda.synchronize()
    assert int(cnt.item()) == 400
    rec = buf.view(400, 19).cpu().numpy().astype(np.float64)
    sim = oracle_sim(oracle_lib, spec)
    E, J = [], []
    for _ in range(400):
        E.append(sim.get("ex")[150])
        sim.step(1)
        J.append(sim.get("j")[0])
    E = np.array(E); J = np.array(J)
    hist = np.stack([np.concatenate([np.zeros(max(0, 15 - n)), E[max(0, n - 15):n + 1]]) for n in range(400)])
    scale = np.abs(E).max()
    assert np.abs(rec[:, :16] - hist).max() <= 1e-4 * scale
    assert np.all(rec[:, 16] == np.float32(spec["plasma"]["density"][150]))
    jscale = np.abs(J).max()
    assert jscale > 0
    assert np.abs(rec[:, 17] - J).max() <= 1e-4 * jscale
    assert np.abs(rec[1:, 18] - J[:-1]).max() <= 1e-4 * jscale and rec[0, 18] == 0


def _closure_spec():
    return spec_2d_cylinder(n=160, ny=120, R=30, center=(95, 60), src=(50, 60), steps=80, seed=9)


def test_closure_constant_network():
    """A network that outputs the constant b3 gives J_n = J_s b3 (1 - rho^{n+1}) / (1 - rho)."""
    from paper_2211_05647_gb300 import Solver
    spec = _closure_spec()
    s = Solver.from_spec(spec)
    flat = np.zeros(18945, np.float32)
    flat[-1] = 0.25
    rho, js = 0.97, 3.0e-2
    s.set_closure(flat, e_scale=1.0, j_scale=js, n_scale=1e18, rho=rho, n_train_max=1e30)
    nk, nc = s.closure_shape()
    assert nk == 0 and nc > 0
    s.step(50)
    J = s.read("j", device=False)
    want = js * 0.25 * (1 - rho ** 50) / (1 - rho)
    assert np.allclose(J, want, rtol=1e-5)


@pytest.mark.parametrize("engine", ["mma", "tcgen05"])
def test_closure_inference_matches_oracle_forward(engine):
    """In-solver closure: after stepping, J of every closure cell equals
    rho J_prev + beta n E^n + J_s MLP(x) with x rebuilt from the E history it
    saw (FP64 oracle forward)."""
    from paper_2211_05647_gb300 import Solver
    spec = _closure_spec()
    s = Solver.from_spec(spec)
    flat = _flat_params(11, scale=0.5)
    dens = spec["plasma"]["density"]
    cells = np.nonzero(dens > 0)[0]
    cells = cells[(cells % 160 >= 1) & (cells // 160 >= 1)]
    nmax = dens.max()
    e_s, j_s, n_s, rho, beta = 0.05, 1e-3, 1e18, 0.95, 3e-21
    s.set_closure(flat, e_scale=e_s, j_scale=j_s, n_scale=n_s, rho=rho, n_train_max=nmax, beta=beta, engine=engine)
    hist = []
    Jprev = np.zeros(len(cells))
    for n in range(60):
        hist.append(s.read("ez", device=False)[cells].astype(np.float64))
        s.step(1)
        J = s.read("j", device=False).astype(np.float64)
        if n == 59:
            H = np.stack(hist[-16:], axis=1) / e_s
            x = np.concatenate([H, (dens[cells] / n_s)[:, None]], axis=1)
            y, _ = M.forward(_oracle_params(flat), x)
            want = rho * Jprev + beta * dens[cells] * hist[-1] + j_s * y
            err = rel_l2(J, want)
            print(f"closure ({engine}) J vs oracle forward: {err:.3e}")
            assert err <= 1e-2
        Jprev = J
    assert s.diagnostics()["finite"]


@pytest.mark.slow
def test_trained_closure_tracks_kinetic_solve():
    """Train on kinetic runs of three seeded density fields, run the closure
    on a fourth: field error against the kinetic solve of the same grid."""
    import torch
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300 import closure as C

    def spec(seed):
        return spec_2d_cylinder(n=256, R=64, center=(150, 128), src=(60, 128), steps=700, seed=seed)

    samples = torch.cat([C.record_samples(spec(100 + k), 700, 0.12, 31 + k, 1_500_000) for k in range(3)])
    sp = spec(7)
    dt = Solver.from_spec(sp).dt
    sc = C.scales(samples, OMEGA0, dt, sp["plasma"]["nu0"])
    x, t = C.dataset(samples, sc)
    params, hist = C.train(x, t, epochs=8, batch=4096, lr=2e-3, seed=3, log=print)
    assert hist[-1] < 0.5 * hist[0]
    kin = Solver.from_spec(sp)
    kin.step(700)
    nmax = float(np.max([np.max(spec(100 + k)["plasma"]["density"]) for k in range(3)]))
    errs = {}
    for name, p in (("drude only", torch.zeros_like(params)), ("trained", params)):
        clo = Solver.from_spec(sp)
        clo.set_closure(p, n_train_max=nmax, **sc)
        clo.step(700)
        errs[name] = max(rel_l2(clo.read(f, device=False), kin.read(f, device=False)) for f in ("ez", "hx", "hy"))
        assert clo.closure_shape()[1] > 0
    print(f"closure vs kinetic after 700 steps (max rel L2 over Ez, Hx, Hy): {errs}")
    assert errs["trained"] <= 1e-2
    assert errs["trained"] < errs["drude only"]


def _random_samples(n, seed):
    rng = np.random.default_rng(seed)
    s = np.zeros((n, 19), np.float32)
    s[:, :16] = rng.standard_normal((n, 16)) * 0.3
    s[:, 16] = rng.uniform(1e17, 8e17, n)
    s[:, 18] = rng.standard_normal(n) * 1e-2
    s[:, 17] = 0.99 * s[:, 18] + rng.standard_normal(n) * 1e-4
    return s


@pytest.mark.parametrize("increment", [True, False])
def test_closure_scales_and_dataset_match_oracle(increment):
    """fdtd_closure_scales / fdtd_closure_dataset against the FP64 oracle
    (oracle/closure_data.py): scales to FP64 rounding, inputs and targets to
    one FP32 rounding (both sides form them in FP64), on a ragged count."""
    import torch
    from oracle import closure_data as CD
    from paper_2211_05647_gb300 import closure as C
    s = _random_samples(300_001, 8)
    dt, nu = 1.25e-12, 0.01 * OMEGA0
    sd = torch.from_numpy(s).cuda()
    sc = C.scales(sd, OMEGA0, dt, nu, increment=increment)
    so = CD.scales(s, OMEGA0, dt, nu, increment=increment)
    for k in so:
        assert abs(sc[k] - so[k]) <= 1e-12 * abs(so[k]), (k, sc[k], so[k])
    x, t = C.dataset(sd, sc)
    xo, to = CD.dataset(s, so)
    x, t = x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(x, xo, rtol=2.4e-7, atol=0)
    np.testing.assert_allclose(t, to, rtol=2.4e-7, atol=1e-30)
    print(f"closure scales (increment={increment}): {sc}")


def test_mlp_gather_is_a_seeded_permutation():
    """Every batch of an epoch is a disjoint slice of one permutation of the
    samples (all of them when the batch divides n); rows are copied whole;
    another epoch gives another order, the same epoch the same one."""
    import torch
    from paper_2211_05647_gb300 import fdtd_plasma as F
    lib = F.load_library()
    for n, batch in ((8192, 1024), (10_007, 1000)):
        x = torch.arange(n * 17, dtype=torch.float32, device="cuda").view(n, 17)
        t = torch.arange(n, dtype=torch.float32, device="cuda")
        xb = torch.empty(batch, 17, dtype=torch.float32, device="cuda")
        tb = torch.empty(batch, dtype=torch.float32, device="cuda")

        def order(epoch):
            idx = []
            for b in range(n // batch):
                assert lib.fdtd_mlp_gather(x.data_ptr(), t.data_ptr(), n, 77, epoch, b * batch, batch, xb.data_ptr(),
                                           tb.data_ptr(), None) == 0
                torch.cuda.synchronize()
                i = tb.cpu().numpy().astype(np.int64)
                assert np.array_equal(xb.cpu().numpy(), x.cpu().numpy()[i])
                idx.append(i)
            return np.concatenate(idx)

        o0, o0b, o1 = order(0), order(0), order(1)
        assert np.unique(o0).size == o0.size == (n // batch) * batch
        assert o0.min() >= 0 and o0.max() < n
        if n % batch == 0:
            assert np.array_equal(np.sort(o0), np.arange(n))
        assert np.array_equal(o0, o0b) and not np.array_equal(o0, o1)
        assert abs(np.corrcoef(np.arange(o0.size), o0)[0, 1]) < 0.05     # shuffled, not near-identity


def test_mlp_init_statistics():
    """He-style initial weights: zero biases, per-layer standard deviations
    sqrt(2/17), sqrt(2/128), sqrt(1/128), zero mean; seeded."""
    from paper_2211_05647_gb300 import closure as C
    p = C.init_params(5, "cuda").cpu().numpy().astype(np.float64)
    q = C.init_params(5, "cuda").cpu().numpy()
    r = C.init_params(6, "cuda").cpu().numpy()
    assert np.array_equal(p.astype(np.float32), q) and not np.array_equal(q, r)
    P = _oracle_params(p.astype(np.float32))
    for b in ("b1", "b2", "b3"):
        assert np.all(P[b] == 0)
    for w, sd in (("W1", math.sqrt(2 / 17)), ("W2", math.sqrt(2 / 128)), ("W3", math.sqrt(1 / 128))):
        v = P[w].ravel()
        assert abs(v.std() / sd - 1) < 6 / math.sqrt(v.size) + 0.01, w
        assert abs(v.mean()) < 5 * sd / math.sqrt(v.size), w


def test_train_epoch_equals_its_steps():
    """fdtd_mlp_train_epoch = gather + loss/grad + Adam (cosine-decayed rate,
    step count iter0 + b + 1) per batch, bit for bit (the tiles' gradients are
    summed in a fixed order); its mean loss is the mean of the batch losses."""
    import torch
    from paper_2211_05647_gb300 import MlpTrainer
    from paper_2211_05647_gb300 import closure as C
    from paper_2211_05647_gb300 import fdtd_plasma as F
    lib = F.load_library()
    rng = np.random.default_rng(12)
    n, batch, lr, total = 5000, 1024, 2e-3, 12
    x = torch.from_numpy(rng.standard_normal((n, 17)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    pa = C.init_params(3, "cuda")
    pb = pa.clone()
    ta = MlpTrainer(pa, batch, lr=lr)
    mean = float(ta.epoch(x, t, 9, 1, 4, total).item())
    tb_ = MlpTrainer(pb, batch, lr=lr)
    xb = torch.empty(batch, 17, dtype=torch.float32, device="cuda")
    tb = torch.empty(batch, dtype=torch.float32, device="cuda")
    losses = []
    for b in range(n // batch):
        assert lib.fdtd_mlp_gather(x.data_ptr(), t.data_ptr(), n, 9, 1, b * batch, batch, xb.data_ptr(), tb.data_ptr(),
                                   None) == 0
        tb_.t = 4 + b
        loss = tb_.step(xb, tb, lr=lr * 0.5 * (1 + math.cos(math.pi * (4 + b) / total)))
        losses.append(float(loss.item()))
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)
    assert abs(mean - np.mean(losses)) <= 1e-6 * abs(np.mean(losses))
