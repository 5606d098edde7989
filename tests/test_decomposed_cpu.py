"""Host side of the domain decomposition (paper_2211_05647_gb300/decomposed.py)
on CPU: the partition of the split axis, and the halo protocol of RankHalo
over torch.distributed with gloo at world sizes 2 and 3.

The ranks step a small FP64 2-D TMz vacuum Yee grid written here in numpy
with the library's storage conventions (Ez on nodes, PEC on the low rows and
columns, zero past the high ones; Hx, Hy staggered; a point soft source), as
sub-domains with ghost rows exactly as the library lays them out, and move
their halos with the same calls a GPU sub-domain answers (halo_bytes,
halo_pack, halo_unpack).  Bit-for-bit equality with the whole grid shows the
protocol exchanges the right planes in the right order."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NY, STEPS, SRC = 21, 30, 60, (7, 17)


class MiniTMz:
    """Rows [origin, origin + planes) of the global NX x NY grid (all of it when
    bounds is None); ghost rows below / above when there is a neighbour."""

    def __init__(self, bounds=None):
        off, ext = bounds if bounds is not None else (0, NY)
        lo, hi = int(off > 0), int(off + ext < NY)
        self.subdomain = dict(lo=lo, hi=hi, offset=off, extent=ext, origin=off - lo, planes=ext + lo + hi)
        n = self.subdomain["planes"]
        self.ez, self.hx, self.hy = np.zeros((n, NX)), np.zeros((n, NX)), np.zeros((n, NX))
        self.step_no = 0

    def step_half(self, half):
        ez, hx, hy, c = self.ez, self.hx, self.hy, 0.5
        if half == 0:
            up = np.vstack([ez[1:], np.zeros((1, NX))])             # zero past the last row
            hx -= c * (up - ez)
            right = np.hstack([ez[:, 1:], np.zeros((ez.shape[0], 1))])
            hy += c * (right - ez)
            return
        upd = c * ((hy[1:, 1:] - hy[1:, :-1]) - (hx[1:, 1:] - hx[:-1, 1:]))
        ez[1:, 1:] += upd
        if self.subdomain["origin"] == 0:
            ez[0, :] = 0.0                                          # PEC row of the global grid
        ez[:, 0] = 0.0
        self.step_no += 1
        t = self.step_no * 0.05
        r = SRC[1] - self.subdomain["origin"]
        if self.subdomain["lo"] <= r < self.subdomain["lo"] + self.subdomain["extent"]:
            ez[r, SRC[0]] += np.sin(2.0 * t) * np.exp(-((t - 1.0) / 0.4) ** 2)

    # the sub-domain halo calls
    def halo_bytes(self, which):
        return NX * 8

    def halo_pack(self, which, out):
        sd = self.subdomain
        row = self.ez[sd["lo"]] if which == "e" else self.hx[sd["lo"] + sd["extent"] - 1]
        out.numpy().view(np.float64)[:] = row
        return out

    def halo_unpack(self, which, buf):
        if which == "e":
            self.ez[-1] = buf.numpy().view(np.float64)
        else:
            self.hx[0] = buf.numpy().view(np.float64)

    def owned(self):
        sd = self.subdomain
        return [a[sd["lo"]:sd["lo"] + sd["extent"]] for a in (self.ez, self.hx, self.hy)]


def _whole():
    g = MiniTMz()
    for _ in range(STEPS):
        g.step_half(0)
        g.step_half(1)
    return g.owned()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2211_05647_gb300.decomposed import RankHalo, partition
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    sub = MiniTMz(partition(NY, world)[rank])
    halo = RankHalo(sub, rank, world, torch.device("cpu"))
    for _ in range(STEPS):
        halo.exchange("e")
        sub.step_half(0)
        halo.exchange("h")
        sub.step_half(1)
    dist.barrier()
    dist.destroy_process_group()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), *sub.owned())


@pytest.mark.parametrize("world", [2, 3])
def test_rank_halo_protocol_matches_whole_grid(tmp_path, world):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    whole = _whole()
    assert np.abs(whole[0]).max() > 0
    for q in range(3):
        got = np.concatenate([p[f"arr_{q}"] for p in parts], axis=0)
        assert np.array_equal(got, whole[q]), q


def test_protocol_in_one_process_and_without_the_h_halo():
    """The same slabs stepped in one process with halo_steps equal the whole
    grid; leaving out the H halo does not (the test can fail)."""
    sys.path.insert(0, ROOT)
    import torch
    from paper_2211_05647_gb300.decomposed import halo_steps, partition
    whole = _whole()
    for skip_h in (False, True):
        subs = [MiniTMz(b) for b in partition(NY, 3)]
        buf = torch.empty(NX * 8, dtype=torch.uint8)
        for _ in range(STEPS):
            for lo, hi in zip(subs[:-1], subs[1:]):
                halo_steps(lo, hi, "e", buf)
            for s in subs:
                s.step_half(0)
            if not skip_h:
                for lo, hi in zip(subs[:-1], subs[1:]):
                    halo_steps(lo, hi, "h", buf)
            for s in subs:
                s.step_half(1)
        got = np.concatenate([s.owned()[0] for s in subs], axis=0)
        assert np.array_equal(got, whole[0]) != skip_h


def test_partition():
    sys.path.insert(0, ROOT)
    from paper_2211_05647_gb300.decomposed import partition
    for n, p in ((30, 3), (31, 4), (4096, 8), (4, 2)):
        b = partition(n, p)
        assert b[0][0] == 0 and sum(e for _, e in b) == n
        assert all(o2 == o1 + e1 for (o1, e1), (o2, _) in zip(b[:-1], b[1:]))
        assert max(e for _, e in b) - min(e for _, e in b) <= 1 and min(e for _, e in b) >= 2
    with pytest.raises(ValueError):
        partition(5, 3)
