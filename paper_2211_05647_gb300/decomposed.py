"""Domain decomposition of the coupled step along the grid's slowest axis.

The curl stencils (Sec. 2, Eq. 1-6) couple each cell only to its neighbours:
the H update of plane k reads E on plane k + 1, the E update of plane k reads
H on plane k - 1.  A grid split into slabs along its slowest axis (y of a 2-D
TMz grid, z of a 3-D one) therefore needs, per step,
    E halo: each slab's first owned plane of tangential E -> the ghost plane
            above the slab below it (before the H half step);
    H halo: each slab's last owned plane of tangential H -> the ghost plane
            below the slab above it (before the kinetic + E half step).
The delta-f rows, the J moment and the Ampere term are cell-local and never
move.  The library's sub-domain handles (fdtd_plasma_create_subdomain) compute
their owned cells bit for bit as the whole grid does; this module only
partitions the axis and moves the halos:
  * DecomposedSolver: several sub-domains in one process (one GPU), halos by
    device-to-device copies on one stream;
  * RankHalo / DistributedSolver: one sub-domain per rank, halos sent to the
    neighbouring ranks with torch.distributed (NCCL between GPUs; the same
    protocol runs over gloo on CPU tensors).
"""
from __future__ import annotations


def partition(n_global: int, parts: int) -> list:
    """Balanced slabs (offset, extent) covering [0, n_global): extents differ by
    at most one plane, each at least 2."""
    if parts < 1 or n_global < 2 * parts:
        raise ValueError(f"cannot split {n_global} planes into {parts} slabs of at least 2")
    base, extra = divmod(n_global, parts)
    out, off = [], 0
    for r in range(parts):
        ext = base + (1 if r < extra else 0)
        out.append((off, ext))
        off += ext
    return out


def split_axis_length(spec: dict) -> int:
    g = spec["grid"]
    if g["ndim"] not in (2, 3):
        raise ValueError("domain decomposition splits 2-D (along y) and 3-D (along z) grids")
    return int(g["ny"] if g["ndim"] == 2 else g["nz"])


def halo_steps(sub_below, sub_above, which: str, buf):
    """One interface's halo, in one process: E goes from the slab above to the
    ghost plane of the slab below, H from the slab below to the ghost plane of
    the slab above (buf: a device tensor of the halo's bytes)."""
    if which == "e":
        sub_above.halo_pack("e", buf)
        sub_below.halo_unpack("e", buf)
    else:
        sub_below.halo_pack("h", buf)
        sub_above.halo_unpack("h", buf)


class DecomposedSolver:
    """A grid as `parts` sub-domains on one device (or given `bounds`), stepped
    with halo exchanges; its fields equal the whole-grid solver's bit for bit."""

    def __init__(self, spec: dict, parts: int = 2, device: int = 0, bounds=None):
        import torch
        from .fdtd_plasma import Solver
        self.torch = torch
        self.spec = spec
        self.ndim = int(spec["grid"]["ndim"])
        self.bounds = list(bounds) if bounds is not None else partition(split_axis_length(spec), parts)
        self.subs = [Solver.from_spec(spec, device=device, subdomain=b) for b in self.bounds]
        self.stream = self.subs[0].stream
        nb = max(s.halo_bytes(w) for s in self.subs for w in ("e", "h"))
        self.buf = torch.empty(max(nb, 1), dtype=torch.uint8, device=self.subs[0].device)

    def exchange(self, which: str):
        for lo, hi in zip(self.subs[:-1], self.subs[1:]):
            halo_steps(lo, hi, which, self.buf[: lo.halo_bytes(which)])

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange("e")
            for s in self.subs:
                s.step_half(0)
            self.exchange("h")
            for s in self.subs:
                s.step_half(1)

    def read(self, name: str):
        """The global array of a field (owned planes of every slab, in order), or
        J / delta f rows concatenated in global slot order (host numpy)."""
        import numpy as np
        parts = []
        for s in self.subs:
            a = s.read(name, device=False)
            if name in ("j", "df"):
                parts.append(a)
                continue
            sd = s.subdomain
            a = a.reshape(sd["planes"], -1)
            parts.append(a[sd["lo"]:sd["lo"] + sd["extent"]])
        return np.concatenate(parts, axis=0).ravel() if name != "df" else np.concatenate(parts, axis=0)

    def close(self):
        for s in self.subs:
            s.close()


class RankHalo:
    """Halo exchange of this rank's sub-domain with the ranks holding the slabs
    below (rank - 1) and above (rank + 1), over torch.distributed.  `sub` is any
    object with halo_bytes / halo_pack / halo_unpack and a `subdomain` dict
    (lo / hi: whether it has a neighbour below / above); buffers live on
    `device` (a CUDA device for NCCL, "cpu" for gloo)."""

    def __init__(self, sub, rank: int, world: int, device, group=None):
        import torch
        self.torch = torch
        self.sub, self.rank, self.world, self.group = sub, rank, world, group
        sd = sub.subdomain
        self.below = rank - 1 if sd["lo"] else None
        self.above = rank + 1 if sd["hi"] else None
        self.send, self.recv = {}, {}
        for w in ("e", "h"):
            nb = sub.halo_bytes(w)
            self.send[w] = torch.empty(nb, dtype=torch.uint8, device=device)
            self.recv[w] = torch.empty(nb, dtype=torch.uint8, device=device)

    def exchange(self, which: str):
        """E: send the first owned plane down, receive the ghost plane above;
        H: send the last owned plane up, receive the ghost plane below."""
        dist = self.torch.distributed
        to, frm = (self.below, self.above) if which == "e" else (self.above, self.below)
        ops = []
        if to is not None:
            self.sub.halo_pack(which, self.send[which])
            ops.append(dist.P2POp(dist.isend, self.send[which], to, self.group))
        if frm is not None:
            ops.append(dist.P2POp(dist.irecv, self.recv[which], frm, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if frm is not None:
            self.sub.halo_unpack(which, self.recv[which])


class DistributedSolver:
    """One sub-domain of the grid per rank (ranks in order along the split
    axis), stepped with halo exchanges between neighbouring ranks."""

    def __init__(self, spec: dict, rank: int, world: int, device: int = 0, group=None):
        import torch
        from .fdtd_plasma import Solver
        self.bounds = partition(split_axis_length(spec), world)
        self.sub = Solver.from_spec(spec, device=device, subdomain=self.bounds[rank])
        self.halo = RankHalo(self.sub, rank, world, torch.device("cuda", device), group=group)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.halo.exchange("e")
            self.sub.step_half(0)
            self.halo.exchange("h")
            self.sub.step_half(1)

    def close(self):
        self.sub.close()
