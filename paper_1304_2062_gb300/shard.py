"""One image spread over several ranks: angle planes for the transforms,
spectrum rows for the diffusion.

Theorem 2 of the paper makes the diffusion of the lifted image one
independent N-vector system per frequency, while the lift, the 2-D
transforms, the restoration and the projection act on each angle plane (or
each pixel over the angles). So with P ranks, rank p owns

* the angle planes p N/P .. (p+1) N/P - 1 for the lift, the forward and
  inverse 2-D DFTs, the restoration and the projection, and
* the spectrum rows p H/P .. (p+1) H/P - 1, with all N angles and all W
  columns, for the Crank-Nicolson integration (se2n_diffuse_rows),

and every restoration interval exchanges the volume twice: planes -> rows
after the forward transform and rows -> planes after the diffusion (two
all-to-alls of N H W / P complex values per rank). The restoration and the
projection need h(t) = max over all N angles, which one all-reduce (max) of
the ranks' per-pixel maxima gives (H W floats).

The arithmetic stays in the stage entry points of the library (or, in the
tests, in the CPU oracle's stages); this module only moves data between the
shards. Two exchanges: DistExchange (one rank a process, torch.distributed:
NCCL across GPUs, point-to-point sends where the backend has no all-to-all,
as gloo on the CPU) and LocalExchange (all ranks in one process, which
hands the blocks over directly).

Static restoration and the maximum projection only (no dynamic
restoration, final restoration, reinjection or mean projection); N and H
must be multiples of P.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BIN_FLAT = 255
BIN_ELSEWHERE = 254  # a pixel lifted to an angle outside the shard


def plane_range(N, P, p):
    """Angle planes of rank p: [r0, r1)."""
    n = N // P
    return p * n, (p + 1) * n


def row_range(H, P, p):
    """Spectrum rows of rank p: [k0, k1)."""
    h = H // P
    return p * h, (p + 1) * h


def local_bins(bins, N, P, p):
    """Orientation bins renumbered for the planes of rank p: a bin inside the
    shard becomes its plane index there, a flat pixel stays flat, and a bin
    outside becomes BIN_ELSEWHERE (no plane of the shard)."""
    r0, r1 = plane_range(N, P, p)
    b = np.asarray(bins).astype(np.int64)
    out = np.where((b >= r0) & (b < r1), b - r0, BIN_ELSEWHERE)
    return np.where(b == BIN_FLAT, BIN_FLAT, out).astype(np.uint8)


@dataclasses.dataclass
class ShardParams:
    N: int
    beta: float
    T: float          # total time over all intervals
    steps: int        # Crank-Nicolson steps an interval
    rounds: int       # restoration intervals
    eps: float = 0.5
    guard: float = 0.1


class LocalExchange:
    """All P ranks live in this process (one GPU or the CPU): blocks are
    handed over without copies."""

    def __init__(self, P):
        self.P = P
        self.ranks = list(range(P))

    def all_to_all(self, send):
        """send[i][q]: block from local rank i to rank q; returns recv[i][s],
        the block rank s sent to local rank i."""
        return [[send[s][q] for s in range(self.P)] for q in range(self.P)]

    def all_reduce_max(self, parts):
        m = parts[0]
        for x in parts[1:]:
            m = m.maximum(x)
        return [m for _ in parts]



class DistExchange:
    """One rank a process over torch.distributed (the default group)."""

    def __init__(self, dist):
        self.dist = dist
        self.P = dist.get_world_size()
        self.rank = dist.get_rank()
        self.ranks = [self.rank]

    def all_to_all(self, send):
        import torch
        mine = [t.contiguous() for t in send[0]]
        recv = [torch.empty_like(t) for t in mine]
        # complex blocks travel as their real views (float pairs)
        wire = lambda t: torch.view_as_real(t) if t.is_complex() else t  # noqa: E731
        if self.dist.get_backend() == "nccl":
            self.dist.all_to_all([wire(t) for t in recv], [wire(t) for t in mine])
        else:
            ops = []
            for q in range(self.P):
                if q == self.rank:
                    recv[q].copy_(mine[q])
                    continue
                ops.append(self.dist.isend(wire(mine[q]), q))
                ops.append(self.dist.irecv(wire(recv[q]), q))
            for op in ops:
                op.wait()
        return [recv]

    def all_reduce_max(self, parts):
        t = parts[0].contiguous()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return [t]



class GpuBackend:
    """The library's stage entry points on one CUDA device: a plan of N/P
    planes a rank for the lift, transforms, restoration and projection, and
    a plan of all N angles for the row-shard diffusion."""

    def __init__(self, H, W, N, P, ranks, angle_conv=0, device=None, stream=None):
        import torch

        from . import se2n
        self.se2n = se2n
        self.torch = torch
        self.H, self.W, self.N, self.P = H, W, N, P
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.plane_plans = {p: se2n.se2n_plan_create(H, W, N // P, angle_conv, stream) for p in ranks}
        self.full_plan = se2n.se2n_plan_create(H, W, N, angle_conv, stream)

    def close(self):
        for pl in self.plane_plans.values():
            pl.close()
        self.full_plan.close()

    def upload(self, f, mask, bins_local):
        t = self.torch
        return (t.tensor(np.ascontiguousarray(f, np.float32), device=self.dev),
                t.tensor(np.ascontiguousarray(mask, np.uint8), device=self.dev),
                t.tensor(np.ascontiguousarray(bins_local, np.uint8), device=self.dev))

    def lift(self, p, f, mask, bins_local):
        vol = self.torch.empty((self.N // self.P, self.H, self.W), dtype=self.torch.complex64, device=self.dev)
        self.se2n.se2n_lift(self.plane_plans[p], f, mask, bins_local, vol)
        return vol

    def forward(self, p, vol):
        self.se2n.se2n_forward(self.plane_plans[p], vol)
        return vol

    def inverse(self, p, vol):
        self.se2n.se2n_inverse(self.plane_plans[p], vol)
        return vol

    def diffuse_rows(self, p, rows, k0, beta, T, steps):
        self.se2n.se2n_diffuse_rows(self.full_plan, rows, k0, beta, T, steps)
        return rows

    def plane_reduce(self, p, vol, proj):
        out = self.torch.empty((self.H, self.W), dtype=self.torch.float32, device=self.dev)
        self.se2n.se2n_project(self.plane_plans[p], vol, proj, out)
        return out

    def mix_given(self, p, vol, f, mask, bins_local, h_t, eps, guard):
        self.se2n.se2n_mix_given(self.plane_plans[p], vol, f, mask, bins_local, h_t, eps, guard)
        return vol

    def cat(self, parts, dim):
        return self.torch.cat(parts, dim=dim)


def inpaint_sharded(backend, exchange, f, mask, bins, prm: ShardParams):
    """The whole method (lift, prm.rounds intervals of diffusion with static
    restoration in between, projection) for the ranks of `exchange` that
    live in this process. Returns {rank: projected image}."""
    P, N = exchange.P, prm.N
    H, W = np.asarray(f).shape
    if N % P or H % P:
        raise ValueError("N and H must be multiples of the rank count")
    n, h = N // P, H // P
    ranks = exchange.ranks
    inputs = {p: backend.upload(f, mask, local_bins(bins, N, P, p)) for p in ranks}
    vols = {p: backend.lift(p, *inputs[p]) for p in ranks}
    Tr = prm.T / prm.rounds
    for i in range(prm.rounds):
        # planes -> rows: rank q receives the rows of q from every rank's planes
        for p in ranks:
            backend.forward(p, vols[p])
        send = [[vols[p][:, q * h:(q + 1) * h, :].contiguous() for q in range(P)] for p in ranks]
        recv = exchange.all_to_all(send)
        rows = {p: backend.cat(recv[j], 0) for j, p in enumerate(ranks)}       # [N][h][W], planes by rank
        for p in ranks:
            backend.diffuse_rows(p, rows[p], p * h, prm.beta, Tr, prm.steps)
        # rows -> planes
        send = [[rows[p][q * n:(q + 1) * n].contiguous() for q in range(P)] for p in ranks]
        recv = exchange.all_to_all(send)
        vols = {p: backend.inverse(p, backend.cat(recv[j], 1)) for j, p in enumerate(ranks)}   # [n][H][W]
        if i < prm.rounds - 1:
            h_t = exchange.all_reduce_max([backend.plane_reduce(p, vols[p], 0) for p in ranks])
            for j, p in enumerate(ranks):
                backend.mix_given(p, vols[p], *inputs[p], h_t[j], prm.eps, prm.guard)
    outs = exchange.all_reduce_max([backend.plane_reduce(p, vols[p], 0) for p in ranks])
    return {p: outs[j] for j, p in enumerate(ranks)}
