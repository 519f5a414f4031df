"""One image spread over several ranks (paper_1304_2062_gb300/shard.py) on
the CPU: the sharded method, with the FP64 oracle's stages as the
arithmetic, must give bitwise the oracle's single-rank result, both with
every rank in one process and with two gloo ranks exchanging over
torch.distributed (point-to-point sends: gloo has no all-to-all).

Every stage is per plane (lift, 2-D transforms), per frequency (the
diffusion, Theorem 2) or per pixel (restoration, projection), and the
maximum over the angles is exact in any order, so splitting the planes and
the frequency rows over the ranks changes no bit of the result.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
import synth
from paper_1304_2062_gb300 import shard


class OracleBackend:
    """The shard module's stage interface on CPU tensors, computed by the
    oracle (complex128)."""

    def __init__(self, H, W, N, P, f, mask, bins):
        self.H, self.W, self.N, self.P = H, W, N, P
        self.h0 = oracle.lift(f, mask, bins, N).real.max(axis=0)

    def upload(self, f, mask, bins_local):
        return np.asarray(f, np.float64), np.asarray(mask, np.uint8), np.asarray(bins_local, np.uint8)

    def lift(self, p, f, mask, bins_local):
        return torch.from_numpy(oracle.lift(f, mask, bins_local, self.N // self.P))

    def forward(self, p, vol):
        vol.copy_(torch.from_numpy(oracle.forward(vol.numpy())))
        return vol

    def inverse(self, p, vol):
        vol.copy_(torch.from_numpy(oracle.inverse(vol.numpy())))
        return vol

    def diffuse_rows(self, p, rows, k0, beta, T, steps):
        h = rows.shape[1]
        full = np.zeros((self.N, self.H, self.W), np.complex128)
        full[:, k0:k0 + h] = rows.numpy()
        kk, ll = np.meshgrid(np.arange(k0, k0 + h), np.arange(self.W), indexing="ij")
        out = oracle.diffuse(full, beta, T, steps, freqs=(kk * self.W + ll).ravel())
        rows.copy_(torch.from_numpy(np.ascontiguousarray(out[:, k0:k0 + h])))
        return rows

    def plane_reduce(self, p, vol, proj):
        return torch.from_numpy(oracle.project(vol.numpy(), proj))

    def mix_given(self, p, vol, f, mask, bins_local, h_t, eps, guard):
        vol.copy_(torch.from_numpy(oracle.mix(vol.numpy(), f, mask, bins_local, eps, guard, ht=h_t.numpy(),
                                              h0=self.h0)))
        return vol

    def cat(self, parts, dim):
        return torch.cat(parts, dim=dim)


def _case(H=32, W=24, N=16):
    w = synth.workload_512(H=H, W=W, steps=20, rounds=3)
    f = w.f.astype(np.float32).astype(np.float64)
    bins = oracle.orient(f, w.mask, N)["bins"]
    prm = shard.ShardParams(N=N, beta=0.25, T=6.0, steps=20, rounds=3)
    ref = oracle.inpaint(f, w.mask, oracle.Params(N=N, beta=0.25, T=6.0, steps=20, rounds=3), bins=bins)["out"]
    return f, w.mask, bins, prm, ref


def test_local_bins_name_only_the_shards_planes():
    bins = np.array([[0, 3, 4, 7], [255, 5, 2, 6]], np.uint8)
    np.testing.assert_array_equal(shard.local_bins(bins, 8, 2, 0), [[0, 3, 254, 254], [255, 254, 2, 254]])
    np.testing.assert_array_equal(shard.local_bins(bins, 8, 2, 1), [[254, 254, 0, 3], [255, 1, 254, 2]])
    assert shard.plane_range(32, 4, 3) == (24, 32) and shard.row_range(512, 4, 1) == (128, 256)


@pytest.mark.parametrize("P", [1, 2, 4])
def test_sharded_in_one_process_is_bitwise_the_single_rank_result(P):
    f, mask, bins, prm, ref = _case()
    H, W = f.shape
    outs = shard.inpaint_sharded(OracleBackend(H, W, prm.N, P, f, mask, bins), shard.LocalExchange(P), f, mask,
                                 bins, prm)
    for p in range(P):
        np.testing.assert_array_equal(outs[p].numpy(), ref)


def test_sharding_rejects_uneven_splits():
    f, mask, bins, prm, _ = _case()
    with pytest.raises(ValueError):
        shard.inpaint_sharded(OracleBackend(32, 24, 16, 3, f, mask, bins), shard.LocalExchange(3), f, mask, bins,
                              prm)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f, mask, bins, prm, ref = _case()
        H, W = f.shape
        outs = shard.inpaint_sharded(OracleBackend(H, W, prm.N, world, f, mask, bins), shard.DistExchange(dist), f,
                                     mask, bins, prm)
        q.put((rank, bool(np.array_equal(outs[rank].numpy(), ref)), float(np.abs(outs[rank].numpy() - ref).max())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_are_bitwise_the_single_rank_result():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(r for r, _, _ in res) == [0, 1]
    for rank, same, diff in res:
        assert same, (rank, diff)
