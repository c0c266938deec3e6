"""The point-sharded adjoint NFFT's host logic on CPU ranks (gloo, world size 2).

The two steps the driver calls on each rank are stood in for here by plain CPU versions
written from Algorithm 2.4 (the spread of the rank's points with the oracle's window
values, and a DFT along one axis with crop and deconvolution); the driver, the
partition of points, slabs and column blocks, and the collectives are the product's.
The assembled result must equal the oracle's Algorithm 2.4 on all points."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import inputs
from oracle import nfft as NF
from oracle import windows as W
from paper_2302_00414_gb300 import shard as SH


class CpuOps:
    """Step 1 and steps 2-3 along one axis of Algorithm 2.4 on the CPU (test stand-ins)."""

    def __init__(self, x, M, Ms, m):
        self.x, self.M, self.Ms, self.m = x, M, Ms, m

    def spread_grid(self, c):
        vals, cand, valid = NF.window_slot_values(W.KB, self.x, self.M, self.Ms, self.m)
        g = NF.spread(self.x, c.numpy(), self.Ms, self.m, NF.tensor_coeffs(vals), cand, valid)
        return torch.from_numpy(np.fft.ifftshift(g).copy())   # l stored at l mod Ms

    def fft_axis(self, t, A, B, nblk):
        M, Ms = self.M, self.Ms
        X = t.numpy().reshape(A, Ms, B)
        k = np.arange(-M // 2, M // 2)
        E = np.exp(-2j * np.pi * np.outer(k, np.arange(Ms)) / Ms)
        Y = np.einsum("il,alb->aib", E, X) / (Ms * W.what1(W.KB, k, M, Ms, self.m))[None, :, None]
        return torch.from_numpy(Y.reshape(A, nblk, M // nblk, B).transpose(1, 0, 2, 3).reshape(-1).copy())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, x, c, M, Ms, m, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = SH.point_range(x.shape[0], world, rank)
        ops = CpuOps(x[a:b], M, Ms, m)
        blk = SH.sharded_adjoint_2d(ops, SH.DistCollectives(), torch.from_numpy(c[a:b]), M, Ms, world)
        parts = [torch.empty_like(blk) for _ in range(world)]
        dist.all_gather(parts, blk)
        if rank == 0:
            out_q.put(SH.assemble(parts, M).numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("N", [3001, 4000])
def test_two_gloo_ranks_equal_single_rank_algorithm(N):
    M, sigma, m = 16, 2.0, 4
    Ms = W.oversampled_size(M, sigma)
    x = inputs.random_points(N, 2, 61)
    c = inputs.samples_complex(N, 62)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_rank_main, args=(2, _free_port(), x, c, M, Ms, m, q), nprocs=2, join=True,
                       start_method="spawn")
    got = q.get(timeout=60)
    ref = NF.adjoint_nfft(x, c, M, sigma, m).reshape(M, M)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_partition_covers_every_point_once():
    for N in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = SH.point_range(N, world, r)
                seen.extend(range(a, b))
            assert seen == list(range(N))
    with pytest.raises(ValueError):
        SH.check_split(12, 24, 5)


def test_emulated_ranks_on_cpu_match_one_rank():
    """The in-process emulation of W ranks (the path the GPU test drives) with the CPU
    stand-ins: W = 1, 2, 4 give the same fhat."""
    M, sigma, m = 16, 2.0, 3
    Ms = W.oversampled_size(M, sigma)
    x = inputs.random_points(2000, 2, 63)
    c = inputs.samples_complex(2000, 64)
    ref = NF.adjoint_nfft(x, c, M, sigma, m).reshape(M, M)
    for world in (1, 2, 4):
        ops, fs = [], []
        for r in range(world):
            a, b = SH.point_range(2000, world, r)
            ops.append(CpuOps(x[a:b], M, Ms, m))
            fs.append(torch.from_numpy(c[a:b]))
        got = SH.assemble(SH.emulate_ranks(ops, fs, M, Ms), M).numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
