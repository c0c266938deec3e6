"""Point-sharded adjoint NFFT over several ranks, one GPU each (d = 2).

The adjoint NFFT of Algorithm 2.4 is linear in the samples, so a point set split over W
ranks is reconstructed from the ranks' parts:

  1. every rank spreads its own points into a whole oversampled grid (step 1,
     infft_spread_grid; with W f for density compensation, Algorithm 3.7);
  2. a reduce-scatter sums the W grids and leaves rank r the slab of grid rows
     [r M_sigma/W, (r+1) M_sigma/W);
  3. every rank transforms its slab along the second axis, crops to I_M and deconvolves
     (steps 2-3 along that axis, infft_fft_axis), writing the result as W column blocks;
  4. an all-to-all sends column block c to rank c, which then holds all M_sigma rows of
     the M/W columns [c M/W, (c+1) M/W);
  5. every rank transforms its columns along the first axis, crops and deconvolves.

Rank r ends with fhat[:, r M/W : (r+1) M/W] (C order over I_M, first index k_0 + M/2).  The
sums over ranks in step 2 change only the order of the additions, so the result equals the
single-GPU adjoint to rounding.  There is one data exchange per axis change, as the
transform needs, and nothing else crosses between ranks.  This is an extension of the
method to several devices; the paper has no multi-device part.

The steps run in the library's kernels (``GpuOps``); the collectives are
``torch.distributed`` calls (``DistCollectives``), or an in-process emulation of the ranks
(``emulate_ranks``) where one process drives every rank's part in turn.
"""
from __future__ import annotations

from typing import List, Sequence


def point_range(N: int, world: int, rank: int):
    """The contiguous block of the caller's point order that rank `rank` spreads."""
    return (rank * N) // world, ((rank + 1) * N) // world


def check_split(M: int, Ms: int, world: int):
    """The slab and column splits need W | M_sigma and W | M."""
    if Ms % world or M % world:
        raise ValueError(f"{world} ranks do not divide M_sigma = {Ms} and M = {M}")


class GpuOps:
    """The library's steps on one rank's plan (device tensors)."""

    def __init__(self, plan, mode: int, stream=None):
        from . import api as A
        self.A, self.plan, self.mode, self.stream = A, plan, mode, stream

    def spread_grid(self, f):
        import torch
        p = self.plan
        grid = torch.empty((p.Ms,) * p.d, dtype=f.dtype, device=f.device)
        self.A._check(self.A.infft_spread_grid(p.handle, self.mode, f.data_ptr(), grid.data_ptr(),
                                               self.A._stream(self.stream)))
        return grid

    def fft_axis(self, x, A: int, B: int, nblk: int):
        import torch
        p = self.plan
        out = torch.empty(A * p.M * B, dtype=x.dtype, device=x.device)
        self.A._check(self.A.infft_fft_axis(p.handle, self.mode, A, B, nblk, x.data_ptr(), out.data_ptr(),
                                            self.A._stream(self.stream)))
        return out


class DistCollectives:
    """reduce-scatter and all-to-all over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def reduce_scatter(self, x):
        import torch
        flat = x.reshape(-1)
        out = torch.empty(flat.numel() // self.world, dtype=x.dtype, device=x.device)
        self.dist.reduce_scatter_tensor(out, flat, group=self.group)
        return out

    def all_to_all(self, x):
        import torch
        out = torch.empty_like(x)
        self.dist.all_to_all_single(out, x, group=self.group)
        return out


def sharded_adjoint_2d(ops, coll, f_local, M: int, Ms: int, world: int):
    """Steps 1-5 above on one rank; returns this rank's M x M/W block of fhat (flat, C order)."""
    check_split(M, Ms, world)
    g = ops.spread_grid(f_local)                                   # 1. whole grid, own points
    slab = coll.reduce_scatter(g)                                  # 2. rows of this rank, summed
    rows = ops.fft_axis(slab, Ms // world, 1, world)               # 3. along x, W column blocks
    cols = coll.all_to_all(rows)                                   # 4. all rows of own columns
    return ops.fft_axis(cols, 1, M // world, 1)                    # 5. along y


# --- in-process emulation of the ranks ------------------------------------------------

def emulate_ranks(ops: Sequence, fs: Sequence, M: int, Ms: int) -> List:
    """Run the W ranks' parts in one process, in turn (the ranks never wait on each other
    inside a kernel): the collectives are done on the tensors here.  ops[r], fs[r]: rank r's
    steps and samples.  Returns the W blocks of fhat."""
    import torch
    W = len(ops)
    check_split(M, Ms, W)
    grids = [ops[r].spread_grid(fs[r]).reshape(-1) for r in range(W)]
    total = grids[0].clone()
    for r in range(1, W):
        total += grids[r]                                           # the reduce of step 2
    n = total.numel() // W
    rows = [ops[r].fft_axis(total[r * n:(r + 1) * n], Ms // W, 1, W) for r in range(W)]
    b = rows[0].numel() // W                                        # one block of step 4
    cols = [torch.cat([rows[s][c * b:(c + 1) * b] for s in range(W)]) for c in range(W)]
    return [ops[c].fft_axis(cols[c], 1, M // W, 1) for c in range(W)]


def assemble(blocks: Sequence, M: int):
    """fhat (M x M) from the W column blocks (M x M/W each, flat)."""
    import torch
    W = len(blocks)
    return torch.cat([blk.reshape(M, M // W) for blk in blocks], dim=1)
