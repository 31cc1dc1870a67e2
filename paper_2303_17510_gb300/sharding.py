"""Residue sharding of one convolution across ranks (one process per GPU).

The residues of a hybrid-dealiased convolution are independent: each one's
forward transforms, mult and backward transform need only the inputs, and its
backward transform is added into the output (Section 2.2, Alg. convolve; for
N-D plans the residues of the outermost axis, Section 5).  A single large
convolution therefore splits across ranks without any exchange until the end:
every rank reads the whole input, computes the partial sum over its own range
of residues (hd_convolve_residues), and one reduction (sum) of the partial
outputs gives the convolution -- an all-reduce when every rank needs the whole
result, a reduce-scatter when each keeps one slice.

This module holds the host side: which residues a rank takes and the
reduction.  The reduction runs on torch.distributed (NCCL on GPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def residue_share(n: int, rank: int, world: int):
    """Contiguous, balanced residue range [r_begin, r_end) of `rank` among
    `world` ranks: the first n % world ranks take one residue more.  Ranks
    beyond n get an empty range."""
    if n < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("residue_share: need n >= 0, world >= 1, 0 <= rank < world")
    q, r = divmod(n, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def _real_view(t: torch.Tensor) -> torch.Tensor:
    return torch.view_as_real(t) if t.is_complex() else t


def reduce_partials(partial, n: int, out: torch.Tensor, group=None, mode: str = "all_reduce"):
    """Runs partial(r_begin, r_end, out) for this rank's residue range, then
    sums the partial outputs over the group.

    mode "all_reduce": every rank ends with the whole result in `out`.
    mode "reduce_scatter": `out` keeps the partial sum and the return value is
    this rank's slice (rank k: elements [k s, (k+1) s) of the flattened output,
    s = numel / world, which must divide evenly) of the whole result.
    """
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    r0, r1 = residue_share(n, rank, world)
    partial(r0, r1, out)
    flat = _real_view(out).reshape(-1)
    if mode == "all_reduce":
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        return out
    if mode == "reduce_scatter":
        if flat.numel() % world:
            raise ValueError("reduce_scatter: the output does not split evenly over the ranks")
        part = torch.empty(flat.numel() // world, dtype=flat.dtype, device=flat.device)
        dist.reduce_scatter_tensor(part, flat, op=dist.ReduceOp.SUM, group=group)
        return torch.view_as_complex(part.view(-1, 2)) if out.is_complex() else part
    raise ValueError(f"reduce_partials: unknown mode {mode!r}")


def convolve_sharded(plan, fs, h, group=None, count: int = 1, batch_stride: int = 0, stream=None,
                     mode: str = "all_reduce"):
    """One convolution (or `count` of them) of `plan` split by residues over the
    ranks of `group`: fs are this rank's copies of the A inputs, h the output
    tensor (one output; pass a list of B tensors for multi-output mults, with
    mode "all_reduce").  Every rank launches only its own residues."""
    n = plan.residues
    if isinstance(h, (list, tuple)):
        if mode != "all_reduce":
            raise ValueError("multi-output plans reduce with all_reduce")
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        r0, r1 = residue_share(n, rank, world)
        plan.convolve_residues(fs, list(h), r0, r1, count, batch_stride, stream)
        for t in h:
            dist.all_reduce(_real_view(t).reshape(-1), op=dist.ReduceOp.SUM, group=group)
        return h
    return reduce_partials(lambda r0, r1, out: plan.convolve_residues(fs, out, r0, r1, count, batch_stride, stream),
                           n, h, group, mode)
