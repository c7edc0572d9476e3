"""Receiver sharding over ranks, one GPU per rank.

Given the tree, receivers are independent (Sec. 2.5: every active element
traces its own rays), so a radiation step splits over ranks by receiver with
no exchange inside the walk:

- every rank builds the same tree (the build is about 1% of the work);
- the active receivers are put in Morton order (the tree's element order,
  so neighbouring receivers share cells and cache lines) and cut into
  contiguous, nearly equal ranges, one per rank;
- J is gathered (each row comes from exactly one rank, no reduction);
- the adjoint's outputs are sums over receivers, so each rank differentiates
  its own rows and the per-element gradients are summed across ranks.

The per-rank computation is passed in as a function, so the same host logic
runs with the CUDA library on GPU ranks or with any other J on CPU ranks.
"""

from __future__ import annotations

import numpy as np
import torch

__all__ = ["morton_rank", "shard_ranges", "local_rows", "gather_rows", "J_sharded",
           "J_backward_sharded", "tree_morton_rank"]


def morton_rank(sorted_index_of_element, active) -> np.ndarray:
    """Positions of `active` in Morton order: argsort of the receivers' places
    in the tree's element order (key, then caller index), stable."""
    key = np.asarray(sorted_index_of_element)[np.asarray(active, dtype=np.int64)]
    return np.argsort(key, kind="stable")


def tree_morton_rank(tree, active) -> np.ndarray:
    """morton_rank for a GPU tree (uses its sorted-to-caller permutation)."""
    perm = tree.export("perm").cpu().numpy().astype(np.int64)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return morton_rank(inv, active)


def shard_ranges(A: int, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges of [0, A), sizes differing by at most one."""
    base, extra = divmod(int(A), int(world))
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def local_rows(order, world: int, rank: int) -> np.ndarray:
    """Rows of the active list (positions into it) that `rank` walks."""
    lo, hi = shard_ranges(len(order), world)[rank]
    return np.asarray(order[lo:hi], dtype=np.int64)


def gather_rows(local: torch.Tensor, rows: np.ndarray, A: int, group=None) -> torch.Tensor:
    """Assembles the full [A, ...] array from every rank's rows (all-gather of
    equal-size padded blocks, then a scatter into place)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = torch.tensor([len(rows)], dtype=torch.int64, device=local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    cap = int(max(int(s.item()) for s in sizes))
    tail = tuple(local.shape[1:])
    pad = torch.zeros((cap,) + tail, dtype=local.dtype, device=local.device)
    pad[:len(rows)] = local
    idx = torch.full((cap,), -1, dtype=torch.int64, device=local.device)
    idx[:len(rows)] = torch.as_tensor(rows, dtype=torch.int64, device=local.device)
    blocks = [torch.empty_like(pad) for _ in range(world)]
    idxs = [torch.empty_like(idx) for _ in range(world)]
    dist.all_gather(blocks, pad, group=group)
    dist.all_gather(idxs, idx, group=group)
    out = torch.empty((A,) + tail, dtype=local.dtype, device=local.device)
    for b, i in zip(blocks, idxs):
        keep = i >= 0
        out[i[keep]] = b[keep]
    return out


def J_sharded(order, active, compute_J, group=None) -> torch.Tensor:
    """J for all of `active`, each rank walking its Morton range:
    compute_J(active_subset) -> [len, nb] tensor."""
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    rows = local_rows(order, world, rank)
    active = np.asarray(active, dtype=np.int64)
    local = compute_J(active[rows])
    return gather_rows(local, rows, len(active), group)


def J_backward_sharded(order, active, gJ, compute_backward, group=None):
    """Per-element gradients of sum(gJ * J): each rank differentiates its own
    rows, compute_backward(active_subset, gJ_subset) -> tuple of tensors, and
    the results are summed over ranks (in place, returned)."""
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    rows = local_rows(order, world, rank)
    active = np.asarray(active, dtype=np.int64)
    rows_t = torch.as_tensor(rows, dtype=torch.int64, device=gJ.device)
    grads = compute_backward(active[rows], gJ[rows_t])
    for g in grads:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return grads
