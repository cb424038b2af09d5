"""Pair sharding across ranks and the one exchange step of the path.

The (i, j) pairs are independent work items (the paper runs its matrix
elements as parallel batches, App. B), so a multi-process run gives each rank
a disjoint set of pairs, balanced by estimated cost, and gathers the
(i, j, H_ij, S_ij) results to rank 0 before the small eigenproblem.  Every
rank holds all states; no collective touches the data path.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Sequence, Tuple

import numpy as np


def pair_cost(bond_i: Sequence[int], bond_j: Sequence[int], mpo_dims: Sequence[int], same: bool) -> float:
    """Work estimate of one pair: contraction GEMMs plus, if rotated, the gate SVDs."""
    N = len(bond_i) - 1
    c = 0.0
    for t in range(N):
        ci, cj, cj2, ci2 = bond_i[t], bond_j[t], bond_j[t + 1], bond_i[t + 1]
        c += 2.0 * ci * mpo_dims[t] * cj * 4 * cj2 + 2.0 * ci2 * 4 * ci * mpo_dims[t + 1] * cj2
    if not same:
        chi = max(bond_j)
        c += (N * (N - 1) / 2) * 12.0 * (4 * chi) ** 3 / 64.0
    return c


def partition_pairs(pairs: Sequence[Tuple[int, int]], costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time greedy split: indices of `pairs` per rank."""
    order = sorted(range(len(pairs)), key=lambda k: (-costs[k], k))
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + costs[k], r))
    for r in range(world):
        out[r].sort()
    return out


def gather_to_root(local: Dict[Tuple[int, int], Tuple[float, float]], M: int, rank: int, world: int):
    """Gather every rank's {(i, j): (H_ij, S_ij)} to rank 0 as symmetric M x M matrices.

    Uses torch.distributed object collectives (gloo or NCCL); returns
    (H, S) on rank 0 and (None, None) elsewhere.  Raises if a pair is missing.
    """
    import torch.distributed as dist
    parts = [None] * world if rank == 0 else None
    dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None, None
    H = np.full((M, M), np.nan)
    S = np.full((M, M), np.nan)
    for part in parts:
        for (i, j), (h, s) in part.items():
            H[i, j] = H[j, i] = h
            S[i, j] = S[j, i] = s
    if np.isnan(H).any():
        raise RuntimeError("pairs missing after the gather")
    return H, S
