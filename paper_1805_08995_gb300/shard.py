"""Splitting a pair list across GPUs (one process per GPU).

Image pairs are matched independently, so the data-parallel split needs no
collective on the data path: each rank matches its own share of the pairs
and the match lists are concatenated afterwards.  Work per pair grows with
N_A * N_B (lookup entries), so the split balances that product.
"""
from __future__ import annotations

import heapq

import numpy as np


def pair_costs(pairs: np.ndarray, img_off: np.ndarray) -> np.ndarray:
    sizes = np.diff(np.asarray(img_off, np.int64))
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    return sizes[pairs[:, 0]] * sizes[pairs[:, 1]] + sizes[pairs[:, 0]]


def shard_pairs(pairs: np.ndarray, img_off: np.ndarray, world: int, rank: int) -> np.ndarray:
    """Indices (ascending) of the pairs rank `rank` of `world` matches.

    Greedy longest-processing-time assignment: pairs in decreasing cost (ties
    by index) go to the least-loaded rank (ties by rank).  Deterministic, so
    every rank computes the same split without communicating."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    cost = pair_costs(pairs, img_off)
    order = np.lexsort((np.arange(len(cost)), -cost))
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(cost), np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(cost[i]), r))
    return np.nonzero(owner == rank)[0]


def images_of(pairs: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Images a shard touches (its codes are all a rank needs to build)."""
    return np.unique(np.asarray(pairs).reshape(-1, 2)[idx])


def merge_shards(P: int, parts) -> tuple:
    """Reassembles (match_off, matches) in input pair order from per-rank
    results [(pair_indices, match_off, matches), ...]."""
    counts = np.zeros(P, np.int64)
    lists = [None] * P
    for idx, off, mt in parts:
        off = np.asarray(off, np.int64)
        for k, i in enumerate(idx):
            lists[int(i)] = np.asarray(mt[off[k]:off[k + 1]], np.uint32)
            counts[int(i)] = off[k + 1] - off[k]
    moff = np.zeros(P + 1, np.uint64)
    moff[1:] = np.cumsum(counts)
    body = [x for x in lists if x is not None and len(x)]
    mt = np.concatenate(body) if body else np.zeros((0, 2), np.uint32)
    return moff, mt.reshape(-1, 2)
