"""Partition of independent scenes and step requests across GPUs.

The batched and served workloads consist of independent scenes: no pair ever
crosses two scenes, so the method needs no exchange between them.  With one
process per GPU, each rank takes a fixed share of the scenes, steps them in
its own batched context (or serves them with its own HBM-budget admission),
and the ranks meet only to report.  These host-side functions fix who owns
what; they are deterministic, so every rank computes the same partition
without communicating.
"""
from __future__ import annotations

import heapq

import numpy as np


def shard_scenes(sizes, world_size: int) -> list[list[int]]:
    """Balanced partition of scenes (by vertex count) over world_size ranks.

    Longest-processing-time-first: scenes in decreasing size (ties by index)
    go to the rank with the least vertices so far (ties by rank).  Each rank's
    list is returned in increasing scene index.  Every scene is owned by
    exactly one rank."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    sizes = np.asarray(sizes, np.int64)
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world_size)]
    heapq.heapify(heap)
    out: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(s) for s in out]


def owner_of(shards: list[list[int]], n_scenes: int) -> np.ndarray:
    """Rank owning each scene (inverse of shard_scenes)."""
    own = np.full(n_scenes, -1, np.int64)
    for r, s in enumerate(shards):
        own[np.asarray(s, np.int64)] = r
    if np.any(own < 0):
        raise ValueError("a scene has no owner")
    return own


def shard_requests(scene_of_request, owner: np.ndarray, rank: int) -> np.ndarray:
    """Indices of the requests (in arrival order) that rank serves: those for
    the scenes it owns.  Requests of one scene stay on one rank, in order."""
    scene_of_request = np.asarray(scene_of_request, np.int64)
    return np.nonzero(owner[scene_of_request] == rank)[0]
