"""Scene and request partition across GPUs (paper_2607_26901_b300/shard.py),
on CPU: every scene and every request is owned by exactly one rank, shares
are balanced, and in a two-rank gloo run (world size 2) the results each rank
computes for its own scenes equal the single-rank results (the scenes are
independent, so no exchange is needed on the data path; the ranks meet only
to report).  The per-scene step here is the FP64 oracle's, standing in for a
rank's batched GPU context."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_26901_b300 import scenes as S
from paper_2607_26901_b300.shard import owner_of, shard_requests, shard_scenes


@pytest.mark.parametrize("ws", [1, 2, 3, 8])
def test_every_scene_owned_once_and_balanced(ws):
    rng = np.random.default_rng(4)
    sizes = np.clip(rng.lognormal(np.log(8192), np.log(2), 512), 1024, 65536).astype(np.int64)
    shards = shard_scenes(sizes, ws)
    assert len(shards) == ws
    flat = np.concatenate([np.asarray(s, np.int64) for s in shards])
    assert sorted(flat.tolist()) == list(range(len(sizes)))
    loads = np.array([sizes[s].sum() for s in shards])
    assert loads.max() - loads.min() <= sizes.max()
    assert shard_scenes(sizes, ws) == shards                      # deterministic
    own = owner_of(shards, len(sizes))
    for r, s in enumerate(shards):
        assert np.all(own[s] == r)


def test_requests_follow_their_scene():
    rng = np.random.default_rng(50)
    n_sc, n_req, ws = 40, 1000, 3
    sizes = rng.integers(100, 5000, n_sc)
    own = owner_of(shard_scenes(sizes, ws), n_sc)
    which = rng.integers(0, n_sc, n_req)
    parts = [shard_requests(which, own, r) for r in range(ws)]
    allr = np.concatenate(parts)
    assert sorted(allr.tolist()) == list(range(n_req))            # each request once
    for r, p in enumerate(parts):
        assert np.all(np.diff(p) > 0)                            # arrival order kept
        assert np.all(own[which[p]] == r)


def _scenes():
    return [S.cloth_on_sphere(n_side=6 + k, radius=0.03, slices=10, stacks=6, lift=0.004, seed=30 + k)
            for k in range(3)] + [S.particle_cloud(27 + 10 * k, seed=40 + k, sphere_radius=0.02) for k in range(3)]


def _step_all(orc, scenes, ids):
    out = {}
    for i in ids:
        sc = scenes[i]
        P = orc.make_params(sc.params, iters=3, capacity=0)
        x3 = sc.x[:, :3].astype(np.float64)
        xo, vo, info, _ = orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris,
                                   orc.rest_lengths(x3, sc.edges), P)
        out[i] = (xo, vo)
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from oracle import oracle as orc
    scenes = _scenes()
    shards = shard_scenes([sc.n_verts for sc in scenes], ws)
    mine = _step_all(orc, scenes, shards[rank])
    gathered = [None] * ws
    dist.all_gather_object(gathered, {k: (v[0].tolist(), v[1].tolist()) for k, v in mine.items()})
    if rank == 0:
        merged = {}
        for g in gathered:
            assert not set(g) & set(merged)                          # no scene stepped twice
            merged.update(g)
        out["merged"] = merged
        out["shards"] = shards
    dist.destroy_process_group()


def test_two_rank_partition_equals_single_rank(orc):
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    merged = out["merged"]
    scenes = _scenes()
    assert sorted(merged) == list(range(len(scenes)))
    assert all(len(s) > 0 for s in out["shards"])
    ref = _step_all(orc, scenes, range(len(scenes)))
    for i, (xo, vo) in ref.items():
        np.testing.assert_array_equal(np.asarray(merged[i][0]), xo)
        np.testing.assert_array_equal(np.asarray(merged[i][1]), vo)
