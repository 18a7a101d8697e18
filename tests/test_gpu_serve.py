"""Serving loop: results are the same alone and in the mix (bitwise), scenes
survive eviction to the host, requests of a scene run in order, and a step
that never finishes is reported as timed out (a host-side stall: no GPU
work is issued for it)."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402


def pool():
    return S.batch(n_scenes=6, seed=21, min_verts=100, max_verts=700, median_verts=300, sphere_slices=16,
                   sphere_stacks=10, plane_capacity=512)


def alone(sc, steps):
    x = torch.as_tensor(sc.x).cuda().contiguous()
    v = torch.as_tensor(sc.v).cuda().contiguous()
    ctx = ccfr.Context.from_scene(sc)
    for _ in range(steps):
        ctx.step(x, v)
    out = x.cpu().numpy(), v.cpu().numpy()
    ctx.close()
    return out


def serve(scenes, steps, budget, slots=3, timeout=30.0):
    sv = ccfr.Server(budget, n_slots=slots, timeout_s=timeout)
    ids = [sv.add_scene(sc) for sc in scenes]
    t = 0.0
    order = []
    for k in range(steps):
        for i in ids:
            order.append(i)
            sv.submit(i, t)
            t += 1e-4
    sv.start()
    n = sv.wait(120.0)
    return sv, ids, order, n


def test_mix_equals_alone_and_order():
    scenes = pool()
    steps = 3
    sv, ids, order, n = serve(scenes, steps, budget=40 << 30)
    assert n == len(order)
    res = sv.results(len(order))
    assert np.all(res["status"] == 0)
    assert np.all(res["t_arrival"] <= res["t_start"] + 1e-9) and np.all(res["t_start"] <= res["t_done"])
    for i in ids:
        own = np.nonzero(np.array(order) == i)[0]
        assert np.all(np.diff(res["t_start"][own]) > 0)            # one scene, arrival order
    for sc, i in zip(scenes, ids):
        xs, vs = sv.state(i)
        xa, va = alone(sc, steps)
        np.testing.assert_array_equal(xs, xa, err_msg=sc.name)
        np.testing.assert_array_equal(vs, va, err_msg=sc.name)
    sv.close()


def test_eviction_keeps_results():
    scenes = pool()
    steps = 2
    # a budget for about two of these scenes at a time
    budget = 2 * max(ccfr.estimate_bytes(sc) for sc in scenes)
    sv, ids, order, n = serve(scenes, steps, budget=budget, slots=2)
    info = sv.info()
    assert info["evictions"] > 0 and info["peak_resident_bytes"] <= info["budget_bytes"]
    res = sv.results(len(order))
    assert np.all(res["status"] == 0)
    for sc, i in zip(scenes, ids):
        xs, vs = sv.state(i)
        xa, va = alone(sc, steps)
        np.testing.assert_array_equal(xs, xa, err_msg=sc.name)
    sv.close()


def test_stalled_step_times_out():
    scenes = pool()[:3]
    sv = ccfr.Server(40 << 30, n_slots=2, timeout_s=0.5)
    ids = [sv.add_scene(sc) for sc in scenes]
    sv.stall(ids[1])
    for i in ids:
        sv.submit(i, 0.0)
    sv.start()
    n = sv.wait(30.0)
    assert n == 3
    res = sv.results(3)
    assert res["status"][1] == 5 and res["status"][0] == 0 and res["status"][2] == 0
    assert res["t_done"][1] - res["t_start"][1] >= 0.5
    sv.close()


def serve_batched(scenes, steps, budget, max_pool_verts, max_scene_verts, slots=3):
    sv = ccfr.Server(budget, n_slots=slots, timeout_s=30.0)
    ids = [sv.add_scene(sc) for sc in scenes]
    sv.set_batching(max_pool_verts, max_scene_verts)
    t = 0.0
    order = []
    for k in range(steps):
        for i in ids:
            order.append(i)
            sv.submit(i, t)
            t += 1e-4
    sv.start()
    n = sv.wait(120.0)
    return sv, ids, order, n


def test_batched_serving_equals_alone():
    """Continuous batching: the scenes are served by pooled batched launches
    (several requests per launch) and every scene ends bitwise where it ends
    stepped alone; requests of one scene still run in order."""
    scenes = pool()
    steps = 3
    sv, ids, order, n = serve_batched(scenes, steps, 40 << 30, max_pool_verts=1 << 20, max_scene_verts=1 << 20)
    assert n == len(order)
    res = sv.results(len(order))
    assert np.all(res["status"] == 0)
    info = sv.info()
    assert info["pools"] >= 1 and 0 < info["pool_launches"] < len(order)
    for i in ids:
        own = np.nonzero(np.array(order) == i)[0]
        assert np.all(np.diff(res["t_start"][own]) > 0)
    for sc, i in zip(scenes, ids):
        xs, vs = sv.state(i)
        xa, va = alone(sc, steps)
        np.testing.assert_array_equal(xs, xa, err_msg=sc.name)
        np.testing.assert_array_equal(vs, va, err_msg=sc.name)
    sv.close()


def test_batched_pools_and_single_scenes_with_eviction():
    """Small pools (a few scenes each) beside scenes served alone (the largest
    ones), with a budget that holds only part of them: pools are evicted and
    re-admitted as units and every result still equals the scene alone."""
    scenes = pool()
    steps = 2
    sizes = sorted(sc.n_verts for sc in scenes)
    est = [ccfr.estimate_bytes(sc) for sc in scenes]
    big = max(est)
    # pools of at most the largest scene's vertex count, the largest scene alone; a budget
    # for about two such units while the scenes need more
    budget = int(2.2 * big)
    assert budget < 0.9 * sum(est)
    sv, ids, order, n = serve_batched(scenes, steps, budget=budget, max_pool_verts=sizes[-1],
                                      max_scene_verts=sizes[-2], slots=2)
    info = sv.info()
    assert info["pools"] >= 2 and info["evictions"] > 0
    assert info["peak_resident_bytes"] <= info["budget_bytes"]
    res = sv.results(len(order))
    assert np.all(res["status"] == 0)
    for sc, i in zip(scenes, ids):
        xs, vs = sv.state(i)
        xa, va = alone(sc, steps)
        np.testing.assert_array_equal(xs, xa, err_msg=sc.name)
        np.testing.assert_array_equal(vs, va, err_msg=sc.name)
    sv.close()
