"""Batched step: several independent scenes in one context.

Each scene's result in the batch must be bitwise identical to its result in
a context of its own (pairs never cross scenes; the candidate predicate is
exact, the per-pair arithmetic does not depend on the grid, and the
projection is independent of the order in which planes arrive), and the
performance knobs (cell size, emission grid, capacity) must not change any
result."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402
from tests.helpers import sort_pairs  # noqa: E402


def small_batch():
    return S.batch(n_scenes=7, seed=11, min_verts=100, max_verts=900, median_verts=300, sphere_slices=16,
                   sphere_stacks=10, plane_capacity=512)


def merged(scenes):
    x = np.concatenate([sc.x for sc in scenes])
    v = np.concatenate([sc.v for sc in scenes])
    return torch.as_tensor(x).cuda().contiguous(), torch.as_tensor(v).cuda().contiguous()


def test_batch_equals_scenes_alone():
    scenes = small_batch()
    assert any("particle" in sc.name for sc in scenes) and any("cloth" in sc.name for sc in scenes)
    x, v = merged(scenes)
    ctx = ccfr.Context.from_scenes(scenes)
    for _ in range(3):
        ctx.step(x, v)
    xb, vb = x.cpu().numpy(), v.cpu().numpy()
    st = ctx.stats()
    assert st["status"] == 0 and st["planes"] > 0
    for k, sc in enumerate(scenes):
        xs = torch.as_tensor(sc.x).cuda().contiguous()
        vs = torch.as_tensor(sc.v).cuda().contiguous()
        c1 = ccfr.Context.from_scene(sc)
        for _ in range(3):
            c1.step(xs, vs)
        o0, o1 = ctx.offsets[k], ctx.offsets[k + 1]
        np.testing.assert_array_equal(xb[o0:o1], xs.cpu().numpy(), err_msg=sc.name)
        np.testing.assert_array_equal(vb[o0:o1], vs.cpu().numpy(), err_msg=sc.name)
        c1.close()
    ctx.close()


def test_batch_candidates_are_union_of_scenes():
    scenes = small_batch()
    x, v = merged(scenes)
    ctx = ccfr.Context.from_scenes(scenes)
    got = ctx.candidates(x)
    want = {"vf": [], "ee": [], "vv": []}
    eoff = toff = 0
    for k, sc in enumerate(scenes):
        c1 = ccfr.Context.from_scene(sc)
        cs = c1.candidates(torch.as_tensor(sc.x).cuda().contiguous())
        vo = int(ctx.offsets[k])
        want["vf"].append(cs["vf"] + np.array([vo, toff]))
        want["ee"].append(cs["ee"] + np.array([eoff, eoff]))
        want["vv"].append(cs["vv"] + vo)
        eoff += len(sc.edges)
        toff += len(sc.tris)
        c1.close()
    for kind in ("vf", "ee", "vv"):
        w = np.concatenate([a.reshape(-1, 2) for a in want[kind]])
        np.testing.assert_array_equal(sort_pairs(got[kind]), sort_pairs(w), err_msg=kind)
    ctx.close()


def test_tuning_does_not_change_results():
    scenes = small_batch()
    outs = []
    for tune in [None, dict(cell_factor=1.0, emit_blocks_per_sm=4), dict(cell_factor=3.0, emit_blocks_per_sm=16,
                                                                          plane_capacity=1024), "auto"]:
        x, v = merged(scenes)
        ctx = ccfr.Context.from_scenes(scenes)
        if tune == "auto":
            t, ms = ctx.autotune(x, v, steps=1)
            assert t["plane_capacity"] % 32 == 0 and t["plane_capacity"] >= 64 and ms > 0
        elif tune:
            ctx.set_tuning(**tune)
        for _ in range(2):
            ctx.step(x, v)
        outs.append(x.cpu().numpy())
        ctx.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_step_active_mask():
    """ccfr_step_active: scenes whose mask byte is 0 keep x and v bitwise; the
    others advance exactly as when stepped alone; a later full step moves the
    paused scenes from where they were."""
    scenes = small_batch()
    x, v = merged(scenes)
    ctx = ccfr.Context.from_scenes(scenes)
    mask = np.array([1, 0, 1, 1, 0, 1, 0][:len(scenes)], np.uint8)
    active = torch.as_tensor(mask).cuda()
    x0, v0 = x.cpu().numpy().copy(), v.cpu().numpy().copy()
    ctx.step_active(x, v, active)
    ctx.step_active(x, v, active)
    ctx.step(x, v)                              # every scene: paused ones take their first step
    xb, vb = x.cpu().numpy(), v.cpu().numpy()
    for k, sc in enumerate(scenes):
        xs = torch.as_tensor(sc.x).cuda().contiguous()
        vs = torch.as_tensor(sc.v).cuda().contiguous()
        c1 = ccfr.Context.from_scene(sc)
        for _ in range(3 if mask[k] else 1):
            c1.step(xs, vs)
        o0, o1 = ctx.offsets[k], ctx.offsets[k + 1]
        np.testing.assert_array_equal(xb[o0:o1], xs.cpu().numpy(), err_msg=sc.name)
        np.testing.assert_array_equal(vb[o0:o1], vs.cpu().numpy(), err_msg=sc.name)
        c1.close()
    # a mask of zeros leaves everything as it is
    x1, v1 = x.clone(), v.clone()
    ctx.step_active(x, v, torch.zeros(len(scenes), dtype=torch.uint8, device="cuda"))
    assert torch.equal(x, x1) and torch.equal(v, v1)
    ctx.close()
    assert not np.array_equal(x0, xb)
