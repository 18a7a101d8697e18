"""GPU edge cases through the C ABI: scenes with no candidate pair at all.

- Two isolated particles far apart: every candidate set is empty, no plane
  is stored, and the step equals the oracle's (free flight with the max-step
  clamp of every iteration).
- One free particle (a one-vertex scene): the step equals the closed form
  min(I r, |dt v + dt^2 g|) along the prediction, as the oracle gives it.
- A scene whose vertices are all static (inverse mass 0): no pair has a
  movable vertex, so there is no candidate; positions stay bitwise and the
  velocities are zero.
"""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S
from tests.helpers import dev_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402


def _oracle_step(orc, sc):
    P = orc.make_params(sc.params, capacity=0)
    x3 = sc.x[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x3, sc.edges)
    return orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, rest, P)


def _gpu_step(sc):
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=64)
    cand = ctx.candidates(x)
    ctx.step(x, v)
    st = ctx.stats()
    ctx.close()
    return cand, st, x.cpu().numpy(), v.cpu().numpy()


def test_no_candidates_step_equals_oracle(orc):
    sc = S.two_particles(dist=0.5, speed=1.0)
    cand, st, x, v = _gpu_step(sc)
    assert all(len(c) == 0 for c in cand.values())
    assert st["status"] == 0 and st["planes"] == 0
    xo, vo, info, _ = _oracle_step(orc, sc)
    assert info.planes == 0
    # |x| ~ 0.25 m in binary32: a few ulp of 3e-8 m
    np.testing.assert_allclose(x[:, :3], xo, rtol=0, atol=1e-6)
    np.testing.assert_allclose(v[:, :3], vo, rtol=0, atol=1e-6 / sc.params["dt"])


def test_one_vertex_scene_free_fall(orc):
    params = S.default_params(1e-3, 1e-3, iters=10)
    v0 = np.array([[0.5, 0.2, -0.1]])
    sc = S._assemble("one_particle", [np.zeros((1, 3))], [np.full(1, 1e3)], [None], [None], params, v=v0)
    cand, st, x, v = _gpu_step(sc)
    assert all(len(c) == 0 for c in cand.values()) and st["status"] == 0
    xo, vo, _, _ = _oracle_step(orc, sc)
    dt, r, g = params["dt"], params["r"], np.array(params["gravity"])
    pred = dt * sc.v[0, :3].astype(np.float64) + dt * dt * g      # the scene stores v in binary32
    want = pred * min(1.0, params["iters"] * r / np.linalg.norm(pred))
    np.testing.assert_allclose(xo[0], want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(x[0, :3], want, rtol=0, atol=1e-8)
    np.testing.assert_allclose(v[0, :3], want / dt, rtol=0, atol=1e-8 / dt)


def test_all_static_scene_stays_put():
    sc = S.particle_over_floor(height=0.004)
    sc.x[:, 3] = 0.0
    cand, st, x, v = _gpu_step(sc)
    assert all(len(c) == 0 for c in cand.values()) and st["status"] == 0
    np.testing.assert_array_equal(x, sc.x)
    np.testing.assert_array_equal(v[:, :3], 0.0)
