"""Contact response and friction (Sec. 3.3) on the GPU against the FP64
oracle: single-iteration and full-substep parity within 1e-5 L (decision
bands excluded), and the physics the oracle is pinned to (force-balance rest
gap, Coulomb deceleration) reproduced by the CUDA path."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402
from tests.helpers import dev_scene  # noqa: E402

TOL_REL = 1e-5
BAND_REL = 1e-7
G = 9.81


def scenes():
    # plane capacity above every count: overflowed vertices get no response
    cloth = S.with_response(S.cloth_on_sphere(n_side=16, radius=0.05, slices=24, stacks=14, lift=0.002, seed=1,
                                              plane_capacity=1024),
                            delta=2e-3, k_resp=200.0, mu_s=0.4, mu_k=0.3)
    # layers jittered by 0.2 mm: an exactly aligned stack ties many distinct contacts
    stack = S.with_response(S.cloth_stack(n_side=16, layers=3, speed=0.1, seed=4, jitter=2e-4, plane_capacity=1024),
                            delta=5e-4, k_resp=2.0, mu_s=0.2, mu_k=0.1)
    floor = S.particle_over_floor(height=0.0016, size=1.0, r=2e-3, xi=1e-3, delta=1e-3, k_resp=1e-3 * G / 4e-4,
                                  mu_s=0.3, mu_k=0.2, v0=(0.3, -0.05, 0.1))
    return {"cloth_on_sphere": cloth, "cloth_stack": stack, "particle_floor": floor}


def oracle_step(orc, sc, iters, capacity):
    L = orc.scene_scale(sc.x)
    P = orc.make_params(sc.params, band=BAND_REL * L, iters=iters, capacity=capacity)
    x3 = sc.x[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x3, sc.edges)
    return orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, rest, P), L


@pytest.mark.parametrize("name", ["cloth_on_sphere", "cloth_stack", "particle_floor"])
@pytest.mark.parametrize("iters", [1, None])
def test_response_step_parity(orc, name, iters):
    sc = scenes()[name]
    it = sc.params["iters"] if iters is None else iters
    K = sc.params["plane_capacity"]
    (xo, vo, info, vband), L = oracle_step(orc, sc, it, K)
    # the response must change the result (no vacuous comparison)
    (xo0, _, _, _), _ = oracle_step(orc, S.with_response(sc, delta=0.0, k_resp=0.0), it, K)
    assert np.abs(xo - xo0).max() > 3 * TOL_REL * L
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=K, iters=it)
    ctx.step(x, v)
    st = ctx.stats()
    ctx.close()
    assert st["status"] == 0 and st["overflow_verts"] == 0
    got = x.cpu().numpy()[:, :3].astype(np.float64)
    ok = vband == 0
    err = np.abs(got - xo).max(axis=1)
    assert ok.mean() > 0.5
    if it == 1:
        assert err[ok].max() <= TOL_REL * L, (name, err[ok].max() / L)
    else:
        # several iterations in one shot: a band decision in an early iteration moves its vertex
        # by up to r and spreads through the later sweeps, so this is a coarse check only; the
        # strict multi-iteration check replays every iteration of the response scenes from the
        # GPU's own state (test_gpu_iterations.py, friction off) within 1e-5 L outside the bands
        assert np.mean(err[ok] <= TOL_REL * L) >= 0.99, (name, np.sort(err[ok])[-5:] / L)


def test_rest_gap_force_balance_on_gpu():
    k = 1e-3 * G / 4e-4
    sc = S.particle_over_floor(height=0.004, r=2e-3, xi=1e-3, iters=10, delta=1e-3, k_resp=k)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=32)
    hs = []
    for _ in range(600):
        ctx.step(x, v)
        hs.append(float(x[0, 1]))
    ctx.close()
    assert min(hs) >= 1e-3 - 1e-7
    assert abs(hs[-1] - (1e-3 + 1e-3 - 4e-4)) <= 1e-6


def test_kinetic_friction_on_gpu():
    mu_k, vx, dt = 0.2, 0.5, 1.0 / 60.0
    k = 1e-3 * G / 4e-4
    sc = S.particle_over_floor(height=1.6e-3, size=1.0, r=2e-3, xi=1e-3, iters=10, delta=1e-3, k_resp=k,
                               mu_k=mu_k, v0=(vx, 0.0, 0.0))
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=32)
    vel = []
    for _ in range(12):
        ctx.step(x, v)
        vel.append(float(v[0, 0]))
    ctx.close()
    np.testing.assert_allclose(np.diff(vel), -mu_k * G * dt, rtol=1e-3)
