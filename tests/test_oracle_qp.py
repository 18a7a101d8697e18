"""The exact closest point of a region (oracle/qp.py) and the report-only
comparison of Alg. 2's result with it.

Pins of the closest-point solver: equality with the enumeration of every
active set of at most three planes on random small regions, the KKT
conditions, and the clamp closed form for mutually perpendicular planes.
Diagnostic (not gated): on test scenes with random candidate displacements,
how often Alg. 2's non-halted result is the closest point of the region
within the parity tolerance 1e-5 L and within ten retraction lengths eps,
and how much longer its displacement is;
printed as one REPORT line per scene.  Alg. 2's result is feasible, so its
distance from the candidate can never be below the closest point's: that
inequality is asserted.
"""
import json

import numpy as np
import pytest

from oracle import qp
from paper_2607_26901_b300 import scenes as S


def _random_region(rng, k):
    N = rng.normal(size=(k, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    d = rng.uniform(0.0, 3e-3, size=k)          # y = 0 (the build position) is inside
    y0 = rng.normal(scale=4e-3, size=3)
    return N, d, y0


@pytest.mark.parametrize("seed", range(40))
def test_qp_equals_active_set_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    N, d, y0 = _random_region(rng, 2 + seed % 6)
    y, act, u = qp.project(y0, N, d)
    ref = qp.brute_force(y0, N, d)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", range(20))
def test_qp_kkt(seed):
    rng = np.random.default_rng(2000 + seed)
    N, d, y0 = _random_region(rng, 3 + seed % 9)
    y, act, u = qp.project(y0, N, d)
    assert np.all(N @ y + d >= -1e-15)                       # primal feasible
    assert np.all(u >= -1e-15)                               # dual feasible
    np.testing.assert_allclose(N[act] @ y + d[act], 0.0, atol=1e-15)   # active planes tight
    np.testing.assert_allclose(y, y0 + N[act].T @ u, atol=1e-15)       # stationarity


def test_qp_perpendicular_planes_clamp():
    """Axis planes y_i >= -a_i: the closest point clamps each coordinate."""
    rng = np.random.default_rng(7)
    a = np.array([0.002, 0.0015, 0.001])
    for _ in range(20):
        y0 = rng.normal(scale=3e-3, size=3)
        y, _, _ = qp.project(y0, np.eye(3), a)
        np.testing.assert_allclose(y, np.maximum(y0, -a), atol=1e-18)


SCENES = {
    "cloth stack 3x10x10": lambda: S.cloth_stack(n_side=10, layers=3, spacing=4e-3, speed=0.0, jitter=3e-4, seed=5),
    "particles 216": lambda: S.particle_cloud(216, seed=13),
    "wires 3x3x16": lambda: S.wires(n_grid=3, n_seg=16, seed=14, grate=True),
}


@pytest.mark.parametrize("name", sorted(SCENES))
def test_alg2_against_closest_point_report(orc, name):
    sc = SCENES[name]()
    P = orc.make_params(sc.params, capacity=0)
    x3 = sc.x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)
    rng = np.random.default_rng(300)
    L = orc.scene_scale(sc.x)
    xp = x3 + rng.normal(scale=1.0e-3, size=x3.shape)
    out, halt, band, nviol = orc.project(x3, xp, sc.x[:, 3], R["offs"], R["planes"], R["key"], R["dlimit"], P)
    n_cmp = n_agree = n_agree_eps = 0
    ratios = []
    for v in np.nonzero((nviol > 0) & (halt == 0))[0]:
        o0, o1 = R["offs"][v], R["offs"][v + 1]
        pl = R["planes"][o0:o1]
        y0 = xp[v] - x3[v]
        y, _, _ = qp.project(y0, pl[:, :3], pl[:, 3])
        assert y is not None
        da = np.linalg.norm(out[v] - xp[v])
        dq = np.linalg.norm(y - y0)
        # Alg. 2's point is feasible (within tau), so it is no closer than the optimum
        assert da >= dq - np.sqrt(len(pl)) * P.tau_feas
        n_cmp += 1
        gap = np.abs(out[v] - x3[v] - y).max()
        n_agree += int(gap <= 1e-5 * L)
        n_agree_eps += int(gap <= 10 * P.eps)
        ratios.append(da / dq if dq > 0 else 1.0)
    assert n_cmp > 0
    line = {"scene": name, "violated_not_halted": n_cmp, "halted": int(halt.sum()),
            "agree_within_1e-5L": n_agree / n_cmp, "agree_within_10eps": n_agree_eps / n_cmp,
            "median_dist_ratio": float(np.median(ratios)), "max_dist_ratio": float(np.max(ratios))}
    print("REPORT", json.dumps(line))
