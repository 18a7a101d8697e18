"""Pins of the oracle's narrow phase (Alg. 3, Eq. 1-3), Plesnik projection
(Alg. 1) and projectOntoConvexRegion (Alg. 2) against closed forms, worked
examples and invariants."""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

GOLDEN = Path(__file__).resolve().parent / "golden"


def least_norm_projection(x0, N, b):
    """Orthogonal projection of x0 onto {x : N x = b} (independent rows):
    x0 + N^T (N N^T)^{-1} (b - N x0)."""
    N = np.atleast_2d(N)
    return x0 + N.T @ np.linalg.solve(N @ N.T, b - N @ x0)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("seed", range(10))
def test_alg1_equals_least_norm_projection(orc, k, seed):
    rng = np.random.default_rng(seed)
    x0 = rng.normal(size=3)
    N = rng.normal(size=(k, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    b = rng.normal(size=k)
    got = orc.ortho_sequence(x0, N, b, eps_dep=1e-12)
    np.testing.assert_allclose(got, least_norm_projection(x0, N, b), atol=1e-11)
    np.testing.assert_allclose(N @ got, b, atol=1e-11)


@pytest.mark.parametrize("seed", range(5))
def test_alg1_skips_dependent_and_duplicate_planes(orc, seed):
    rng = np.random.default_rng(50 + seed)
    x0 = rng.normal(size=3)
    N = rng.normal(size=(2, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    b = rng.normal(size=2)
    ref = least_norm_projection(x0, N, b)
    # a repeated plane is dependent: the result is unchanged
    got = orc.ortho_sequence(x0, np.vstack([N, N[:1]]), np.concatenate([b, b[:1]]), 1e-12)
    np.testing.assert_allclose(got, ref, atol=1e-10)
    # a consistent combination of the first two is dependent as well
    c = rng.normal(size=2)
    n3 = c @ N
    got = orc.ortho_sequence(x0, np.vstack([N, n3]), np.concatenate([b, [c @ b]]), 1e-12)
    np.testing.assert_allclose(got, ref, atol=1e-9)


def test_alg1_fourth_plane_in_3d_is_ignored(orc):
    rng = np.random.default_rng(3)
    x0 = rng.normal(size=3)
    N = rng.normal(size=(4, 3))
    b = rng.normal(size=4)
    got = orc.ortho_sequence(x0, N, b, 1e-12)
    np.testing.assert_allclose(got, np.linalg.solve(N[:3], b[:3]), atol=1e-10)


def _params(sc, **kw):
    from oracle import oracle
    return oracle.make_params(sc.params, **kw)


def test_worked_examples_golden(orc):
    """Hand-derived worked examples of Eq. 1-3 and Alg. 2 (tests/golden)."""
    cases = json.loads((GOLDEN / "worked_examples.json").read_text())["cases"]
    for c in cases:
        x4 = np.array(c["x4"], np.float32)
        tris = np.array(c["tris"], np.int32).reshape(-1, 3)
        edges = S.canonical_edges(np.array(c["edges"], np.int32).reshape(-1, 2))
        p = S.default_params(c["r"], c["xi"])
        P = orc.make_params(p, capacity=0)
        R = orc.build_regions(x4[:, :3].astype(np.float64), x4, edges, tris, P)
        v = c["vertex"]
        o0, o1 = R["offs"][v], R["offs"][v + 1]
        assert o1 - o0 == len(c["planes"])
        got = R["planes"][o0:o1]
        want = np.array(c["planes"], float)
        order_g = np.lexsort(got.T[::-1])
        order_w = np.lexsort(want.T[::-1])
        np.testing.assert_allclose(got[order_g], want[order_w], atol=1e-9)
        xp = x4[:, :3].astype(np.float64).copy()
        xp[v] = c["candidate"]
        out, halt, band, nviol = orc.project(x4[:, :3].astype(np.float64), xp, x4[:, 3], R["offs"],
                                             R["planes"], R["key"], R["dlimit"], P)
        np.testing.assert_allclose(out[v], c["projected"], atol=1e-12)
        assert halt[v] == c["halt"]


def _build(orc, sc, **kw):
    P = _params(sc, **kw)
    x3 = sc.x[:, :3].astype(np.float64)
    return P, x3, orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)


@pytest.mark.parametrize("make", [
    lambda: S.cloth_on_sphere(n_side=10, radius=0.04, slices=16, stacks=10, lift=0.004, seed=11),
    lambda: S.cloth_stack(n_side=8, layers=3, spacing=4e-3, speed=0.0, jitter=3e-4, seed=12),
    lambda: S.particle_cloud(125, seed=13),
    lambda: S.wires(n_grid=3, n_seg=12, seed=14, grate=True),
])
def test_regions_contain_current_configuration(orc, make):
    """With every gap >= xi, each plane has rho(x) = d >= 0 (x lies in its region);
    normals are unit; the two sides of a pair get opposite normals and shares
    summing to 1 (d_A + d_B = phi)."""
    sc = make()
    P, x3, R = _build(orc, sc, capacity=0)
    assert R["planes"].shape[0] > 0
    np.testing.assert_allclose(np.linalg.norm(R["planes"][:, :3], axis=1), 1.0, atol=1e-12)
    mind = orc.min_distances(x3, sc.x, sc.edges, sc.tris, 1.0)
    assert mind.min() >= sc.params["xi"]
    assert np.all(R["planes"][:, 3] >= 0)
    assert np.all(R["phi"] < 2 * sc.params["r"])
    # shares: per key, the planes of the two sides sum (in d/phi) to 1 per receiving side
    keys = R["key"]
    vert = np.repeat(np.arange(len(x3)), np.diff(R["offs"]))
    w = sc.x[:, 3].astype(np.float64)
    for k in np.unique(keys)[:400]:
        idx = np.nonzero(keys == k)[0]
        n = R["planes"][idx, :3]
        # two opposite normals at most
        ref = n[0]
        dots = n @ ref
        assert np.all(np.abs(np.abs(dots) - 1) < 1e-12)
        phi = R["phi"][idx[0]]
        if phi > 0:
            sides = {}
            for i, dd in zip(idx, dots):
                sides.setdefault(dd > 0, []).append(R["planes"][i, 3] / phi)
            # each side's share is the same for all its movable vertices
            tot = sum(v[0] for v in sides.values())
            if len(sides) == 2:
                assert abs(tot - 1.0) < 1e-9
            else:
                # only one side movable: the other side's inverse mass is 0
                assert abs(tot - 1.0) < 1e-9
        assert np.all(w[vert[idx]] > 0)


def test_large_triangle_caught_by_closest_point(orc):
    """A point under the middle of a triangle whose vertices are all far away
    still gets a plane (Sec. 4.2 large-triangle test)."""
    sc = S.large_triangle("point", size=0.1, height=4e-3)
    P, x3, R = _build(orc, sc, capacity=0)
    tri_far = np.linalg.norm(x3[1:4] - x3[0], axis=1).min()
    assert tri_far > 2 * sc.params["r"] + sc.params["xi"]
    assert R["offs"][1] - R["offs"][0] == 1
    n = R["planes"][0, :3]
    np.testing.assert_allclose(n, [0, -1, 0], atol=1e-7)
    assert abs(R["planes"][0, 3] - (4e-3 - sc.params["xi"])) < 1e-9
    sc2 = S.large_triangle("edge", size=0.1, height=4e-3)
    P, x3, R = _build(orc, sc2, capacity=0)
    # both edge endpoints get the edge-face plane (EE with the triangle's edges is far)
    assert R["offs"][2] - R["offs"][0] >= 2


@pytest.mark.parametrize("seed", range(8))
def test_alg2_result_is_feasible_or_halted(orc, seed):
    """Output satisfies every plane (rho >= -tau) or equals the build position."""
    rng = np.random.default_rng(200 + seed)
    sc = S.cloth_stack(n_side=8, layers=3, spacing=4e-3, speed=0.0, jitter=3e-4, seed=seed)
    P, x3, R = _build(orc, sc, capacity=0)
    xp = x3 + rng.normal(scale=1.5e-3, size=x3.shape)
    out, halt, band, nviol = orc.project(x3, xp, sc.x[:, 3], R["offs"], R["planes"], R["key"],
                                         R["dlimit"], P)
    assert nviol.sum() > 0
    for v in range(len(x3)):
        o0, o1 = R["offs"][v], R["offs"][v + 1]
        if halt[v]:
            np.testing.assert_array_equal(out[v], x3[v])
            continue
        pl = R["planes"][o0:o1]
        rho = (out[v] - x3[v]) @ pl[:, :3].T + pl[:, 3]
        assert np.all(rho >= -P.tau_feas)
        if nviol[v] == 0:
            np.testing.assert_array_equal(out[v], xp[v])


def test_alg2_single_plane_closed_form(orc):
    """One violated plane: projection onto it, then the eps retraction towards x."""
    sc = S.particle_over_floor(height=2.5e-3)   # phi = 1.5 mm < 2r = 2 mm
    P, x3, R = _build(orc, sc, capacity=0)
    assert R["offs"][1] == 1
    n, d = R["planes"][0, :3], R["planes"][0, 3]
    xp = x3.copy()
    xp[0] += np.array([4e-4, -5e-3, -2e-4])
    out, halt, _, nviol = orc.project(x3, xp, sc.x[:, 3], R["offs"], R["planes"], R["key"], R["dlimit"], P)
    y = xp[0] - x3[0]
    y_plane = y + (-d - n @ y) * n
    L = np.linalg.norm(y_plane)
    want = x3[0] + (L - P.eps) / L * y_plane
    np.testing.assert_allclose(out[0], want, atol=1e-15)
    assert nviol[0] == 1 and halt[0] == 0


def test_overflow_rule_is_safe(orc):
    """A vertex with more planes than the capacity moves at most max(0, min d)
    and still satisfies all its planes."""
    rng = np.random.default_rng(5)
    sc = S.cloth_stack(n_side=8, layers=3, spacing=4e-3, speed=0.0, jitter=3e-4, seed=4)
    P, x3, R = _build(orc, sc, capacity=4)
    over = np.nonzero(R["vflag"] & 1)[0]
    assert len(over) > 0
    xp = x3 + rng.normal(scale=2e-3, size=x3.shape)
    out, halt, band, nviol = orc.project(x3, xp, sc.x[:, 3], R["offs"], R["planes"], R["key"], R["dlimit"], P)
    for v in over:
        o0, o1 = R["offs"][v], R["offs"][v + 1]
        pl = R["planes"][o0:o1]
        assert np.linalg.norm(out[v] - x3[v]) <= max(0.0, pl[:, 3].min()) + 1e-15
        rho = (out[v] - x3[v]) @ pl[:, :3].T + pl[:, 3]
        assert np.all(rho >= -1e-15)
