"""Pins of the oracle's closest-point geometry (Alg. 3's closestPointOnFace and
closestPointOnEdge) against brute force: dense sampling of the primitives."""
import numpy as np
import pytest


def _sample_triangle(a, b, c, m=160):
    u, v = np.meshgrid(np.linspace(0, 1, m), np.linspace(0, 1, m), indexing="ij")
    u, v = u.ravel(), v.ravel()
    keep = u + v <= 1.0
    u, v = u[keep], v[keep]
    w = 1.0 - u - v
    return w[:, None] * a + u[:, None] * b + v[:, None] * c


@pytest.mark.parametrize("seed", range(12))
def test_closest_point_triangle_vs_sampling(orc, seed):
    rng = np.random.default_rng(seed)
    a, b, c = rng.normal(size=(3, 3))
    # points in every Voronoi region: around vertices, edges and the face
    for p in [a + rng.normal(size=3) * 0.5, (a + b) / 2 + rng.normal(size=3),
              (a + b + c) / 3 + rng.normal(size=3) * 0.3, c - 2 * (a + b - 2 * c), rng.normal(size=3) * 3]:
        q, bary = orc.closest_point_triangle(p, a, b, c)
        assert np.all(bary >= -1e-12) and abs(bary.sum() - 1) < 1e-12
        np.testing.assert_allclose(q, bary[0] * a + bary[1] * b + bary[2] * c, atol=1e-12)
        d = np.linalg.norm(p - q)
        S = _sample_triangle(a, b, c)
        ds = np.linalg.norm(S - p, axis=1)
        # analytic minimum can only be below the sampled minimum, by at most the sampling step
        h = max(np.linalg.norm(b - a), np.linalg.norm(c - a), np.linalg.norm(c - b)) / 159
        assert d <= ds.min() + 1e-12
        assert ds.min() - d <= h


def test_closest_point_triangle_regions(orc):
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    # interior: straight below
    q, bary = orc.closest_point_triangle(np.array([0.2, 0.3, 0.7]), a, b, c)
    np.testing.assert_allclose(q, [0.2, 0.3, 0.0], atol=1e-15)
    np.testing.assert_allclose(bary, [0.5, 0.2, 0.3], atol=1e-15)
    # vertex regions
    np.testing.assert_allclose(orc.closest_point_triangle(np.array([-1.0, -1, 0]), a, b, c)[0], a)
    np.testing.assert_allclose(orc.closest_point_triangle(np.array([2.0, -0.5, 1]), a, b, c)[0], b)
    np.testing.assert_allclose(orc.closest_point_triangle(np.array([-0.5, 2.0, -1]), a, b, c)[0], c)
    # edge regions
    np.testing.assert_allclose(orc.closest_point_triangle(np.array([0.5, -1.0, 0.3]), a, b, c)[0], [0.5, 0, 0])
    np.testing.assert_allclose(orc.closest_point_triangle(np.array([1.0, 1.0, 0.0]), a, b, c)[0], [0.5, 0.5, 0])


@pytest.mark.parametrize("seed", range(12))
def test_closest_segments_vs_sampling(orc, seed):
    rng = np.random.default_rng(100 + seed)
    p1, q1, p2, q2 = rng.normal(size=(4, 3))
    s, t = orc.closest_segments(p1, q1, p2, q2)
    assert 0 <= s <= 1 and 0 <= t <= 1
    d = np.linalg.norm(p1 + s * (q1 - p1) - p2 - t * (q2 - p2))
    m = 801
    S = np.linspace(0, 1, m)
    A = p1 + S[:, None] * (q1 - p1)
    B = p2 + S[:, None] * (q2 - p2)
    D = np.linalg.norm(A[:, None, :] - B[None, :, :], axis=2)
    h = (np.linalg.norm(q1 - p1) + np.linalg.norm(q2 - p2)) / (m - 1)
    assert d <= D.min() + 1e-12
    assert D.min() - d <= h


def test_closest_segments_parallel_and_crossing(orc):
    # parallel, overlapping: distance is the line distance
    s, t = orc.closest_segments(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]),
                                np.array([0.5, 0.2, 0]), np.array([1.5, 0.2, 0]))
    A = np.array([s, 0, 0])
    B = np.array([0.5 + t, 0.2, 0])
    assert abs(np.linalg.norm(A - B) - 0.2) < 1e-12
    # crossing skew segments: closest points are the crossing points
    s, t = orc.closest_segments(np.array([-1.0, 0, 0]), np.array([1.0, 0, 0]),
                                np.array([0.0, -1, 0.3]), np.array([0.0, 1, 0.3]))
    assert abs(s - 0.5) < 1e-12 and abs(t - 0.5) < 1e-12


def test_distance_helpers_and_intersections(orc):
    from paper_2607_26901_b300 import scenes as S
    # an edge through the middle of a triangle is one edge-triangle intersection
    x = np.array([[0.0, 0, 0], [1, 0, 0], [0, 0, 1], [0.2, -0.5, 0.2], [0.2, 0.5, 0.2]])
    tris = np.array([[0, 1, 2]])
    edges = np.array([[0, 1], [0, 2], [1, 2], [3, 4]])
    assert orc.count_edge_triangle_intersections(x, edges, tris) == 1
    x[3:, 0] = 2.0
    assert orc.count_edge_triangle_intersections(x, edges, tris) == 0
    # min distance of a point above a static triangle
    sc = S.large_triangle("point", height=3e-3)
    d = orc.min_distances(sc.x[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, 0.01)
    assert abs(d[0] - 3e-3) < 1e-9
