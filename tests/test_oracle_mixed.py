"""Pins of the oracle's mixed-scene readings X1-X5 (rods, soft volumes, cloth
and particles in one simulation; Sec. 5's coupled codimensional scene):

- the closest point of a segment against brute-force sampling;
- a point-edge plane against the geometry worked out by hand;
- the point-edge candidate set against an independent numpy definition
  (isolated points, free edges, binary32 padded boxes);
- the inside of a volume takes no part in collision;
- the volume constraint: a linearised projection, so the residual after one
  sweep is quadratic in the initial error, momentum is preserved and a rigid
  motion changes nothing;
- a link's compliance: zero restores the rest length in one sweep, a huge one
  leaves the vertices in place;
- particles resting on a static rod never enter its offset xi, and the mixed
  scene stays free of edge-triangle intersections.
"""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

G = 9.81


def extra_of(orc, sc, x3=None):
    x3 = sc.x[:, :3].astype(np.float64) if x3 is None else x3
    return orc.Extra(x3, sc.links, sc.link_compliance, sc.tets, sc.volume_compliance)


def test_closest_point_segment_brute_force(orc):
    rng = np.random.default_rng(1)
    ts = np.linspace(0.0, 1.0, 200001)
    for _ in range(40):
        p, a, b = rng.normal(size=(3, 3))
        t = orc.closest_point_segment(p, a, b)
        d = np.linalg.norm(a[None, :] + ts[:, None] * (b - a)[None, :] - p[None, :], axis=1)
        assert abs(t - ts[np.argmin(d)]) <= 1e-5
    z = np.zeros(3)
    assert orc.closest_point_segment(np.ones(3), z, z) == 0.0


def test_point_edge_plane_worked_example(orc):
    """Rod (-5, 0, 0)-(5, 0, 0) mm, both ends movable (w = 1000 and 3000), a
    particle (w = 2000) at (1, 2.5, 0.5) mm: the foot of the perpendicular is
    (1, 0, 0) mm at t = 0.6, so the segment point's inverse mass is
    0.4 * 1000 + 0.6 * 3000 = 2200, the separation (0, 2.5, 0.5) mm,
    dist = sqrt(6.5) mm and phi = dist - xi."""
    mm = 1e-3
    x = np.array([[-5 * mm, 0, 0, 1000.0], [5 * mm, 0, 0, 3000.0], [1 * mm, 2.5 * mm, 0.5 * mm, 2000.0]],
                 np.float32)
    edges = np.array([[0, 1]], np.int32)
    tris = np.zeros((0, 3), np.int32)
    params = S.default_params(2e-3, 1e-3)
    P = orc.make_params(params, capacity=0)
    x3 = x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, x, edges, tris, P)
    dist = np.linalg.norm(x3[2] - np.array([x3[2, 0], 0.0, 0.0]))
    np.testing.assert_allclose(dist, np.sqrt(6.5) * mm, rtol=1e-6)
    phi = dist - 1e-3
    n = (x3[2] - np.array([x3[2, 0], 0.0, 0.0])) / dist
    t = (x3[2, 0] - x3[0, 0]) / (x3[1, 0] - x3[0, 0])     # 0.6 up to the binary32 storage
    assert abs(t - 0.6) < 1e-6
    wp, we = 2000.0, (1 - t) * 1000.0 + t * 3000.0
    assert R["cand"][3] == 1 and R["acc"][3] == 1
    offs, planes, keys = R["offs"], R["planes"], R["key"]
    for v, nn, share in ((2, n, wp / (wp + we)), (0, -n, we / (wp + we)), (1, -n, we / (wp + we))):
        assert offs[v + 1] - offs[v] == 1
        k = offs[v]
        np.testing.assert_allclose(planes[k, :3], nn, atol=1e-12)
        np.testing.assert_allclose(planes[k, 3], share * phi, rtol=1e-9)
        assert int(keys[k]) >> 62 == 3
    # the two sides' shares add up to phi: the pair's gap is split once
    np.testing.assert_allclose(planes[offs[2], 3] + planes[offs[0], 3], phi, rtol=1e-12)


def numpy_ve_candidates(x4, edges, tris, pad, in_constraints):
    """Point-edge candidates written from their definition: isolated points
    (no edge, triangle, link or tetrahedron) against edges of no triangle,
    binary32 boxes enlarged by pad, one vertex movable."""
    x = np.asarray(x4, np.float32)
    n = len(x)
    used = np.zeros(n, bool)
    used[np.asarray(edges).ravel()] = True
    if len(tris):
        used[np.asarray(tris).ravel()] = True
    used[np.asarray(in_constraints, np.int64)] = True
    iso = np.nonzero(~used)[0]
    tri_edges = set()
    for t in np.asarray(tris):
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            tri_edges.add((min(a, b), max(a, b)))
    pad = np.float32(pad)
    out = []
    for p in iso:
        plo, phi = x[p, :3] - pad, x[p, :3] + pad
        for e, (a, b) in enumerate(np.asarray(edges)):
            if (a, b) in tri_edges:
                continue
            elo = np.minimum(x[a, :3], x[b, :3]) - pad
            ehi = np.maximum(x[a, :3], x[b, :3]) + pad
            if np.all(plo <= ehi) and np.all(elo <= phi) and (x[p, 3] > 0 or x[a, 3] > 0 or x[b, 3] > 0):
                out.append((p, e))
    return np.array(sorted(out), np.int32).reshape(-1, 2)


@pytest.mark.parametrize("patch", [False, True])
def test_point_edge_candidates_match_definition(orc, patch):
    sc = S.particles_on_rod(cloth_patch=patch)
    # a cloth-edge neighbour for one particle: cloth edges are not free
    ref = numpy_ve_candidates(sc.x, sc.edges, sc.tris, sc.params["pad"],
                              np.concatenate([sc.links.ravel(), sc.tets.ravel()]))
    ex = extra_of(orc, sc)
    for brute in (True, False):
        got = orc.candidates(sc.x, sc.edges, sc.tris, sc.params["pad"], brute=brute, extra=ex)
        np.testing.assert_array_equal(got["ve"], ref)
    assert len(ref) > 0


def test_no_point_edge_pairs_with_triangle_edges(orc):
    """Isolated points next to a cloth meet its faces (vertex-face), never its
    edges: the edges of triangles are not free."""
    sc = S.cloth_on_sphere(n_side=8, radius=0.03, slices=12, stacks=8, lift=0.006, seed=5)
    x = sc.x.copy()
    # drop two isolated points onto the cloth, 1.5 mm above two of its vertices
    extra_pts = x[[10, 20]].copy()
    extra_pts[:, 1] += 1.5e-3
    x4 = np.concatenate([x, extra_pts], 0)
    c = orc.candidates(x4, sc.edges, sc.tris, sc.params["pad"])
    assert len(c["ve"]) == 0
    assert np.isin(np.arange(len(x), len(x4)), c["vf"][:, 0]).all()


def test_volume_interior_takes_no_part_in_collision(orc):
    sc = S.codimensional(rod_seg=16, cube_n=3)
    in_tets = np.unique(sc.tets)
    on_surface = np.unique(np.concatenate([sc.edges.ravel(), sc.tris.ravel()]))
    interior = np.setdiff1d(in_tets, on_surface)
    assert len(interior) > 0
    ex = extra_of(orc, sc)
    c = orc.candidates(sc.x, sc.edges, sc.tris, sc.params["pad"], extra=ex)
    assert not np.isin(c["vf"][:, 0], interior).any()
    assert not np.isin(c["vv"].ravel(), interior).any() and not np.isin(c["ve"][:, 0], interior).any()
    P = orc.make_params(sc.params, capacity=0)
    R = orc.build_regions(sc.x[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, P, extra=ex)
    assert np.all(np.diff(R["offs"])[interior] == 0)


def one_tet_step(orc, x3, rest3, w=1.0, compliance=0.0):
    """One substep (one iteration, no gravity, at rest) of a lone tetrahedron
    whose only constraint is its volume."""
    x4 = np.zeros((4, 4), np.float32)
    x4[:, :3] = x3
    x4[:, 3] = w
    params = S.default_params(2e-3, 1e-3, iters=1)
    params["gravity"] = (0.0, 0.0, 0.0)
    P = orc.make_params(params, capacity=0)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    ex = orc.Extra(rest3, None, None, tets, compliance)
    x, v, info, _ = orc.step(x3.astype(np.float64), np.zeros((4, 3)), x4, np.zeros((0, 2), np.int32),
                             np.zeros((0, 3), np.int32), np.zeros(0), P, extra=ex)
    return x, ex.vol6_rest[0]


def test_volume_constraint_is_a_linearised_projection(orc):
    rest = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.02, 0.09, 0.0], [0.03, 0.02, 0.08]])
    ratios = []
    for eps in (1e-2, 1e-3, 1e-4):
        x0 = rest.copy()
        x0[3, 2] -= eps * 0.08                       # flatten the apex by eps of the height
        x, v6 = one_tet_step(orc, x0, rest)
        c0 = orc.tet_volumes6(x0, [[0, 1, 2, 3]])[0] - v6
        c1 = orc.tet_volumes6(x, [[0, 1, 2, 3]])[0] - v6
        assert abs(c1) < abs(c0)
        ratios.append(abs(c1) / c0 ** 2 * abs(v6))
        # equal masses: the correction moves no mass centre (the gradients sum to 0)
        np.testing.assert_allclose((x - x0).sum(axis=0), 0.0, atol=1e-15)
    # Newton-like: the residual is second order in the initial error
    assert max(ratios) < 10.0 and min(ratios) > 0.01
    # a rigid rotation of the rest shape is no error: nothing moves
    th = 0.3
    Rz = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    xr = rest @ Rz.T + np.array([0.01, -0.02, 0.005])
    x, _ = one_tet_step(orc, xr, rest)
    np.testing.assert_allclose(x, xr, atol=1e-15)


def test_volume_compliance_halves_the_first_order_correction(orc):
    """XPBD with compliance alpha (X2): one sweep from lambda = 0 scales the
    first-order correction of a constraint by S / (S + alpha / dt^2), where
    S = sum_i w_i |grad_i C|^2.  With alpha = S dt^2 the residual is half the
    initial error, up to second order.  The gradients are taken by central
    differences of the signed volume, which is linear in each coordinate."""
    rest = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.02, 0.09, 0.0], [0.03, 0.02, 0.08]])
    x0 = rest.copy()
    x0[3, 2] -= 1e-4 * 0.08
    h = 1e-6
    S2 = 0.0
    for i in range(4):
        for a in range(3):
            xp, xm = x0.copy(), x0.copy()
            xp[i, a] += h
            xm[i, a] -= h
            g = (orc.tet_volumes6(xp, [[0, 1, 2, 3]])[0] - orc.tet_volumes6(xm, [[0, 1, 2, 3]])[0]) / (2 * h)
            S2 += 1.0 * g * g
    dt = S.default_params(2e-3, 1e-3)["dt"]
    x, v6 = one_tet_step(orc, x0, rest, compliance=S2 * dt * dt)
    c0 = orc.tet_volumes6(x0, [[0, 1, 2, 3]])[0] - v6
    c1 = orc.tet_volumes6(x, [[0, 1, 2, 3]])[0] - v6
    assert abs(c1 / c0 - 0.5) < 1e-3


def test_link_compliance_limits(orc):
    """Two vertices joined by one link, stretched 1 mm beyond its 10 mm rest
    length: compliance 0 restores the rest length in one sweep; a compliance
    far above w dt^2 leaves the vertices (almost) where they are."""
    rest = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0]])
    x0 = np.array([[0.0, 0.0, 0.0], [0.011, 0.0, 0.0]])
    x4 = np.zeros((2, 4), np.float32)
    x4[:, :3] = x0
    x4[:, 3] = 1000.0
    params = S.default_params(2e-3, 1e-3, iters=1)
    params["gravity"] = (0.0, 0.0, 0.0)
    P = orc.make_params(params, capacity=0)
    out = []
    for comp in (0.0, 1e9):
        ex = orc.Extra(rest, np.array([[0, 1]]), np.array([comp]))
        x, v, info, _ = orc.step(x0.copy(), np.zeros((2, 3)), x4, np.zeros((0, 2), np.int32),
                                 np.zeros((0, 3), np.int32), np.zeros(0), P, extra=ex)
        out.append(np.linalg.norm(x[1] - x[0]))
    np.testing.assert_allclose(out[0], 0.01, rtol=1e-12)
    np.testing.assert_allclose(out[1], 0.011, rtol=1e-6)


def test_particles_rest_on_a_static_rod(orc):
    """Particles straight above a static rod (no lateral offset: a point on a
    line is otherwise unstable and slides off) fall onto it, never come closer
    than xi, and come to rest within r of that offset."""
    sc = S.particles_on_rod(pinned_rod=False, n_particles=6, height=2.5e-3, speed=0.2)
    n_rod = len(sc.edges) + 1
    sc.x[n_rod:, 2] = 0.0
    ex = extra_of(orc, sc)
    P = orc.make_params(sc.params, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    a, b = x[0], x[n_rod - 1]
    gaps = []
    for _ in range(60):
        x, v, info, _ = orc.step(x, v, sc.x, sc.edges, sc.tris, rest, P, extra=ex)
        for p in range(n_rod, sc.n_verts):
            t = orc.closest_point_segment(x[p], a, b)
            gaps.append(np.linalg.norm(x[p] - (a + t * (b - a))))
    xi = sc.params["xi"]
    assert min(gaps) >= xi * (1 - 1e-6)
    # they came down onto the rod (within r of the offset) and stopped
    assert np.all(np.array(gaps[-(sc.n_verts - n_rod):]) < xi + sc.params["r"])
    assert np.abs(v[n_rod:, 1]).max() < 0.05


def test_mixed_scene_stays_intersection_free(orc):
    sc = S.codimensional(rod_seg=16, cube_n=3)
    ex = extra_of(orc, sc)
    P = orc.make_params(sc.params, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    for _ in range(4):
        x, v, info, _ = orc.step(x, v, sc.x, sc.edges, sc.tris, rest, P, extra=ex)
        assert orc.count_edge_triangle_intersections(x, sc.edges, sc.tris) == 0
