"""Pins of the oracle's simulation step (Alg. 4): closed forms for free fall,
resting contact and head-on particles, the XPBD edge-constraint sweep, the
edge colouring, and the non-penetration invariants over short trajectories."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S


def run(orc, sc, steps, *, iters=None, early_exit=False, capacity=None, check=None):
    P = orc.make_params(sc.params, iters=iters, early_exit=early_exit, capacity=capacity)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    infos = []
    for s in range(steps):
        x, v, info, _ = orc.step(x, v, sc.x, sc.edges, sc.tris, rest, P)
        infos.append((info.iters_run, info.planes, info.violated, info.halts, info.overflow))
        if check is not None:
            check(x, s)
    return x, v, infos


def free_particle(v0, r=1e-3, iters=10):
    p = np.zeros((1, 3))
    params = S.default_params(r, 1e-3, iters=iters)
    return S._assemble("free", [p], [np.full(1, 1e3)], [None], [None], params, v=np.array([v0]))


@pytest.mark.parametrize("v0,iters", [((0.0, 0.0, 0.0), 10), ((0.5, 0.2, -0.1), 10),
                                      ((3.0, 0.0, 0.0), 10), ((0.0, 1.0, 0.0), 3)])
def test_free_fall_closed_form(orc, v0, iters):
    """No contacts: the step moves along the prediction by min(I r, |dt v + dt^2 g|)."""
    sc = free_particle(v0, iters=iters)
    dt, r = sc.params["dt"], sc.params["r"]
    g = np.array(sc.params["gravity"])
    pred = dt * np.array(v0) + dt * dt * g
    want = pred * min(1.0, iters * r / np.linalg.norm(pred))
    x, v, _ = run(orc, sc, 1)
    np.testing.assert_allclose(x[0], want, atol=1e-15)
    np.testing.assert_allclose(v[0], want / dt, atol=1e-12)


def test_early_exit_when_converged(orc):
    sc = free_particle((0.0, 0.0, 0.0), r=0.01)
    _, _, infos = run(orc, sc, 1, early_exit=True)
    assert infos[0][0] == 1
    sc = free_particle((3.0, 0.0, 0.0), r=1e-3)
    _, _, infos = run(orc, sc, 1, early_exit=True)
    assert infos[0][0] == sc.params["iters"]


def test_particle_rests_on_floor(orc):
    """A particle landing on a static plane never goes below xi and comes to
    rest at a gap in [xi, xi + 10 eps]."""
    sc = S.particle_over_floor(height=0.004, r=1e-3, xi=1e-3, iters=10)
    xi, eps = sc.params["xi"], sc.params["eps"]
    gaps = []
    x, v, infos = run(orc, sc, 60, check=lambda x, s: gaps.append(x[0, 1]))
    assert min(gaps) >= xi - 1e-12
    assert xi <= gaps[-1] <= xi + 10 * eps
    assert max(i[1] for i in infos) >= 1


def test_two_particles_head_on(orc):
    """Equal masses closing head-on: each moves at most (dist - xi)/2 towards
    the other and the pair ends at distance >= xi."""
    sc = S.two_particles(dist=0.006, speed=1.0, xi=2e-3, r=1e-3)
    x0 = sc.x[:, :3].astype(np.float64)
    dist0 = np.linalg.norm(x0[1] - x0[0])
    x, v, _ = run(orc, sc, 5)
    assert np.linalg.norm(x[1] - x[0]) >= sc.params["xi"] - 1e-12
    for i in range(2):
        moved_towards = abs(x[i, 0] - x0[i, 0])
        assert moved_towards <= 0.5 * (dist0 - sc.params["xi"]) + 1e-12
    # symmetric
    np.testing.assert_allclose(x[0, 0], -x[1, 0], atol=1e-15)


def test_edge_colours_valid_and_first_fit(orc):
    sc = S.cloth_on_sphere(n_side=12, radius=0.04, slices=16, stacks=10, seed=3)
    col, nc = orc.edge_colors(sc.edges, sc.n_verts)
    assert nc == col.max() + 1
    inc = {}
    for e, (a, b) in enumerate(sc.edges):
        inc.setdefault(a, []).append(e)
        inc.setdefault(b, []).append(e)
    for e, (a, b) in enumerate(sc.edges):
        nb = [f for f in inc[a] + inc[b] if f != e]
        assert all(col[f] != col[e] for f in nb)
        earlier = {col[f] for f in nb if f < e}
        assert all(c in earlier for c in range(col[e]))


def test_xpbd_sweep_satisfies_last_colour(orc):
    """One Gauss-Seidel sweep of alpha = 0 edge constraints: the constraints of
    the last colour hold exactly (nothing moves their vertices afterwards)."""
    rng = np.random.default_rng(0)
    sc = S.cloth_stack(n_side=6, layers=1, spacing=0.01, speed=0.0, seed=1)
    sc.params["gravity"] = (0.0, 0.0, 0.0)
    x = sc.x[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    v = rng.normal(scale=0.02, size=x.shape)     # moves stay well inside r
    P = orc.make_params(sc.params, iters=1)
    xn, vn, info, _ = orc.step(x, v, sc.x, sc.edges, sc.tris, rest, P)
    assert info.planes == 0
    col, nc = orc.edge_colors(sc.edges, sc.n_verts)
    last = col == nc - 1
    e = sc.edges[last]
    L = np.linalg.norm(xn[e[:, 0]] - xn[e[:, 1]], axis=1)
    np.testing.assert_allclose(L, rest[last], atol=1e-14)
    np.testing.assert_allclose(vn, (xn - x) / sc.params["dt"], atol=1e-12)


def _invariants(orc, sc, xi_tol=1e-9):
    def check(x, s):
        m = orc.min_distances(x, sc.x, sc.edges, sc.tris, 4 * sc.params["xi"])
        assert m.min() >= sc.params["xi"] - xi_tol, (s, m)
        assert orc.count_edge_triangle_intersections(x, sc.edges, sc.tris) == 0
    return check


@pytest.mark.parametrize("make,steps", [
    (lambda: S.cloth_on_sphere(n_side=10, radius=0.03, slices=16, stacks=10, lift=0.006, seed=21,
                               steps=12), 12),
    (lambda: S.cloth_stack(n_side=8, layers=3, spacing=4e-3, speed=0.5, seed=22, iters=10), 4),
    (lambda: S.wires(n_grid=3, n_seg=16, seed=23), 6),
    (lambda: S.particle_cloud(64, seed=24, sphere_radius=0.02), 8),
    (lambda: S.card_stack(n_cards=8, xi=1e-3), 5),
])
def test_trajectory_is_penetration_free(orc, make, steps):
    """After every step no non-adjacent pair is closer than xi and no edge
    crosses a triangle (Sec. 3.1 safety argument; Sec. 4.3 zero violations)."""
    sc = make()
    x, v, infos = run(orc, sc, steps, check=_invariants(orc, sc))
    assert sum(i[1] for i in infos) > 0          # contacts were active


def test_card_stack_stays_static(orc):
    """Aligned cards resting with degenerate (identical) planes stay put: the
    stack keeps its spacing under gravity (Sec. 4.2 degeneration test)."""
    sc = S.card_stack(n_cards=10, xi=1e-3, gap_factor=1.5)
    y0 = sc.x[:, 1].astype(np.float64)
    x, v, infos = run(orc, sc, 6, check=_invariants(orc, sc))
    assert np.all(x[:, 1] >= 0.0)
    cards = sc.x[:, 3] > 0
    # every card stays above the previous one by at least xi
    yc = x[cards, 1].reshape(-1, 4).mean(axis=1)
    assert np.all(np.diff(yc) >= sc.params["xi"] - 1e-9)
    assert np.all(yc <= y0[cards].reshape(-1, 4).mean(axis=1) + 1e-12)


def test_threads_do_not_change_results(orc):
    """The oracle's OpenMP loops run over independent queries, pairs,
    vertices and same-colour constraints, and every list is put in its one
    order (by vertex and key) before use: one thread and all threads give
    bitwise the same regions and the same step."""
    sc = S.cloth_stack(n_side=10, layers=3, speed=0.5, seed=8, iters=4)
    P = orc.make_params(sc.params, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    outs = []
    try:
        for threads in (1, 0):
            orc.set_threads(threads)
            R = orc.build_regions(x, sc.x, sc.edges, sc.tris, P)
            xs, vs, info, band = orc.step(x, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, rest, P)
            outs.append((R, xs, vs, (info.planes, info.violated, info.halts, info.iters_run), band))
    finally:
        orc.set_threads(0)
    (R1, x1, v1, i1, b1), (R2, x2, v2, i2, b2) = outs
    for k in ("offs", "planes", "phi", "key", "vflag"):
        np.testing.assert_array_equal(R1[k], R2[k])
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(b1, b2)
    assert i1 == i2 and i1[0] > 0 and i1[1] > 0


def test_relabelled_particles_give_the_same_step(orc):
    """Vertex ids only name things: relabelling the particles of a cloud (the
    static sphere keeps its ids) permutes the step's result bit for bit.  A
    point-point plane is the same for either order of the pair (the normal
    and the shares are antisymmetric and symmetric in exact arithmetic and in
    IEEE arithmetic alike), and the pair keys only break exact ties."""
    sc = S.particle_cloud(125, seed=17)
    n = 125
    rng = np.random.default_rng(17)
    sc.v[:n, :3] = rng.uniform(-0.5, 0.5, size=(n, 3)).astype(np.float32)
    perm = rng.permutation(n)                      # old particle i becomes particle perm[i]
    sc2 = sc.copy()
    sc2.x[perm] = sc.x[:n]
    sc2.v[perm] = sc.v[:n]
    outs = []
    for s in (sc, sc2):
        P = orc.make_params(s.params, capacity=0)
        x = s.x[:, :3].astype(np.float64)
        x1, v1, info, _ = orc.step(x, s.v[:, :3].astype(np.float64), s.x, s.edges, s.tris,
                                   orc.rest_lengths(x, s.edges), P)
        outs.append((x1, v1, info.planes, info.violated, info.halts))
    (xa, va, *ia), (xb, vb, *ib) = outs
    np.testing.assert_array_equal(xb[perm], xa[:n])
    np.testing.assert_array_equal(vb[perm], va[:n])
    np.testing.assert_array_equal(xb[n:], xa[n:])
    assert ia == ib and ia[1] > 0
