"""Seeded input generators: determinism and the stated recipes (CPU)."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S


def test_generators_are_deterministic():
    a = S.cloth_stack(n_side=16, layers=3, seed=5)
    b = S.cloth_stack(n_side=16, layers=3, seed=5)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.v, b.v)
    c = S.cloth_stack(n_side=16, layers=3, seed=6)
    assert not np.array_equal(a.v, c.v)


def test_stack_velocity_recipes():
    iid = S.cloth_stack(n_side=32, layers=4, seed=2)
    sm = S.cloth_stack(n_side=32, layers=4, seed=2, velocity="smooth")
    np.testing.assert_array_equal(iid.x, sm.x)
    for sc in (iid, sm):
        assert np.abs(sc.v[:, :3]).max() <= 0.5 + 1e-6
    # the smooth field reaches the stated bound on every component
    assert np.allclose(np.abs(sm.v[:, :3]).max(axis=0), 0.5, atol=1e-6)
    # and is smooth: neighbouring grid vertices (4 mm apart) move almost alike,
    # unlike the iid draws
    n = 32
    grid = sm.v[: n * n, :3].reshape(n, n, 3)
    d_smooth = np.abs(np.diff(grid, axis=1)).max()
    grid_iid = iid.v[: n * n, :3].reshape(n, n, 3)
    d_iid = np.abs(np.diff(grid_iid, axis=1)).max()
    assert d_smooth < 0.1 and d_iid > 0.5
    with pytest.raises(ValueError):
        S.cloth_stack(n_side=8, layers=2, velocity="other")


def test_card_stack_recipe():
    sc = S.card_stack(xi=1e-3)
    movable = sc.x[:, 3] > 0
    assert movable.sum() == 52 * 4
    y = np.sort(sc.x[movable, 1].reshape(-1, 4).mean(axis=1))
    np.testing.assert_allclose(np.diff(y), 1.5e-3, rtol=1e-5)


def test_workload_recipes_have_their_stated_sizes():
    """The three single-scene workloads at full size: vertex, edge and
    triangle counts and the parameters their recipes state."""
    c1 = S.config(1)
    assert (c1.n_verts, len(c1.tris)) == (1024 + 2002, 1922 + 4000)
    assert (c1.params["r"], c1.params["xi"], c1.params["iters"]) == (5e-3, 1e-3, 10)
    assert int((c1.x[:, 3] > 0).sum()) == 1024                 # the sphere is static
    c2 = S.config(2)
    assert (c2.n_verts, len(c2.edges), len(c2.tris)) == (262144, 782340, 520200)
    assert (c2.params["r"], c2.params["xi"], c2.params["iters"], c2.params["plane_capacity"]) == \
        (2e-3, 1e-3, 20, 1024)
    assert np.abs(c2.v[:, :3]).max() <= 0.5
    c3 = S.config(3)
    strands = int((c3.x[:, 3] > 0).sum())
    assert strands == 128 * 128 * 65 and len(c3.tris) == 0
    assert (c3.params["r"], c3.params["xi"], c3.params["iters"]) == (1e-3, 5e-4, 10)


def test_batch_recipe():
    """512 independent scenes of uneven sizes: movable vertices within the
    clipped range (a cloth's side is rounded), about a fifth particle clouds,
    each over a static sphere."""
    scenes = S.batch()
    assert len(scenes) == 512
    movable = np.array([int((s.x[:, 3] > 0).sum()) for s in scenes])
    assert movable.min() >= 1024 - 2 * 32 and movable.max() <= 65536 + 2 * 256 + 1
    n_particles = sum("particle_cloud" in s.name for s in scenes)
    assert 0.12 < n_particles / 512 < 0.28
    assert all((s.x[:, 3] == 0).any() for s in scenes)
    assert movable.sum() == 5340148                 # the seeded recipe: about 5.3 M movable vertices
