"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars: candidate sets bit-exact; plane counts per vertex exact and planes as
multisets keyed by the pair key, each plane's offset within the step ball
|n - n_ref| 2r + |d - d_ref| <= 1e-5 L (the contact normal of a pair at
distance dist carries a binary32 error ~ u * size / dist, so the bound is
stated where the projection uses the plane: within |x' - x| <= 2r); projected
and stepped positions within 1e-5 L per coordinate (L = scene bounding-box
diagonal), excluding only vertices whose decisions the oracle reports inside
a decision band (|rho| or |phi - 2r| within BAND_REL L where the decision
can change the result, dependence tests within a factor 10 of eps_dep,
near-tied sort keys of distinct planes); each excluded vertex must still be a
valid outcome (halted at its build position, or inside every plane of its
oracle region within tau + 1e-5 L, and within the step bound in a step)."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S
from tests.helpers import band_vertices_valid, csr_to_padded, dev_scene, gpu_regions_by_vertex, sort_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402

TOL_REL = 1e-5
BAND_REL = 1e-7


def small_scenes():
    return {
        "soup": S.triangle_soup(n_tris=300, seed=1, n_points=200, box=0.03),
        "cloth_sphere_small": S.cloth_on_sphere(n_side=12, radius=0.04, slices=20, stacks=12, lift=0.006, seed=5),
        "stack_small": S.cloth_stack(n_side=20, layers=3, speed=0.5, seed=7, plane_capacity=1024),
        "wires_small": S.wires(n_grid=4, n_seg=24, seed=3),
        "particles": S.particle_cloud(343, seed=4, sphere_radius=0.03),
        "cards": S.card_stack(n_cards=12),
    }


SCENES = list(small_scenes().keys()) + ["config1"]


def get_scene(name):
    if name == "config1":
        return S.config(1)
    return small_scenes()[name]


_CAP = {}


def capacity_for(sc, orc=None, margin=1.5):
    """Plane capacity covering the largest per-vertex count at the initial
    state (with a margin for the counts growing during a trajectory)."""
    key = (sc.name, sc.n_verts, len(sc.edges), len(sc.tris), margin)
    if key not in _CAP:
        from oracle import oracle as O
        R = O.build_regions(sc.x[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris,
                            O.make_params(sc.params, capacity=0))
        m = int(np.diff(R["offs"]).max()) if sc.n_verts else 0
        _CAP[key] = max(64, int(np.ceil(m * margin / 32.0)) * 32)
    return _CAP[key]


@pytest.mark.parametrize("name", SCENES)
def test_candidates_bit_exact(orc, name):
    sc = get_scene(name)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=capacity_for(sc))
    got = ctx.candidates(x)
    ref = orc.candidates(sc.x, sc.edges, sc.tris, sc.params["pad"])
    for k in ("vf", "ee", "vv"):
        np.testing.assert_array_equal(sort_pairs(got[k]), ref[k].reshape(-1, 2), err_msg=k)
    assert sum(len(ref[k]) for k in ref) > 0
    ctx.close()


@pytest.mark.parametrize("name", SCENES)
def test_regions_parity(orc, name):
    sc = get_scene(name)
    L = orc.scene_scale(sc.x)
    K = capacity_for(sc)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, flags=ccfr.FLAG_STORE_KEYS, plane_capacity=K)
    ctx.build_regions(x)
    reg = ctx.regions(keys=True)
    g = gpu_regions_by_vertex(reg)
    gcount = reg["count"].cpu().numpy()
    P = orc.make_params(sc.params, band=BAND_REL * L, capacity=K)
    x3 = sc.x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)
    offs = R["offs"]
    band = (R["vflag"] & 2) != 0
    checked = 0
    r2 = 2.0 * sc.params["r"]
    worst = 0.0
    for vtx in range(sc.n_verts):
        if band[vtx]:
            continue
        n_ref = offs[vtx + 1] - offs[vtx]
        assert gcount[vtx] == n_ref, (vtx, gcount[vtx], n_ref)
        if n_ref == 0:
            continue
        assert n_ref <= K
        gp, gk = g[vtx]
        rp = R["planes"][offs[vtx]:offs[vtx + 1]]
        rk = R["key"][offs[vtx]:offs[vtx + 1]]
        og, orr = np.argsort(gk, kind="stable"), np.argsort(rk, kind="stable")
        np.testing.assert_array_equal(gk[og], rk[orr])
        dn = np.abs(gp[og, :3] - rp[orr, :3]).max(axis=1)
        dd = np.abs(gp[og, 3] - rp[orr, 3])
        e = dn * r2 + dd
        i = int(np.argmax(e))
        worst = max(worst, float(e[i]))
        assert e[i] <= TOL_REL * L, (vtx, hex(int(rk[orr][i])), gp[og][i], rp[orr][i], e[i], TOL_REL * L)
        checked += 1
    assert checked > 0
    assert band.mean() < 0.05
    ctx.close()


def test_overflow_rule_parity(orc):
    """Vertices with more planes than the capacity: counts match, and the
    step of such a vertex is bounded by max(0, min d) on both sides."""
    sc = S.cloth_stack(n_side=12, layers=3, speed=0.5, seed=4)
    L = orc.scene_scale(sc.x)
    K = 64
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=K, iters=1)
    ctx.build_regions(x)
    reg = ctx.regions()
    P = orc.make_params(sc.params, band=BAND_REL * L, capacity=K, iters=1)
    x3 = sc.x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)
    ref_cnt = np.diff(R["offs"])
    band = (R["vflag"] & 2) != 0
    gcnt = reg["count"].cpu().numpy()
    np.testing.assert_array_equal(gcnt[~band], ref_cnt[~band])
    over = (ref_cnt > K) & ~band
    assert over.sum() > 0
    dmin = reg["dmin_drop"].cpu().numpy()
    gp = reg["planes"].cpu().numpy()
    for vtx in np.nonzero(over)[0]:
        g_all = min(float(gp[vtx, :, 3].min()), float(dmin[vtx]))
        assert abs(g_all - R["dlimit"][vtx]) <= TOL_REL * L
    xo, vo, info, vband = orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris,
                                   orc.rest_lengths(x3, sc.edges), P)
    ctx.step(x, v)
    got = x.cpu().numpy()[:, :3].astype(np.float64)
    ok = vband == 0
    assert np.abs(got - xo)[ok].max() <= TOL_REL * L
    assert ctx.stats()["overflow_verts"] > 0
    ctx.close()


def _candidate_positions(sc, seed, scale):
    rng = np.random.default_rng(seed)
    xp = sc.x.copy()
    mov = sc.x[:, 3] > 0
    xp[mov, :3] += rng.normal(scale=scale, size=(mov.sum(), 3)).astype(np.float32)
    return xp


@pytest.mark.parametrize("name", SCENES)
def test_project_parity_on_oracle_planes(orc, name):
    """Alg. 2 on identical (binary32) planes and inputs: GPU vs oracle."""
    sc = get_scene(name)
    L = orc.scene_scale(sc.x)
    K = capacity_for(sc, margin=1.0)
    P = orc.make_params(sc.params, band=BAND_REL * L, capacity=K)
    x3 = sc.x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)
    planes32, cnt = csr_to_padded(R["offs"], R["planes"], K)
    assert cnt.max() <= K
    flat = np.concatenate([planes32[v, :cnt[v]].astype(np.float64) for v in range(sc.n_verts)] + [np.zeros((0, 4))])
    xp = _candidate_positions(sc, 11, 0.6 * sc.params["r"])
    out, halt, band, nviol = orc.project(x3, xp[:, :3].astype(np.float64), sc.x[:, 3], R["offs"], flat, R["key"],
                                         None, P)
    x, _ = dev_scene(sc)
    xio = torch.as_tensor(xp).cuda().contiguous()
    ctx = ccfr.Context.from_scene(sc, plane_capacity=K)
    ctx.load_regions(torch.as_tensor(planes32).cuda(), torch.as_tensor(cnt).cuda())
    h = torch.zeros(sc.n_verts, dtype=torch.uint8, device="cuda")
    ctx.project(x, xio, h)
    got = xio.cpu().numpy()[:, :3].astype(np.float64)
    ok = band == 0
    viol = nviol > 0
    assert (viol & ok).sum() >= 0.5 * viol.sum() > 0, (int((viol & ok).sum()), int(viol.sum()))
    err = np.abs(got - out).max(axis=1)
    bad = np.nonzero(ok & (err > TOL_REL * L))[0]
    assert len(bad) == 0, [(int(b), float(err[b]), int(nviol[b]), int(halt[b]), int(cnt[b])) for b in bad[:5]]
    np.testing.assert_array_equal(h.cpu().numpy()[ok], halt[ok])
    # band-excluded vertices: a valid outcome (halted at x, or inside every plane)
    invalid = band_vertices_valid(orc, sc, P, x3, got, band != 0, L)
    assert not invalid, invalid[:10]
    ctx.close()


@pytest.mark.parametrize("name", SCENES)
def test_build_and_project_parity(orc, name):
    """ccfr_build_regions + ccfr_project against the oracle's build + project."""
    sc = get_scene(name)
    L = orc.scene_scale(sc.x)
    K = capacity_for(sc, margin=1.0)
    P = orc.make_params(sc.params, band=BAND_REL * L, capacity=K)
    x3 = sc.x[:, :3].astype(np.float64)
    R = orc.build_regions(x3, sc.x, sc.edges, sc.tris, P)
    xp = _candidate_positions(sc, 12, 0.6 * sc.params["r"])
    out, halt, band, nviol = orc.project(x3, xp[:, :3].astype(np.float64), sc.x[:, 3], R["offs"], R["planes"],
                                         R["key"], R["dlimit"], P)
    x, _ = dev_scene(sc)
    xio = torch.as_tensor(xp).cuda().contiguous()
    ctx = ccfr.Context.from_scene(sc, plane_capacity=K)
    ctx.build_regions(x)
    ctx.project(x, xio)
    got = xio.cpu().numpy()[:, :3].astype(np.float64)
    ok = (band == 0) & ((R["vflag"] & 2) == 0)
    err = np.abs(got - out).max(axis=1)
    bad = np.nonzero(ok & (err > TOL_REL * L))[0]
    assert len(bad) == 0, [(int(b), float(err[b]), int(nviol[b]), int(halt[b])) for b in bad[:5]]
    viol = nviol > 0
    assert (viol & ok).sum() >= 0.5 * viol.sum()
    invalid = band_vertices_valid(orc, sc, P, x3, got, ~ok, L)
    assert not invalid, invalid[:10]
    ctx.close()


def _oracle_step(orc, sc, iters, L):
    P = orc.make_params(sc.params, band=BAND_REL * L, iters=iters, capacity=capacity_for(sc))
    x3 = sc.x[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x3, sc.edges)
    return orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, rest, P)


@pytest.mark.parametrize("name", SCENES)
def test_single_iteration_step_parity(orc, name):
    sc = get_scene(name)
    L = orc.scene_scale(sc.x)
    xo, vo, info, vband = _oracle_step(orc, sc, 1, L)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=capacity_for(sc), iters=1)
    ctx.step(x, v)
    st = ctx.stats()
    assert st["status"] == 0 and st["iterations"] == 1
    got = x.cpu().numpy()[:, :3].astype(np.float64)
    ok = vband == 0
    err = np.abs(got - xo)[ok].max()
    assert err <= TOL_REL * L, (err, TOL_REL * L, int((~ok).sum()))
    gv = v.cpu().numpy()[:, :3].astype(np.float64)
    assert np.abs(gv - vo)[ok].max() <= TOL_REL * L / sc.params["dt"]
    P = orc.make_params(sc.params, band=BAND_REL * L, iters=1, capacity=capacity_for(sc))
    invalid = band_vertices_valid(orc, sc, P, sc.x[:, :3].astype(np.float64), got, ~ok, L,
                                  step_bound=sc.params["r"])
    assert not invalid, invalid[:10]
    ctx.close()


def test_full_step_parity_config1(orc):
    """Alg. 4 with 10 iterations on the 1k-vertex cloth over the sphere."""
    sc = S.config(1)
    L = orc.scene_scale(sc.x)
    xo, vo, info, vband = _oracle_step(orc, sc, sc.params["iters"], L)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=capacity_for(sc))
    ctx.step(x, v)
    got = x.cpu().numpy()[:, :3].astype(np.float64)
    err_all = np.abs(got - xo).max(axis=1)
    assert err_all[vband == 0].max() <= TOL_REL * L
    assert (vband != 0).sum() <= 0.01 * sc.n_verts
    ctx.close()


def test_step_is_deterministic():
    sc = S.cloth_stack(n_side=24, layers=3, speed=0.5, seed=3, plane_capacity=1024)
    outs = []
    for _ in range(2):
        x, v = dev_scene(sc)
        ctx = ccfr.Context.from_scene(sc)
        for _ in range(2):
            ctx.step(x, v)
        outs.append((x.cpu().numpy().copy(), v.cpu().numpy().copy()))
        ctx.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("make,steps", [
    (lambda: S.config(1), 20),
    (lambda: S.cloth_stack(n_side=24, layers=4, speed=0.5, seed=9, plane_capacity=1024), 6),
    (lambda: S.wires(n_grid=6, n_seg=32, seed=5), 10),
    (lambda: S.particle_cloud(512, seed=6, sphere_radius=0.03), 10),
])
def test_gpu_trajectory_penetration_free(orc, make, steps):
    """Zero intersections and every non-adjacent pair at least xi apart after
    every GPU step (checked by the oracle's brute-force distance tests)."""
    sc = make()
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=capacity_for(sc))
    xi = sc.params["xi"]
    tol = 1e-6 * orc.scene_scale(sc.x)
    for s in range(steps):
        ctx.step(x, v)
        xs = x.cpu().numpy()[:, :3].astype(np.float64)
        m = orc.min_distances(xs, sc.x, sc.edges, sc.tris, 4 * xi)
        assert m.min() >= xi - tol, (s, m)
        if len(sc.tris):
            assert orc.count_edge_triangle_intersections(xs, sc.edges, sc.tris) == 0
    st = ctx.stats()
    assert st["status"] == 0 and st["planes"] > 0
    ctx.close()


def test_step_host_matches_device():
    sc = S.cloth_on_sphere(n_side=16, radius=0.05, slices=20, stacks=12, seed=2)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc, plane_capacity=256)
    ctx.step(x, v)
    ctx2 = ccfr.Context.from_scene(sc, plane_capacity=256)
    xh, vh = sc.x.copy(), sc.v.copy()
    ctx2.step_host(xh, vh)
    np.testing.assert_array_equal(x.cpu().numpy(), xh)
    np.testing.assert_array_equal(v.cpu().numpy(), vh)
