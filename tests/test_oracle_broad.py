"""Pins of the oracle's candidate sets (padded-AABB predicate of Sec. 4.1 with
the exclusions of Alg. 3): the C sweep equals the C brute force, and both
equal an independent numpy brute force written here from the definition."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S


def numpy_candidates(x4, edges, tris, pad):
    """Definition written out: binary32 boxes lo = fl32(min - pad), hi = fl32(max + pad);
    overlap on all three axes; VF: v not in t; EE: e < f, no shared vertex;
    VV: isolated p < q; some vertex of the pair movable."""
    p = x4[:, :3].astype(np.float32)
    w = x4[:, 3]
    pad = np.float32(pad)

    def boxes(ids):
        c = p[ids]                          # (n, k, 3)
        return (c.min(1) - pad).astype(np.float32), (c.max(1) + pad).astype(np.float32)

    def ov(alo, ahi, blo, bhi):
        return np.all((alo[:, None, :] <= bhi[None, :, :]) & (blo[None, :, :] <= ahi[:, None, :]), axis=2)

    out = {}
    n = len(p)
    vlo, vhi = boxes(np.arange(n)[:, None])
    if len(tris):
        tlo, thi = boxes(tris)
        m = ov(vlo, vhi, tlo, thi)
        m &= ~np.any(np.arange(n)[:, None, None] == tris[None, :, :], axis=2)
        mov = (w[:, None] > 0) | np.any(w[tris] > 0, axis=1)[None, :]
        m &= mov
        out["vf"] = np.argwhere(m)
    else:
        out["vf"] = np.zeros((0, 2), int)
    if len(edges):
        elo, ehi = boxes(edges)
        m = ov(elo, ehi, elo, ehi)
        ne = len(edges)
        m &= np.arange(ne)[:, None] < np.arange(ne)[None, :]
        sh = np.zeros((ne, ne), bool)
        for i in range(2):
            for j in range(2):
                sh |= edges[:, i][:, None] == edges[:, j][None, :]
        m &= ~sh
        mv = np.any(w[edges] > 0, axis=1)
        m &= mv[:, None] | mv[None, :]
        out["ee"] = np.argwhere(m)
    else:
        out["ee"] = np.zeros((0, 2), int)
    iso = S.isolated_points(x4, edges)
    if len(iso):
        m = ov(vlo[iso], vhi[iso], vlo[iso], vhi[iso])
        m &= iso[:, None] < iso[None, :]
        m &= (w[iso][:, None] > 0) | (w[iso][None, :] > 0)
        ij = np.argwhere(m)
        out["vv"] = np.stack([iso[ij[:, 0]], iso[ij[:, 1]]], 1) if len(ij) else np.zeros((0, 2), int)
    else:
        out["vv"] = np.zeros((0, 2), int)
    return out


def _scenes():
    yield S.triangle_soup(n_tris=70, seed=1, n_points=40)
    yield S.triangle_soup(n_tris=50, seed=2, box=0.02, n_points=0)
    yield S.cloth_on_sphere(n_side=8, radius=0.03, slices=12, stacks=8, lift=0.006, seed=5)
    yield S.cloth_stack(n_side=7, layers=3, spacing=4e-3, speed=0.0, jitter=3e-4, seed=7)
    yield S.particle_cloud(64, seed=3)
    yield S.card_stack(n_cards=6)


@pytest.mark.parametrize("k", range(6))
def test_candidates_match_definition(orc, k):
    sc = list(_scenes())[k]
    pad = sc.params["pad"]
    ref = numpy_candidates(sc.x, sc.edges, sc.tris, pad)
    brute = orc.candidates(sc.x, sc.edges, sc.tris, pad, brute=True)
    sweep = orc.candidates(sc.x, sc.edges, sc.tris, pad, brute=False)
    for kind in ("vf", "ee", "vv"):
        r = ref[kind][np.lexsort((ref[kind][:, 1], ref[kind][:, 0]))] if len(ref[kind]) else ref[kind]
        np.testing.assert_array_equal(brute[kind], r.reshape(-1, 2))
        np.testing.assert_array_equal(sweep[kind], r.reshape(-1, 2))
    assert sum(len(v) for v in ref.values()) > 0


def test_candidates_superset_of_close_pairs(orc):
    """Every non-adjacent pair closer than 2*pad is a candidate (box enlargement argument)."""
    sc = S.cloth_stack(n_side=6, layers=2, spacing=4e-3, speed=0.0, jitter=5e-4, seed=9)
    pad = sc.params["pad"]
    cand = orc.candidates(sc.x, sc.edges, sc.tris, pad)
    x = sc.x[:, :3].astype(np.float64)
    got = {tuple(p) for p in cand["ee"]}
    for e in range(len(sc.edges)):
        for f in range(e + 1, len(sc.edges)):
            A, B = sc.edges[e], sc.edges[f]
            if set(A) & set(B):
                continue
            s, t = orc.closest_segments(x[A[0]], x[A[1]], x[B[0]], x[B[1]])
            d = np.linalg.norm(x[A[0]] + s * (x[A[1]] - x[A[0]]) - x[B[0]] - t * (x[B[1]] - x[B[0]]))
            if d < 2 * pad * (1 - 1e-6):
                assert (e, f) in got
