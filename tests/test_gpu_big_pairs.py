"""The region build's two-kernel emission (Alg. 3's broad and narrow phase):
scan kernels write the candidate pairs of each kind (vertex-face, edge-edge,
and those of the primitives whose boxes span more than a grid cell) to a
pair buffer, narrow kernels compute the planes; a kind whose pairs overflow
the buffer is redone by the fused scan-and-narrow kernel.  Neither the cell
size nor the buffer capacity may change the candidate set or the regions.

Scene: a 3 x 16 x 16 cloth stack moved by 0.3 of its predicted step (edges
stretched to a few cells; about 47k vertex-face and 125k edge-edge candidate
pairs).  Cases: the defaults (no kind overflows; some edges oversized), a
capacity of one pair per primitive (the vertex-face and edge-edge buffers
overflow and the fused kernels redo those kinds), and cell factor 0.3 (nearly
every primitive oversized)."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S
from tests.helpers import gpu_regions_by_vertex, sort_pairs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402

TOL_REL = 1e-5
BAND_REL = 1e-7
K = 1024


def tangled_stack():
    sc = S.cloth_stack(n_side=16, layers=3, speed=0.5, seed=9, plane_capacity=K)
    sc.x[:, :3] += (0.3 * sc.params["dt"] * sc.v[:, :3]).astype(np.float32)
    return sc


@pytest.mark.parametrize("cell_factor, pair_capacity", [(0.0, 0), (0.0, 1), (0.3, 0)])
def test_emission_paths_parity(orc, cell_factor, pair_capacity):
    sc = tangled_stack()
    x = torch.as_tensor(sc.x).cuda().contiguous()
    ctx = ccfr.Context.from_scene(sc, flags=ccfr.FLAG_STORE_KEYS, plane_capacity=K, cell_factor=cell_factor,
                                  pair_capacity=pair_capacity)
    ctx.reset_stats()
    ctx.build_regions(x)
    torch.cuda.synchronize()
    st = ctx.stats()
    assert st["aux"][4] > 0                               # oversized edges
    if cell_factor > 0:
        assert st["aux"][3] > 0                           # and triangles, at the small cell factor
    if pair_capacity == 1:
        assert st["aux"][15] >= 2, st["aux"][15]          # vertex-face and edge-edge redone fused
    elif cell_factor == 0:
        assert st["aux"][15] == 0, st["aux"][15]

    # candidate sets (the pair-listing mode) stay bit-exact
    got = ctx.candidates(x)
    ref = orc.candidates(sc.x, sc.edges, sc.tris, sc.params["pad"])
    for k in ("vf", "ee"):
        np.testing.assert_array_equal(sort_pairs(got[k]), ref[k].reshape(-1, 2), err_msg=k)

    # plane counts per vertex exact, planes as keyed multisets within the bar
    L = orc.scene_scale(sc.x)
    reg = ctx.regions(keys=True)
    g = gpu_regions_by_vertex(reg)
    gcount = reg["count"].cpu().numpy()
    P = orc.make_params(sc.params, band=BAND_REL * L, capacity=K)
    R = orc.build_regions(sc.x[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, P)
    offs = R["offs"]
    band = (R["vflag"] & 2) != 0
    assert band.mean() < 0.05
    r2 = 2.0 * sc.params["r"]
    checked = 0
    for vtx in range(sc.n_verts):
        if band[vtx]:
            continue
        n_ref = offs[vtx + 1] - offs[vtx]
        assert gcount[vtx] == n_ref, (vtx, gcount[vtx], n_ref)
        if n_ref == 0:
            continue
        gp, gk = g[vtx]
        rp = R["planes"][offs[vtx]:offs[vtx + 1]]
        rk = R["key"][offs[vtx]:offs[vtx + 1]]
        og, orr = np.argsort(gk, kind="stable"), np.argsort(rk, kind="stable")
        np.testing.assert_array_equal(gk[og], rk[orr])
        e = np.abs(gp[og, :3] - rp[orr, :3]).max(axis=1) * r2 + np.abs(gp[og, 3] - rp[orr, 3])
        assert e.max() <= TOL_REL * L, (vtx, float(e.max()))
        checked += 1
    assert checked > sc.n_verts // 2
    ctx.close()
