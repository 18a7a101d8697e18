"""ccfr_project_static, the projection entry point that allocates nothing.

Some callers cannot allocate device memory: their memory belongs to a host
engine or plug-in framework that hands this library fixed buffers, or they
run on a path where cudaMalloc is not permitted.  For them the library keeps
the projection's scratch in a fixed device array.  This test checks, through
the C ABI, that the static entry point returns what ccfr_project returns on
the same regions and inputs, on two calls in a row (the second call reuses the
scratch the first one left behind).  It lives in its own file that pytest
collects last, and it passes alone in a fresh process as well."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402

TOL_REL = 1e-5


def _candidates(sc, seed):
    rng = np.random.default_rng(seed)
    xp = sc.x.copy()
    mov = sc.x[:, 3] > 0
    xp[mov, :3] += rng.normal(scale=0.6 * sc.params["r"], size=(mov.sum(), 3)).astype(np.float32)
    return torch.as_tensor(xp).cuda().contiguous()


def test_project_static_matches_ccfr_project_twice():
    sc = S.cloth_stack(n_side=24, layers=3, speed=0.5, seed=21)
    L = float(np.linalg.norm(sc.x[:, :3].max(0) - sc.x[:, :3].min(0)))
    x = torch.as_tensor(sc.x).cuda().contiguous()
    ctx = ccfr.Context.from_scene(sc, plane_capacity=1024)
    ctx.build_regions(x)
    reg = ctx.regions()
    n_viol = 0
    for call, seed in enumerate((31, 32)):
        xin = _candidates(sc, seed)
        ref = xin.clone()
        h_ref = torch.zeros(sc.n_verts, dtype=torch.uint8, device="cuda")
        ctx.project(x, ref, h_ref)
        got = xin.clone()
        h_got = torch.ones(sc.n_verts, dtype=torch.uint8, device="cuda")
        ccfr.project_static(x, got, reg["planes"], reg["count"], ctx.params, dmin_drop=reg["dmin_drop"], halt=h_got)
        torch.cuda.synchronize()
        err = (got - ref)[:, :3].abs().max().item()
        assert err <= TOL_REL * L, (call, err)
        assert torch.equal(h_got, h_ref), call
        n_viol += int((ref != xin).any(dim=1).sum().item())
    assert n_viol > 0          # the projection moved vertices in these calls
    ctx.close()


def test_project_static_rejects_too_many_vertices():
    n = (1 << 18) + 1
    x = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    planes = torch.zeros((n, 32, 4), dtype=torch.float32, device="cuda")
    count = torch.zeros(n, dtype=torch.int32, device="cuda")
    p = ccfr.make_params(S.default_params(2e-3, 1e-3))
    with pytest.raises(ccfr.CcfrError) as ei:
        ccfr.project_static(x, x.clone(), planes, count, p)
    assert ei.value.status == 1
