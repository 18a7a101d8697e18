"""Per-iteration parity at the benchmarked sizes: the 262,144-vertex cloth stack
(4 x 256 x 256, 20 iterations) and the 1,201,202-vertex wires (128 x 128
strands of 64 segments over a grate, 10 iterations), each in the launch
configuration bench.py times (one context, the scene's plane capacity, default
tuning).  After one substep into the tangled state, ccfr_step_record records the next substep's prediction x~
and the collision-free iterate x_c after every iteration; the FP64 oracle
replays the first and the last iteration from the GPU's own state before
each (compliance 0: the XPBD multipliers do not affect positions) and every
movable vertex is compared within 1e-5 L outside the oracle's decision bands
(at least a quarter of them must be compared); every band vertex must be a
valid outcome (halted, or inside every oracle plane within tau + 1e-5 L and
within the step bound r)."""
import json
import os

import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S
from tests.helpers import band_vertices_valid, dev_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_26901_b300 import ccfr  # noqa: E402

TOL_REL = 1e-5
BAND_REL = 1e-7
U32 = 2.0 ** -24


def cond_band(ymax, r, L):
    """Alg. 1 steps whose dependence measure is small enough that binary32
    rounding of the planes and the iterate, about u (|y| + 2r) times
    |dir| / |beta|, reaches half the tolerance (the band of the small-scene
    iteration test)."""
    return 2.0 * U32 * (ymax + 2.0 * r) / (TOL_REL * L)


@pytest.mark.parametrize("cfg", [2, 3])
def test_fullsize_iterations(orc, cfg):
    orc.set_threads(0)
    sc = S.config(cfg)
    assert sc.params["compliance"] == 0.0
    iters = sc.params["iters"]
    K = sc.params["plane_capacity"]
    L = orc.scene_scale(sc.x)
    x, v = dev_scene(sc)
    ctx = ccfr.Context.from_scene(sc)
    ctx.step(x, v)                                  # into the tangled state of the bench's substeps
    x_start = x.cpu().numpy()[:, :3].astype(np.float64)
    ctx.reset_stats()
    xt, its = ctx.step_record(x, v, iters)
    st = ctx.stats()
    assert st["status"] == 0 and st["iterations"] == iters and st["overflow_verts"] == 0
    ctx.close()

    xt = xt.cpu().numpy()[:, :3].astype(np.float64)
    its = its.cpu().numpy()[:, :, :3].astype(np.float64)
    mov = sc.x[:, 3] > 0
    dt = sc.params["dt"]
    g = np.asarray(sc.params["gravity"], np.float64)
    rest = orc.rest_lengths(sc.x[:, :3].astype(np.float64), sc.edges)
    for i in (0, iters - 1):
        xc = x_start if i == 0 else its[i - 1]
        vel = np.where(mov[:, None], (xt - xc - dt * dt * g) / dt, 0.0)
        cb = cond_band(float(np.abs(xt - xc)[mov].max()) * np.sqrt(3.0), sc.params["r"], L)
        P = orc.make_params(sc.params, band=BAND_REL * L, iters=1, capacity=K, cond_band=cb)
        xo, _, info, vband = orc.step(xc, vel, sc.x, sc.edges, sc.tris, rest, P)
        y = its[i]
        err = np.abs(y - xo).max(axis=1)
        ok = (vband == 0) & mov
        bad = np.nonzero(ok & (err > TOL_REL * L))[0]
        assert len(bad) == 0, (i, len(bad), [(int(b), float(err[b] / L)) for b in bad[:5]])
        invalid = band_vertices_valid(orc, sc, P, xc, y, (vband != 0) & mov, L, step_bound=sc.params["r"])
        assert not invalid, (i, len(invalid), invalid[:10])
        n_excl = int(((vband != 0) & mov).sum())
        frac = n_excl / max(int(mov.sum()), 1)
        # (a tangled full-size state has many vertices resting on contact planes, whose
        # decisions fall in the rho band: more are excluded than in the small scenes' first
        # substep, and each of them was checked above to be a valid outcome)
        assert frac <= 0.75, frac
        name = "cloth_stack 4x256x256" if cfg == 2 else "wires 128x128x64"
        line = {"case": f"{name}, iteration {i + 1} of the second substep", "verts": sc.n_verts,
                "compared": int(ok.sum()), "band_excluded": n_excl, "excluded_frac": frac,
                "max_err_rel": float(err[ok].max() / L) if ok.any() else 0.0,
                "median_err_rel": float(np.median(err[ok]) / L) if ok.any() else 0.0}
        print("ITERATIONS", json.dumps(line))
        path = os.environ.get("CCFR_PRECISION_REPORT")
        if path:
            with open(path, "a") as f:
                f.write(json.dumps(line) + "\n")
