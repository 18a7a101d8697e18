"""Shared helpers of the GPU parity tests: moving scenes to the device and
reshaping the oracle's CSR regions.  No method arithmetic lives here."""
from __future__ import annotations

import numpy as np


def dev_scene(scene):
    import torch
    x = torch.as_tensor(scene.x).cuda().contiguous()
    v = torch.as_tensor(scene.v).cuda().contiguous()
    return x, v


def oracle_params(orc, scene, **kw):
    return orc.make_params(scene.params, **kw)


def sort_pairs(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a).reshape(-1, 2)
    if len(a) == 0:
        return a
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def gpu_regions_by_vertex(reg: dict):
    """{vertex: (planes (k,4) float64, keys (k,) uint64)} of the GPU lists, for
    vertices that did not overflow."""
    planes = reg["planes"].cpu().numpy()
    count = reg["count"].cpu().numpy()
    keys = reg["keys"].cpu().numpy().view(np.uint64)
    K = planes.shape[1]
    out = {}
    for v in np.nonzero(count)[0]:
        c = int(count[v])
        if c > K:
            continue
        out[int(v)] = (planes[v, :c].astype(np.float64), keys[v, :c])
    return out


def csr_to_padded(offs, planes4, K):
    """Oracle CSR planes -> (N, K, 4) float32 plus counts (for ccfr_load_regions)."""
    n = len(offs) - 1
    out = np.zeros((n, K, 4), np.float32)
    cnt = np.zeros(n, np.int32)
    for v in range(n):
        o0, o1 = offs[v], offs[v + 1]
        c = min(o1 - o0, K)
        out[v, :c] = planes4[o0:o0 + c]
        cnt[v] = o1 - o0
    return out, cnt


def band_vertices_valid(orc, sc, P, x_build, y, band_mask, L, tol_rel=1e-5, step_bound=None, extra=None):
    """Validity of the GPU's result at vertices the oracle excludes from the
    position comparison (a decision inside a band, where either branch is a
    correct outcome of the method).  Each such movable vertex must either have
    halted (y equal to its build position, bitwise) or satisfy every plane of
    its oracle region, except planes of band pairs, within the final-check
    tolerance tau plus tol_rel L (the plane parity bar), and move at most
    step_bound when given (plus the binary32 rounding of the positions).
    extra: the links and tetrahedra of a mixed scene (oracle.Extra).
    Returns a list of (vertex, reason, amount) for the violations."""
    x_build = np.asarray(x_build, np.float64)
    R = orc.build_regions(x_build, sc.x, sc.edges, sc.tris, P, extra=extra)
    r2 = 2.0 * P.r
    u32 = 2.0 ** -24
    bad = []
    for v in np.nonzero(band_mask & (sc.x[:, 3] > 0))[0]:
        d = y[v] - x_build[v]
        if np.all(d == 0.0):
            continue
        if step_bound is not None:
            slack = 1e-6 * step_bound + 4 * u32 * (np.abs(x_build[v]).sum() + step_bound)
            if np.linalg.norm(d) > step_bound + slack:
                bad.append((int(v), "step", float(np.linalg.norm(d) - step_bound)))
                continue
        o0, o1 = R["offs"][v], R["offs"][v + 1]
        keep = np.abs(R["phi"][o0:o1] - r2) > P.band
        pl = R["planes"][o0:o1][keep]
        rho = pl[:, :3] @ d + pl[:, 3]
        if len(rho) and rho.min() < -(P.tau_feas + tol_rel * L):
            bad.append((int(v), "plane", float(rho.min())))
    return bad
