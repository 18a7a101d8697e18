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
