"""ctypes front end of the FP64 CCFR oracle (``ccfr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module to compute what the CUDA library must
reproduce.  The library itself never imports it, and nothing here calls the
library.  ``build()`` compiles the C source with gcc into ``oracle/_build``.

Each wrapper names the part of the paper its C function follows; the C file's
header lists the readings (R1-R16) taken where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "ccfr_oracle.c"
_LIB = _HERE / "_build" / "libccfr_oracle.so"
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("r", C.c_double), ("xi", C.c_double), ("delta", C.c_double),
        ("pad", C.c_float),
        ("eps", C.c_double), ("eps_dep", C.c_double), ("tau_feas", C.c_double),
        ("band", C.c_double), ("dep_band", C.c_double), ("cond_band", C.c_double),
        ("n_max", C.c_int), ("iters", C.c_int), ("capacity", C.c_int), ("early_exit", C.c_int),
        ("dt", C.c_double), ("g", C.c_double * 3), ("compliance", C.c_double),
        ("k_resp", C.c_double), ("delta_v", C.c_double), ("mu_s", C.c_double), ("mu_k", C.c_double),
    ]


class OrcExtra(C.Structure):
    """Constraints beyond the collision edges (readings X1-X3 of the C file)."""
    _fields_ = [
        ("nl", C.c_int), ("links", C.c_void_p), ("link_compliance", C.c_void_p), ("link_rest", C.c_void_p),
        ("ntet", C.c_int), ("tets", C.c_void_p), ("vol6_rest", C.c_void_p), ("volume_compliance", C.c_double),
    ]


class OrcStepInfo(C.Structure):
    _fields_ = [
        ("iters_run", C.c_int),
        ("planes", C.c_long), ("violated", C.c_long), ("halts", C.c_long),
        ("overflow", C.c_long), ("shortened", C.c_long),
        ("any_band", C.c_int),
    ]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no fast-math, no FMA contraction; OpenMP
    over independent queries, pairs and vertices, which leaves every result
    bitwise the same for any thread count)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                           "-fPIC", "-shared", "-o", str(tmp), str(_SRC), "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        P = C.c_void_p
        _lib.orc_candidates.restype = C.c_long
        _lib.orc_candidates.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int, C.c_float, C.c_int, P, P]
        _lib.orc_candidates_ext.restype = C.c_long
        _lib.orc_candidates_ext.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int, C.POINTER(OrcExtra), C.c_float,
                                            C.c_int, P, P]
        _lib.orc_build.restype = C.c_void_p
        _lib.orc_build.argtypes = [P, P, C.c_int, P, C.c_int, P, C.c_int, C.POINTER(OrcParams)]
        _lib.orc_build_ext.restype = C.c_void_p
        _lib.orc_build_ext.argtypes = [P, P, C.c_int, P, C.c_int, P, C.c_int, C.POINTER(OrcExtra),
                                       C.POINTER(OrcParams)]
        _lib.orc_region_counts.argtypes = [P, P, C.c_int, P, C.c_int, P, C.c_int, C.POINTER(OrcParams), P, P]
        _lib.orc_regions_total.restype = C.c_long
        _lib.orc_regions_total.argtypes = [P]
        _lib.orc_regions_export.argtypes = [P, P, P, P, P, P, P, P]
        _lib.orc_regions_free.argtypes = [P]
        _lib.orc_project.restype = C.c_long
        _lib.orc_project.argtypes = [P, P, P, C.c_int, P, P, P, P, C.POINTER(OrcParams), P, P, P]
        _lib.orc_ortho_sequence.argtypes = [P, P, P, C.c_int, C.c_double, P]
        _lib.orc_edge_colors.restype = C.c_int
        _lib.orc_edge_colors.argtypes = [P, C.c_int, C.c_int, P]
        _lib.orc_step.restype = C.c_int
        _lib.orc_step.argtypes = [P, P, P, C.c_int, P, C.c_int, P, C.c_int, P,
                                  C.POINTER(OrcParams), P, C.POINTER(OrcStepInfo)]
        _lib.orc_step_ext.restype = C.c_int
        _lib.orc_step_ext.argtypes = [P, P, P, C.c_int, P, C.c_int, P, C.c_int, P, C.POINTER(OrcExtra),
                                      C.POINTER(OrcParams), P, C.POINTER(OrcStepInfo)]
        _lib.orc_step_hist.restype = C.c_int
        _lib.orc_step_hist.argtypes = [P, P, P, C.c_int, P, C.c_int, P, C.c_int, P, C.POINTER(OrcExtra),
                                       C.POINTER(OrcParams), P, C.POINTER(OrcStepInfo), P]
        _lib.orc_set_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_tet_colors.restype = C.c_int
        _lib.orc_tet_colors.argtypes = [P, C.c_int, C.c_int, P]
        _lib.orc_tet_volumes6.argtypes = [P, P, C.c_int, P]
        _lib.orc_closest_point_segment.restype = C.c_double
        _lib.orc_closest_point_segment.argtypes = [P, P, P]
        _lib.orc_rest_lengths.argtypes = [P, P, C.c_int, P]
        _lib.orc_min_distances.argtypes = [P, P, C.c_int, P, C.c_int, P, C.c_int, C.c_double, P]
        _lib.orc_count_edge_triangle_intersections.restype = C.c_long
        _lib.orc_count_edge_triangle_intersections.argtypes = [P, C.c_int, P, C.c_int, P, C.c_int]
        _lib.orc_closest_point_triangle.argtypes = [P, P, P, P, P, P]
        _lib.orc_closest_segments.argtypes = [P, P, P, P, P, P]
        _lib.orc_response.argtypes = [P, P, P, P, P, P, C.c_long, C.c_double, C.POINTER(OrcParams),
                                      C.POINTER(C.c_int)]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def make_params(p: dict, *, band: float = 0.0, capacity: int | None = None,
                iters: int | None = None, early_exit: bool = False,
                eps_dep: float | None = None, dep_band: float = 10.0, cond_band: float = 0.0) -> OrcParams:
    g = p.get("gravity", (0.0, -9.81, 0.0))
    o = OrcParams()
    o.r, o.xi, o.delta = p["r"], p["xi"], p.get("delta", 0.0)
    o.pad = np.float32(p["pad"])
    o.eps, o.eps_dep, o.tau_feas = p["eps"], p["eps_dep"] if eps_dep is None else eps_dep, p["tau_feas"]
    o.band = band
    o.dep_band = dep_band
    o.cond_band = cond_band
    o.n_max = p["n_max"]
    o.iters = p["iters"] if iters is None else iters
    o.capacity = p.get("plane_capacity", 0) if capacity is None else capacity
    o.early_exit = int(early_exit)
    o.dt = p["dt"]
    o.g[0], o.g[1], o.g[2] = g
    o.compliance = p.get("compliance", 0.0)
    o.k_resp = p.get("k_resp", 0.0)
    o.delta_v = p.get("delta_v", 0.0)
    o.mu_s, o.mu_k = p.get("mu_s", 0.0), p.get("mu_k", 0.0)
    return o


class Extra:
    """Links, tetrahedra and their rest values for the mixed-scene readings
    X1-X5 (rest lengths and rest volumes from the rest positions in FP64).
    Holds the arrays the C structure points to."""

    def __init__(self, rest_x3, links=None, link_compliance=None, tets=None, volume_compliance=0.0):
        rest_x3 = _c(rest_x3, np.float64)
        self.links = _c(np.zeros((0, 2)) if links is None else links, np.int32).reshape(-1, 2)
        self.link_compliance = _c(np.zeros(len(self.links)) if link_compliance is None else link_compliance,
                                  np.float64)
        self.link_rest = rest_lengths(rest_x3, self.links) if len(self.links) else np.zeros(0)
        self.tets = _c(np.zeros((0, 4)) if tets is None else tets, np.int32).reshape(-1, 4)
        self.vol6_rest = tet_volumes6(rest_x3, self.tets) if len(self.tets) else np.zeros(0)
        self.s = OrcExtra()
        self.s.nl = len(self.links)
        self.s.links = _p(self.links)
        self.s.link_compliance = _p(self.link_compliance)
        self.s.link_rest = _p(self.link_rest)
        self.s.ntet = len(self.tets)
        self.s.tets = _p(self.tets)
        self.s.vol6_rest = _p(self.vol6_rest)
        self.s.volume_compliance = float(volume_compliance)

    def ref(self):
        return C.byref(self.s)


def _xref(extra):
    return None if extra is None else extra.ref()


def candidates(x4: np.ndarray, edges: np.ndarray, tris: np.ndarray, pad: float, brute: bool = False,
               extra: Extra | None = None):
    """Candidate sets C_VF, C_EE, C_VV and C_VE (X4) under the binary32
    padded-AABB predicate with the exclusions of Alg. 3, each sorted
    lexicographically."""
    L = lib()
    x4 = _c(x4, np.float32)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    counts = np.zeros(4, np.int64)
    args = (_p(x4), len(x4), _p(e), len(e), _p(t), len(t), _xref(extra), C.c_float(pad), int(brute))
    tot = L.orc_candidates_ext(*args, None, _p(counts))
    out = np.zeros((max(tot, 1), 2), np.int32)
    L.orc_candidates_ext(*args, _p(out), _p(counts))
    c0, c1, c2, c3 = (int(c) for c in counts)
    return {"vf": out[:c0], "ee": out[c0:c0 + c1], "vv": out[c0 + c1:c0 + c1 + c2],
            "ve": out[c0 + c1 + c2:c0 + c1 + c2 + c3]}


def build_regions(x3: np.ndarray, x4w: np.ndarray, edges, tris, params: OrcParams, extra: Extra | None = None):
    """Per-vertex constraint sets (Alg. 3 over all vertices, plus the
    vertex-edge pairs of X4), CSR by vertex, planes sorted by key within a
    vertex."""
    L = lib()
    x3 = _c(x3, np.float64)
    x4w = _c(x4w, np.float32)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    n = len(x3)
    h = L.orc_build_ext(_p(x3), _p(x4w), n, _p(e), len(e), _p(t), len(t), _xref(extra), C.byref(params))
    try:
        tot = L.orc_regions_total(h)
        offs = np.zeros(n + 1, np.int64)
        planes = np.zeros((max(tot, 1), 4), np.float64)
        phi = np.zeros(max(tot, 1), np.float64)
        key = np.zeros(max(tot, 1), np.uint64)
        dlimit = np.zeros(n, np.float64)
        vflag = np.zeros(n, np.uint8)
        ca = np.zeros(8, np.int64)
        L.orc_regions_export(h, _p(offs), _p(planes), _p(phi), _p(key), _p(dlimit), _p(vflag), _p(ca))
    finally:
        L.orc_regions_free(h)
    return {"offs": offs, "planes": planes[:tot], "phi": phi[:tot], "key": key[:tot],
            "dlimit": dlimit, "vflag": vflag, "cand": ca[:4], "acc": ca[4:]}


def region_counts(x3, x4w, edges, tris, params: OrcParams):
    """Planes per vertex (Alg. 3 over all pairs) and the per-vertex flags
    (bit 0 overflow, bit 1 a band pair, |phi - 2r| <= band), without
    exporting the planes."""
    L = lib()
    x3 = _c(x3, np.float64)
    x4w = _c(x4w, np.float32)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    n = len(x3)
    count = np.zeros(n, np.int64)
    vflag = np.zeros(n, np.uint8)
    L.orc_region_counts(_p(x3), _p(x4w), n, _p(e), len(e), _p(t), len(t), C.byref(params), _p(count), _p(vflag))
    return count, vflag


def project(x3, xp3, w, offs, planes4, keys, dlimit, params: OrcParams):
    """Alg. 2 (+ Alg. 1, retraction, halt, final check) for every vertex.
    Returns (x_star, halt, band, nviol)."""
    L = lib()
    x3 = _c(x3, np.float64)
    out = _c(xp3, np.float64).copy()
    w = _c(w, np.float64)
    offs = _c(offs, np.int64)
    planes4 = _c(planes4, np.float64).reshape(-1, 4)
    keys = _c(keys, np.uint64)
    dl = None if dlimit is None else _c(dlimit, np.float64)
    n = len(x3)
    halt = np.zeros(n, np.uint8)
    band = np.zeros(n, np.uint8)
    nviol = np.zeros(n, np.int32)
    if planes4.size == 0:
        planes4 = np.zeros((1, 4))
        keys = np.zeros(1, np.uint64)
    L.orc_project(_p(x3), _p(out), _p(w), n, _p(offs), _p(planes4), _p(keys), _p(dl),
                  C.byref(params), _p(halt), _p(band), _p(nviol))
    return out, halt, band, nviol


def ortho_sequence(x0, normals, b, eps_dep=1e-12):
    """Alg. 1 applied to planes n_i . x = b_i in order from x0 (no retraction)."""
    L = lib()
    x0 = _c(x0, np.float64)
    normals = _c(normals, np.float64).reshape(-1, 3)
    b = _c(b, np.float64)
    out = np.zeros(3)
    L.orc_ortho_sequence(_p(x0), _p(normals), _p(b), len(b), C.c_double(eps_dep), _p(out))
    return out


def response(y, x, xn, planes4, phi, keys, w, params: OrcParams):
    """Contact response (Sec. 3.3, readings F1-F7) of one vertex at iterate y
    with build position x and substep start xn.  Returns (y', band)."""
    L = lib()
    y = np.array(y, dtype=np.float64).copy()
    x = _c(x, np.float64)
    xn = _c(xn, np.float64)
    planes4 = _c(planes4, np.float64).reshape(-1, 4)
    phi = _c(phi, np.float64)
    keys = _c(keys, np.uint64)
    band = C.c_int(0)
    L.orc_response(_p(y), _p(x), _p(xn), _p(planes4), _p(phi), _p(keys), len(phi), C.c_double(w),
                   C.byref(params), C.byref(band))
    return y, band.value


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: all host cores); returns
    the number in use."""
    return int(lib().orc_set_threads(int(n)))


def edge_colors(edges, n):
    L = lib()
    e = _c(edges, np.int32)
    col = np.zeros(max(len(e), 1), np.int32)
    nc = L.orc_edge_colors(_p(e), len(e), n, _p(col))
    return col[: len(e)], nc


def tet_colors(tets, n):
    L = lib()
    t = _c(tets, np.int32).reshape(-1, 4)
    col = np.zeros(max(len(t), 1), np.int32)
    nc = L.orc_tet_colors(_p(t), len(t), n, _p(col))
    return col[: len(t)], nc


def tet_volumes6(x3, tets):
    """Six times the signed volume of each tetrahedron (X2)."""
    L = lib()
    x3 = _c(x3, np.float64)
    t = _c(tets, np.int32).reshape(-1, 4)
    out = np.zeros(max(len(t), 1))
    L.orc_tet_volumes6(_p(x3), _p(t), len(t), _p(out))
    return out[: len(t)]


def closest_point_segment(p, a, b):
    """Parameter t in [0, 1] of the point of segment ab closest to p."""
    L = lib()
    args = [_c(v, np.float64) for v in (p, a, b)]
    return float(L.orc_closest_point_segment(*[_p(v) for v in args]))


def rest_lengths(x3, edges):
    L = lib()
    x3 = _c(x3, np.float64)
    e = _c(edges, np.int32)
    out = np.zeros(max(len(e), 1))
    L.orc_rest_lengths(_p(x3), _p(e), len(e), _p(out))
    return out[: len(e)]


def step(x3, v3, x4w, edges, tris, rest, params: OrcParams, extra: Extra | None = None,
         halt_history: bool = False):
    """One substep of Alg. 4 (with the links and tetrahedra of X1-X3 when
    extra is given).  Returns (x, v, info, vband), plus with halt_history a
    (iterations, n) uint8 array of the vertices that halted in each
    iteration."""
    L = lib()
    x = _c(x3, np.float64).copy()
    v = _c(v3, np.float64).copy()
    x4w = _c(x4w, np.float32)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    rest = _c(rest, np.float64)
    vband = np.zeros(len(x), np.uint8)
    info = OrcStepInfo()
    hist = np.zeros((max(params.iters, 1), len(x)), np.uint8) if halt_history else None
    args = (_p(x), _p(v), _p(x4w), len(x), _p(e), len(e), _p(t), len(t), _p(rest), _xref(extra),
            C.byref(params), _p(vband), C.byref(info))
    rc = L.orc_step_hist(*args, _p(hist)) if halt_history else L.orc_step_ext(*args)
    if rc != 0:
        raise RuntimeError("oracle step failed (edge colouring needs more than 64 colours)")
    if halt_history:
        return x, v, info, vband, hist[: info.iters_run]
    return x, v, info, vband


def min_distances(x3, x4w, edges, tris, cutoff):
    """(min VF, min EE, min VV) distance over non-adjacent pairs, capped at cutoff."""
    L = lib()
    x3 = _c(x3, np.float64)
    x4w = _c(x4w, np.float32)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    out = np.zeros(3)
    L.orc_min_distances(_p(x3), _p(x4w), len(x3), _p(e), len(e), _p(t), len(t), C.c_double(cutoff), _p(out))
    return out


def count_edge_triangle_intersections(x3, edges, tris):
    L = lib()
    x3 = _c(x3, np.float64)
    e = _c(edges, np.int32)
    t = _c(tris, np.int32)
    return int(L.orc_count_edge_triangle_intersections(_p(x3), len(x3), _p(e), len(e), _p(t), len(t)))


def closest_point_triangle(p, a, b, c):
    L = lib()
    args = [_c(v, np.float64) for v in (p, a, b, c)]
    q = np.zeros(3)
    bary = np.zeros(3)
    L.orc_closest_point_triangle(*[_p(v) for v in args], _p(q), _p(bary))
    return q, bary


def closest_segments(p1, q1, p2, q2):
    L = lib()
    args = [_c(v, np.float64) for v in (p1, q1, p2, q2)]
    s = np.zeros(1)
    t = np.zeros(1)
    L.orc_closest_segments(*[_p(v) for v in args], _p(s), _p(t))
    return float(s[0]), float(t[0])


def scene_scale(x4: np.ndarray) -> float:
    """Diagonal L of the scene's bounding box (the parity tolerance scale)."""
    p = np.asarray(x4)[:, :3].astype(np.float64)
    return float(np.linalg.norm(p.max(0) - p.min(0)))
