"""Python binding of libccfr.so (the C ABI declared in include/ccfr.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (contiguous, float32 for
positions/velocities/planes, int32 for topology); they are passed by
``data_ptr()`` together with the current CUDA stream.  There is no CPU
fallback: if the library is missing the import fails.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libccfr.so"

FLAG_STORE_KEYS = 1 << 0
FLAG_EARLY_EXIT = 1 << 1
FLAG_NO_GRAPH = 1 << 2

STATUS = {0: "ok", 1: "invalid argument", 2: "capacity exceeded", 3: "device allocation failed",
          4: "CUDA runtime error", 5: "timeout", 6: "non-finite input", 7: "call out of order"}


class CcfrError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class Params(C.Structure):
    _fields_ = [("r", C.c_float), ("xi", C.c_float), ("delta", C.c_float), ("pad", C.c_float),
                ("eps_retract", C.c_float), ("eps_dep", C.c_float), ("tau_feas", C.c_float),
                ("max_passes", C.c_int), ("solver_iters", C.c_int), ("plane_capacity", C.c_int),
                ("cell_size", C.c_float), ("cell_factor", C.c_float), ("dt", C.c_float), ("gravity", C.c_float * 3),
                ("compliance", C.c_float), ("flags", C.c_uint),
                ("response_stiffness", C.c_float), ("delta_v", C.c_float), ("mu_s", C.c_float), ("mu_k", C.c_float),
                ("pair_capacity", C.c_int)]


class Mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int), ("n_edges", C.c_int), ("n_tris", C.c_int),
                ("edges", C.c_void_p), ("tris", C.c_void_p), ("rest_x", C.c_void_p)]


class MeshExt(C.Structure):
    """ccfr_mesh_ext: collision topology plus links and tetrahedra."""
    _fields_ = [("mesh", Mesh), ("n_links", C.c_int), ("links", C.c_void_p), ("link_compliance", C.c_void_p),
                ("n_tets", C.c_int), ("tets", C.c_void_p), ("volume_compliance", C.c_float)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in
                ("cand_vf", "cand_ee", "cand_vv", "pairs_vf", "pairs_ee", "pairs_vv", "planes_vf", "planes_ee",
                 "planes_vv", "planes",
                 "overflow_verts", "violated_verts", "halts", "ee_fp64", "feas_fp64", "feas_halts",
                 "iterations", "steps")] + [("aux", C.c_ulonglong * 16), ("max_planes", C.c_uint),
                                            ("error_flags", C.c_uint), ("cand_ve", C.c_ulonglong),
                                            ("pairs_ve", C.c_ulonglong), ("planes_ve", C.c_ulonglong)]

    def as_dict(self) -> dict:
        d = {n: getattr(self, n) for n, _ in self._fields_}
        d["aux"] = [int(v) for v in self.aux]
        return {k: (v if k == "aux" else int(v)) for k, v in d.items()}


class Tuning(C.Structure):
    _fields_ = [("cell_factor", C.c_float), ("emit_blocks_per_sm", C.c_int), ("plane_capacity", C.c_int)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class ServerInfo(C.Structure):
    _fields_ = [(n, C.c_long) for n in ("scenes", "requests", "done", "failed", "admissions", "evictions")] + \
               [(n, C.c_size_t) for n in ("resident_bytes", "peak_resident_bytes", "budget_bytes")] + \
               [(n, C.c_long) for n in ("pools", "pool_launches")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def lib():
    """Load libccfr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"libccfr.so not built ({_LIB_PATH}); run python -m paper_2607_26901_b300.build_lib")
        L = C.CDLL(str(_LIB_PATH))
        P = C.c_void_p
        sig = {
            "ccfr_create": [C.POINTER(Mesh), C.POINTER(Params), P, C.POINTER(P)],
            "ccfr_create_ext": [C.POINTER(MeshExt), C.POINTER(Params), P, C.POINTER(P)],
            "ccfr_destroy": [P],
            "ccfr_build_regions": [P, P, P],
            "ccfr_project": [P, P, P, P, P],
            "ccfr_step": [P, P, P, P],
            "ccfr_step_host": [P, P, P, P],
            "ccfr_step_timed": [P, P, P, P, C.c_int, P],
            "ccfr_step_record": [P, P, P, P, P, P],
            "ccfr_step_active": [P, P, P, P, P],
            "ccfr_get_candidates": [P, P, P, C.c_long, P, C.c_long, P, C.c_long, P, P],
            "ccfr_copy_regions": [P, P, P, P, P, P],
            "ccfr_load_regions": [P, P, P, C.c_int, P],
            "ccfr_get_info": [P, P, P, P],
            "ccfr_get_stats": [P, C.POINTER(Stats)],
            "ccfr_reset_stats": [P, P],
            "ccfr_project_static": [P, P, P, P, P, C.c_int, C.c_int, C.POINTER(Params), P, P],
            "ccfr_create_batch": [C.POINTER(Mesh), C.POINTER(Params), C.c_int, P, C.POINTER(P)],
            "ccfr_set_tuning": [P, C.POINTER(Tuning)],
            "ccfr_get_tuning": [P, C.POINTER(Tuning)],
            "ccfr_autotune": [P, P, P, C.c_int, C.POINTER(Tuning), C.POINTER(C.c_double), P],
            "ccfr_server_create": [C.c_size_t, C.c_int, C.c_double, C.POINTER(P)],
            "ccfr_server_add_scene": [P, C.c_int, C.c_int, C.c_int, P, P, P, P, C.POINTER(Params), C.POINTER(C.c_int)],
            "ccfr_server_submit": [P, C.c_int, C.c_double, C.POINTER(C.c_long)],
            "ccfr_server_start": [P],
            "ccfr_server_set_batching": [P, C.c_int, C.c_int],
            "ccfr_server_preload": [P, C.c_double, C.POINTER(C.c_int)],
            "ccfr_server_wait": [P, C.c_double, C.POINTER(C.c_long)],
            "ccfr_server_results": [P, C.c_long, P, P, P, P],
            "ccfr_server_get_state": [P, C.c_int, P, P],
            "ccfr_server_get_info": [P, C.POINTER(ServerInfo)],
            "ccfr_server_set_stall": [P, C.c_int, C.c_int],
            "ccfr_server_stop": [P],
            "ccfr_server_destroy": [P],
            "ccfr_estimate_bytes": [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.ccfr_stage_name.argtypes = [C.c_int]
        L.ccfr_stage_name.restype = C.c_char_p
        L.ccfr_status_string.argtypes = [C.c_int]
        L.ccfr_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return ["ccfr_create", "ccfr_create_ext", "ccfr_destroy", "ccfr_build_regions", "ccfr_project", "ccfr_step",
            "ccfr_step_host", "ccfr_step_timed", "ccfr_step_record", "ccfr_step_active", "ccfr_stage_name", "ccfr_get_candidates", "ccfr_copy_regions", "ccfr_load_regions",
            "ccfr_get_info", "ccfr_get_stats", "ccfr_reset_stats", "ccfr_status_string",
            "ccfr_project_static", "ccfr_create_batch", "ccfr_set_tuning", "ccfr_get_tuning", "ccfr_autotune",
            "ccfr_server_create", "ccfr_server_add_scene", "ccfr_server_submit", "ccfr_server_start",
            "ccfr_server_set_batching",
            "ccfr_server_preload",
            "ccfr_server_wait", "ccfr_server_results", "ccfr_server_get_state", "ccfr_server_get_info",
            "ccfr_server_set_stall", "ccfr_server_stop", "ccfr_server_destroy", "ccfr_estimate_bytes"]


def _check(rc: int, what: str):
    if rc != 0:
        raise CcfrError(rc, what)


def make_params(p: dict, flags: int = 0, plane_capacity: int | None = None,
                iters: int | None = None, cell_size: float = 0.0, cell_factor: float = 0.0,
                pair_capacity: int = 0) -> Params:
    o = Params()
    o.r, o.xi, o.delta, o.pad = p["r"], p["xi"], p.get("delta", 0.0), p["pad"]
    o.eps_retract, o.eps_dep, o.tau_feas = p["eps"], p["eps_dep"], p["tau_feas"]
    o.max_passes = p["n_max"]
    o.solver_iters = p["iters"] if iters is None else iters
    o.plane_capacity = p.get("plane_capacity", 64) if plane_capacity is None else plane_capacity
    o.cell_size = cell_size
    o.cell_factor = cell_factor
    o.dt = p["dt"]
    g = p.get("gravity", (0.0, -9.81, 0.0))
    o.gravity[0], o.gravity[1], o.gravity[2] = g
    o.compliance = p.get("compliance", 0.0)
    o.flags = flags
    o.response_stiffness = p.get("k_resp", 0.0)
    o.delta_v = p.get("delta_v", 0.0)
    o.mu_s, o.mu_k = p.get("mu_s", 0.0), p.get("mu_k", 0.0)
    o.pair_capacity = pair_capacity
    return o


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def project_static(x, x_io, planes, count, params: Params, dmin_drop=None, halt=None, stream=None):
    """ccfr_project_static: the projection on caller-held regions, for callers
    that cannot allocate device memory (all scratch is a fixed device array
    inside the library; at most 262,144 vertices; overlapping calls race)."""
    n = int(count.shape[0])
    cap = int(planes.shape[1])
    _check(lib().ccfr_project_static(_ptr(x), _ptr(x_io), _ptr(planes), _ptr(count), _ptr(dmin_drop), n, cap,
                                     C.byref(params), _ptr(halt), _stream(stream)), "ccfr_project_static")


class Context:
    """One scene on the current CUDA device (wraps a ccfr_ctx)."""

    def __init__(self, edges, tris, n_verts: int, params: Params, rest_x=None, stream=None, links=None,
                 link_compliance=None, tets=None, volume_compliance: float = 0.0):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device())
        self.edges = torch.as_tensor(np.asarray(edges, np.int32).reshape(-1, 2)).to(dev).contiguous()
        self.tris = torch.as_tensor(np.asarray(tris, np.int32).reshape(-1, 3)).to(dev).contiguous()
        self.n_verts = int(n_verts)
        rest = None
        if rest_x is not None:
            rest = torch.as_tensor(np.asarray(rest_x, np.float32).reshape(-1, 4)).to(dev).contiguous()
        m = Mesh(self.n_verts, int(self.edges.shape[0]), int(self.tris.shape[0]),
                 self.edges.data_ptr() if self.edges.numel() else None,
                 self.tris.data_ptr() if self.tris.numel() else None,
                 rest.data_ptr() if rest is not None else None)
        self.params = params
        h = C.c_void_p()
        if links is None and tets is None:
            _check(lib().ccfr_create(C.byref(m), C.byref(params), _stream(stream), C.byref(h)), "ccfr_create")
        else:
            lk = torch.as_tensor(np.asarray(links if links is not None else np.zeros((0, 2)), np.int32)
                                 .reshape(-1, 2)).to(dev).contiguous()
            lc = torch.as_tensor(np.asarray(link_compliance if link_compliance is not None else np.zeros(len(lk)),
                                            np.float32).reshape(-1)).to(dev).contiguous()
            tt = torch.as_tensor(np.asarray(tets if tets is not None else np.zeros((0, 4)), np.int32)
                                 .reshape(-1, 4)).to(dev).contiguous()
            me = MeshExt(m, int(lk.shape[0]), lk.data_ptr() if lk.numel() else None,
                         lc.data_ptr() if lc.numel() else None, int(tt.shape[0]), tt.data_ptr() if tt.numel() else None,
                         float(volume_compliance))
            _check(lib().ccfr_create_ext(C.byref(me), C.byref(params), _stream(stream), C.byref(h)), "ccfr_create_ext")
        self.h = h
        nv, cap, ncol = C.c_int(), C.c_int(), C.c_int()
        _check(lib().ccfr_get_info(h, C.byref(nv), C.byref(cap), C.byref(ncol)), "ccfr_get_info")
        self.capacity = cap.value
        self.n_colors = ncol.value

    @classmethod
    def from_scene(cls, scene, flags: int = 0, plane_capacity: int | None = None, iters: int | None = None,
                   cell_size: float = 0.0, cell_factor: float = 0.0, pair_capacity: int = 0, stream=None):
        p = make_params(scene.params, flags, plane_capacity, iters, cell_size, cell_factor, pair_capacity)
        ext = {}
        if len(getattr(scene, "links", ())) or len(getattr(scene, "tets", ())):
            ext = dict(links=scene.links, link_compliance=scene.link_compliance, tets=scene.tets,
                       volume_compliance=scene.volume_compliance)
        return cls(scene.edges, scene.tris, scene.n_verts, p, rest_x=scene.x, stream=stream, **ext)

    @classmethod
    def from_scenes(cls, scenes, flags: int = 0, plane_capacity: int | None = None, stream=None):
        """One context for several independent scenes (ccfr_create_batch).
        Vertices are numbered scene after scene; see `offsets`."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device())
        n = len(scenes)
        meshes = (Mesh * n)()
        params = (Params * n)()
        keep = []
        for k, sc in enumerate(scenes):
            e = torch.as_tensor(np.asarray(sc.edges, np.int32).reshape(-1, 2)).to(dev).contiguous()
            t = torch.as_tensor(np.asarray(sc.tris, np.int32).reshape(-1, 3)).to(dev).contiguous()
            r = torch.as_tensor(np.asarray(sc.x, np.float32)).to(dev).contiguous()
            keep += [e, t, r]
            meshes[k] = Mesh(sc.n_verts, int(e.shape[0]), int(t.shape[0]), e.data_ptr() if e.numel() else None,
                             t.data_ptr() if t.numel() else None, r.data_ptr())
            params[k] = make_params(sc.params, flags, plane_capacity)
        h = C.c_void_p()
        _check(lib().ccfr_create_batch(meshes, params, n, _stream(stream), C.byref(h)), "ccfr_create_batch")
        self.h = h
        self.params = params[0]
        self.offsets = np.concatenate([[0], np.cumsum([sc.n_verts for sc in scenes])]).astype(np.int64)
        self.n_verts = int(self.offsets[-1])
        nv, cap, ncol = C.c_int(), C.c_int(), C.c_int()
        _check(lib().ccfr_get_info(h, C.byref(nv), C.byref(cap), C.byref(ncol)), "ccfr_get_info")
        self.capacity = cap.value
        self.n_colors = ncol.value
        return self

    def set_tuning(self, cell_factor: float = 0.0, emit_blocks_per_sm: int = 0, plane_capacity: int = 0):
        t = Tuning(cell_factor, emit_blocks_per_sm, plane_capacity)
        _check(lib().ccfr_set_tuning(self.h, C.byref(t)), "ccfr_set_tuning")
        self.capacity = self.tuning()["plane_capacity"]

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().ccfr_get_tuning(self.h, C.byref(t)), "ccfr_get_tuning")
        return t.as_dict()

    def autotune(self, x, v, steps: int = 1, plane_capacity: int = 0, stream=None) -> tuple[dict, float]:
        """Pick cell size and emission grid (and the capacity when plane_capacity is 0)."""
        t = Tuning(0.0, 0, plane_capacity)
        ms = C.c_double()
        _check(lib().ccfr_autotune(self.h, _ptr(x), _ptr(v), steps, C.byref(t), C.byref(ms), _stream(stream)),
               "ccfr_autotune")
        self.capacity = t.plane_capacity
        return t.as_dict(), ms.value

    def close(self):
        if getattr(self, "h", None):
            lib().ccfr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the three calls of the method -------------------------------------
    def build_regions(self, x, stream=None):
        _check(lib().ccfr_build_regions(self.h, _ptr(x), _stream(stream)), "ccfr_build_regions")

    def project(self, x, x_io, halt=None, stream=None):
        _check(lib().ccfr_project(self.h, _ptr(x), _ptr(x_io), _ptr(halt), _stream(stream)), "ccfr_project")

    def step(self, x, v, stream=None):
        _check(lib().ccfr_step(self.h, _ptr(x), _ptr(v), _stream(stream)), "ccfr_step")

    def step_active(self, x, v, active, stream=None):
        """ccfr_step_active: step only the scenes whose byte in `active`
        (uint8 CUDA tensor, one per scene) is nonzero (batched contexts)."""
        _check(lib().ccfr_step_active(self.h, _ptr(x), _ptr(v), _ptr(active), _stream(stream)), "ccfr_step_active")

    def step_timed(self, x, v, stream=None) -> dict:
        """One step launched kernel by kernel; returns {stage: ms}."""
        n = 17
        out = (C.c_double * n)()
        _check(lib().ccfr_step_timed(self.h, _ptr(x), _ptr(v), out, n, _stream(stream)), "ccfr_step_timed")
        return {lib().ccfr_stage_name(i).decode(): out[i] for i in range(n)}

    def step_record(self, x, v, iters: int, stream=None):
        """ccfr_step_record: one substep that also returns the prediction x~
        and the collision-free iterate after each of the `iters` solver
        iterations (device tensors, (N, 4) and (iters, N, 4))."""
        torch = self.torch
        xt = torch.empty_like(x)
        its = torch.empty((iters,) + tuple(x.shape), dtype=x.dtype, device=x.device)
        _check(lib().ccfr_step_record(self.h, _ptr(x), _ptr(v), _ptr(xt), _ptr(its), _stream(stream)),
               "ccfr_step_record")
        return xt, its

    def step_host(self, x_host: np.ndarray, v_host: np.ndarray, stream=None):
        assert x_host.dtype == np.float32 and x_host.flags.c_contiguous
        assert v_host.dtype == np.float32 and v_host.flags.c_contiguous
        _check(lib().ccfr_step_host(self.h, x_host.ctypes.data_as(C.c_void_p),
                                    v_host.ctypes.data_as(C.c_void_p), _stream(stream)), "ccfr_step_host")

    # --- observability --------------------------------------------------------
    def candidates(self, x, cap: int | None = None, stream=None) -> dict:
        torch = self.torch
        cap = cap or 1 << 16
        while True:
            bufs = [torch.empty((cap, 2), dtype=torch.int32, device=x.device) for _ in range(3)]
            counts = (C.c_long * 3)()
            rc = lib().ccfr_get_candidates(self.h, _ptr(x), _ptr(bufs[0]), cap, _ptr(bufs[1]), cap,
                                           _ptr(bufs[2]), cap, counts, _stream(stream))
            if rc == 2:
                cap = max(counts) + 16
                continue
            _check(rc, "ccfr_get_candidates")
            return {k: bufs[i][: counts[i]].cpu().numpy() for i, k in enumerate(("vf", "ee", "vv"))}

    def regions(self, keys: bool = False, stream=None) -> dict:
        torch = self.torch
        dev = torch.device("cuda", torch.cuda.current_device())
        planes = torch.empty((self.n_verts, self.capacity, 4), dtype=torch.float32, device=dev)
        count = torch.empty(self.n_verts, dtype=torch.int32, device=dev)
        dmin = torch.empty(self.n_verts, dtype=torch.float32, device=dev)
        kt = torch.empty((self.n_verts, self.capacity), dtype=torch.int64, device=dev) if keys else None
        _check(lib().ccfr_copy_regions(self.h, _ptr(planes), _ptr(kt), _ptr(count), _ptr(dmin), _stream(stream)),
               "ccfr_copy_regions")
        out = {"planes": planes, "count": count, "dmin_drop": dmin}
        if keys:
            out["keys"] = kt
        return out

    def load_regions(self, planes, count, stream=None):
        cap = int(planes.shape[1])
        _check(lib().ccfr_load_regions(self.h, _ptr(planes), _ptr(count), cap, _stream(stream)), "ccfr_load_regions")

    def stats(self) -> dict:
        s = Stats()
        rc = lib().ccfr_get_stats(self.h, C.byref(s))
        if rc not in (0, 6):
            _check(rc, "ccfr_get_stats")
        d = s.as_dict()
        d["status"] = rc
        return d

    def reset_stats(self, stream=None):
        _check(lib().ccfr_reset_stats(self.h, _stream(stream)), "ccfr_reset_stats")


def estimate_bytes(scene, plane_capacity: int | None = None) -> int:
    """Device bytes a resident scene takes (what the server charges)."""
    b = C.c_size_t()
    k = plane_capacity or scene.params.get("plane_capacity", 64)
    _check(lib().ccfr_estimate_bytes(scene.n_verts, len(scene.edges), len(scene.tris), k, C.byref(b)),
           "ccfr_estimate_bytes")
    return b.value


class Server:
    """Serving loop (ccfr_server_*): step requests for registered scenes,
    device-resident state, HBM-budget admission, n_slots concurrent steps."""

    def __init__(self, hbm_budget_bytes: int, n_slots: int = 8, timeout_s: float = 30.0):
        h = C.c_void_p()
        _check(lib().ccfr_server_create(int(hbm_budget_bytes), n_slots, timeout_s, C.byref(h)), "ccfr_server_create")
        self.h = h
        self.n_verts = []

    def add_scene(self, scene, flags: int = 0, plane_capacity: int | None = None) -> int:
        p = make_params(scene.params, flags, plane_capacity)
        e = np.ascontiguousarray(scene.edges, np.int32)
        t = np.ascontiguousarray(scene.tris, np.int32)
        x = np.ascontiguousarray(scene.x, np.float32)
        v = np.ascontiguousarray(scene.v, np.float32)
        sid = C.c_int()
        ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a.size else None  # noqa: E731
        _check(lib().ccfr_server_add_scene(self.h, scene.n_verts, len(e), len(t), ptr(e), ptr(t), ptr(x), ptr(v),
                                           C.byref(p), C.byref(sid)), "ccfr_server_add_scene")
        self.n_verts.append(scene.n_verts)
        return sid.value

    def submit(self, scene_id: int, t_arrival: float) -> int:
        rid = C.c_long()
        _check(lib().ccfr_server_submit(self.h, scene_id, t_arrival, C.byref(rid)), "ccfr_server_submit")
        return rid.value

    def set_batching(self, max_pool_verts: int, max_scene_verts: int):
        """Continuous batching: small scenes grouped into pools stepped by one
        batched launch each (ccfr_server_set_batching)."""
        _check(lib().ccfr_server_set_batching(self.h, int(max_pool_verts), int(max_scene_verts)),
               "ccfr_server_set_batching")

    def preload(self, fraction: float = 0.9) -> int:
        n = C.c_int()
        _check(lib().ccfr_server_preload(self.h, fraction, C.byref(n)), "ccfr_server_preload")
        return n.value

    def start(self):
        _check(lib().ccfr_server_start(self.h), "ccfr_server_start")

    def wait(self, timeout_s: float) -> int:
        n = C.c_long()
        rc = lib().ccfr_server_wait(self.h, timeout_s, C.byref(n))
        if rc not in (0, 5):
            _check(rc, "ccfr_server_wait")
        return n.value

    def results(self, n: int) -> dict:
        ta, ts, td = np.zeros(n), np.zeros(n), np.zeros(n)
        st = np.zeros(n, np.int32)
        f = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        _check(lib().ccfr_server_results(self.h, n, f(ta), f(ts), f(td), f(st)), "ccfr_server_results")
        return {"t_arrival": ta, "t_start": ts, "t_done": td, "status": st}

    def state(self, scene_id: int):
        n = self.n_verts[scene_id]
        x = np.zeros((n, 4), np.float32)
        v = np.zeros((n, 4), np.float32)
        _check(lib().ccfr_server_get_state(self.h, scene_id, x.ctypes.data_as(C.c_void_p),
                                           v.ctypes.data_as(C.c_void_p)), "ccfr_server_get_state")
        return x, v

    def info(self) -> dict:
        i = ServerInfo()
        _check(lib().ccfr_server_get_info(self.h, C.byref(i)), "ccfr_server_get_info")
        return i.as_dict()

    def stall(self, scene_id: int, on: bool = True):
        _check(lib().ccfr_server_set_stall(self.h, scene_id, int(on)), "ccfr_server_set_stall")

    def close(self):
        if getattr(self, "h", None):
            lib().ccfr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
