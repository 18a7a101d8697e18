"""Seeded synthetic scenes for CCFR (inputs only).

This module builds the arrays that both the CUDA library and the FP64 oracle
consume: positions with inverse masses, velocities, triangles, edges and the
per-scene parameters.  It holds none of the method's arithmetic (no distances,
no planes, no projections); it only lays out geometry and draws seeded random
numbers with numpy's PCG64 (``numpy.random.default_rng``).

Units are metres, seconds and kilograms.  Movable vertices carry the inverse
of their mass in ``x[:, 3]``; static obstacle vertices carry 0, which is how
the paper's narrow phase (Alg. 3) treats immovable primitives (zero inverse
mass gives them no share of the separation).

The workloads stand in for the paper's own scenes (Sec. 4.2), whose assets
are not available: a cloth dropped on a sphere, a self-colliding cloth stack,
codimensional wires falling on a grate, and particle clouds.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np


@dataclass
class Scene:
    name: str
    x: np.ndarray                  # (N, 4) float32: xyz + inverse mass
    v: np.ndarray                  # (N, 4) float32: xyz velocity, w unused (0)
    tris: np.ndarray               # (T, 3) int32
    edges: np.ndarray              # (E, 2) int32, a < b, sorted lexicographically
    params: dict = field(default_factory=dict)
    # XPBD constraints that are no collision primitives (mixed scenes): extra
    # distance links with their compliances, and tetrahedra with one volume
    # compliance
    links: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    link_compliance: np.ndarray = field(default_factory=lambda: np.zeros(0, np.float32))
    tets: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int32))
    volume_compliance: float = 0.0

    @property
    def n_verts(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_movable(self) -> int:
        return int(np.count_nonzero(self.x[:, 3] > 0))

    def copy(self) -> "Scene":
        return Scene(self.name, self.x.copy(), self.v.copy(), self.tris.copy(),
                     self.edges.copy(), dict(self.params), self.links.copy(), self.link_compliance.copy(),
                     self.tets.copy(), self.volume_compliance)


def default_params(r: float, xi: float, *, delta: float = 0.0, dt: float = 1.0 / 60.0,
                   iters: int = 10, steps: int = 20, plane_capacity: int = 64,
                   k_resp: float = 0.0, delta_v: float | None = None, mu_s: float = 0.0,
                   mu_k: float = 0.0) -> dict:
    """Parameter set of one scene.

    r, xi, delta follow the paper's parameter table (Table 3); eps is the
    retraction margin of Sec. 3.2 (1e-6 in scene units), eps_dep the
    dependence tolerance of Alg. 1, n_max the pass budget of Alg. 2, and
    tau_feas the tolerance of the final feasibility check.  ``pad`` is the
    AABB enlargement r + xi/2 + delta/2 of Sec. 4.1, rounded once to binary32
    so that every consumer evaluates the same candidate predicate.  The
    contact response of Sec. 3.3 acts when delta > 0: stiffness k_resp,
    occlusion transition width delta_v (default delta / 2), friction
    coefficients mu_s, mu_k.
    """
    pad = np.float32(np.float32(r) + np.float32(0.5) * np.float32(xi)
                     + np.float32(0.5) * np.float32(delta))
    return dict(r=float(r), xi=float(xi), delta=float(delta), pad=float(pad),
                eps=1e-6, eps_dep=1e-6, tau_feas=1e-7, n_max=1,
                dt=float(dt), iters=int(iters), steps=int(steps),
                gravity=(0.0, -9.81, 0.0), compliance=0.0,
                plane_capacity=int(plane_capacity), k_resp=float(k_resp),
                delta_v=float(0.5 * delta if delta_v is None else delta_v), mu_s=float(mu_s), mu_k=float(mu_k))


def with_response(sc: "Scene", delta: float, k_resp: float, mu_s: float = 0.0, mu_k: float = 0.0,
                  delta_v: float | None = None) -> "Scene":
    """Copy of a scene with the contact response of Sec. 3.3 switched on
    (the AABB pad is re-derived with the repulsion range included)."""
    p = sc.params
    q = default_params(p["r"], p["xi"], delta=delta, dt=p["dt"], iters=p["iters"], steps=p["steps"],
                       plane_capacity=p["plane_capacity"], k_resp=k_resp, delta_v=delta_v, mu_s=mu_s, mu_k=mu_k)
    q["gravity"] = p["gravity"]
    q["compliance"] = p["compliance"]
    out = sc.copy()
    out.params = q
    return out


def canonical_edges(e: np.ndarray) -> np.ndarray:
    """Unique undirected edges (min, max), sorted lexicographically."""
    if len(e) == 0:
        return np.zeros((0, 2), np.int32)
    e = np.sort(np.asarray(e, np.int64).reshape(-1, 2), axis=1)
    key = np.unique(e[:, 0] * (int(e.max()) + 1) + e[:, 1])
    m = int(e.max()) + 1
    return np.stack([key // m, key % m], 1).astype(np.int32)


def edges_of_tris(tris: np.ndarray) -> np.ndarray:
    """Unique undirected edges of a triangle list, (min, max), lexicographic."""
    if len(tris) == 0:
        return np.zeros((0, 2), np.int32)
    t = np.asarray(tris)
    return canonical_edges(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]], axis=0))


def _grid_tris(nx: int, nz: int, base: int = 0) -> np.ndarray:
    """Quads of an nx-by-nz vertex grid (row-major in z), split on one diagonal."""
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(nz - 1), indexing="ij")
    v00 = (i * nz + j).ravel()
    v10 = ((i + 1) * nz + j).ravel()
    v01 = (i * nz + j + 1).ravel()
    v11 = ((i + 1) * nz + j + 1).ravel()
    t = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    return (t + base).astype(np.int32)


def _cloth_grid(n_side: int, spacing: float, center, rng, jitter: float) -> np.ndarray:
    i, j = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    off = (n_side - 1) * spacing / 2.0
    p = np.zeros((n_side * n_side, 3))
    p[:, 0] = i.ravel() * spacing - off + center[0]
    p[:, 1] = center[1]
    p[:, 2] = j.ravel() * spacing - off + center[2]
    if jitter > 0:
        p += rng.uniform(-jitter, jitter, size=p.shape)
    return p


@lru_cache(maxsize=16)
def _unit_uv_sphere(slices: int, stacks: int):
    pts = [(0.0, 1.0, 0.0)]
    for i in range(1, stacks):
        th = np.pi * i / stacks
        for j in range(slices):
            ph = 2.0 * np.pi * j / slices
            pts.append((np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)))
    pts.append((0.0, -1.0, 0.0))
    south = len(pts) - 1
    tris = []

    def ring(i, j):
        return 1 + (i - 1) * slices + (j % slices)

    for j in range(slices):
        tris.append((0, ring(1, j + 1), ring(1, j)))
    for i in range(1, stacks - 1):
        for j in range(slices):
            a, b = ring(i, j), ring(i, j + 1)
            c, d = ring(i + 1, j), ring(i + 1, j + 1)
            tris.append((a, b, d))
            tris.append((a, d, c))
    for j in range(slices):
        tris.append((south, ring(stacks - 1, j), ring(stacks - 1, j + 1)))
    p = np.asarray(pts)
    t = np.asarray(tris, np.int32)
    p.setflags(write=False)
    t.setflags(write=False)
    return p, t, edges_of_tris(t)


def uv_sphere(radius: float, slices: int, stacks: int, center=(0.0, 0.0, 0.0)):
    """UV sphere: 2 poles + (stacks-1) rings of `slices` vertices.

    slices=50, stacks=41 gives 2,002 vertices and 4,000 triangles.
    """
    p, t, _ = _unit_uv_sphere(slices, stacks)
    return p * radius + np.asarray(center), t.copy()


def _assemble(name, parts_p, parts_w, parts_tris, parts_edges, params, v=None) -> Scene:
    base = 0
    tris, edges = [], []
    for p, t, e in zip(parts_p, parts_tris, parts_edges):
        if t is not None and len(t):
            tris.append(np.asarray(t) + base)
        if e is not None and len(e):
            edges.append(np.asarray(e) + base)
        base += len(p)
    P = np.concatenate(parts_p, 0)
    W = np.concatenate(parts_w, 0)
    x = np.zeros((len(P), 4), np.float32)
    x[:, :3] = P
    x[:, 3] = W
    T = np.concatenate(tris, 0).astype(np.int32) if tris else np.zeros((0, 3), np.int32)
    E = canonical_edges(np.concatenate(edges, 0)) if edges else np.zeros((0, 2), np.int32)
    vel = np.zeros((len(P), 4), np.float32)
    if v is not None:
        vel[:, :3] = v
    return Scene(name, x, vel, T, E, params)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def cloth_on_sphere(n_side: int = 32, spacing: float = 0.01, jitter: float = 1e-3,
                    radius: float = 0.10, slices: int = 50, stacks: int = 41,
                    lift: float = 0.02, seed: int = 1, iters: int = 10, steps: int = 20,
                    cloth_mass: float = 1e-3, plane_capacity: int = 256) -> Scene:
    """Square cloth dropped on a static UV sphere.

    Defaults: 32x32 vertices at 1 cm (1,922 triangles) with seeded +-1 mm
    jitter per coordinate, 2 cm above a static 4,000-triangle sphere of
    radius 10 cm; r = 5 mm, xi = 1 mm, dt = 1/60 s, 10 iterations.
    """
    rng = np.random.default_rng(seed)
    cp = _cloth_grid(n_side, spacing, (0.0, radius + lift, 0.0), rng, jitter)
    ct = _grid_tris(n_side, n_side)
    sp, st = uv_sphere(radius, slices, stacks)
    params = default_params(5e-3, 1e-3, iters=iters, steps=steps,
                            plane_capacity=plane_capacity)
    return _assemble("cloth_on_sphere", [cp, sp],
                     [np.full(len(cp), 1.0 / cloth_mass), np.zeros(len(sp))],
                     [ct, st], [edges_of_tris(ct), edges_of_tris(st)], params)


def smooth_velocity(p: np.ndarray, speed: float, rng, n_waves: int = 4,
                    wavelengths=(0.25, 1.0)) -> np.ndarray:
    """Seeded smooth velocity field: per component a sum of n_waves sinusoids
    sin(k . p + phase) with random directions, wavelengths uniform in the given
    range (metres) and random phases and amplitudes, scaled so that the largest
    magnitude of each component over the points is `speed`."""
    v = np.zeros((len(p), 3))
    for c in range(3):
        acc = np.zeros(len(p))
        for _ in range(n_waves):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            k = 2.0 * np.pi / rng.uniform(*wavelengths) * d
            acc += rng.uniform(0.5, 1.0) * np.sin(p @ k + rng.uniform(0.0, 2.0 * np.pi))
        m = np.abs(acc).max()
        v[:, c] = acc * (speed / m if m > 0 else 0.0)
    return v


def cloth_stack(n_side: int = 256, layers: int = 4, spacing: float = 4e-3,
                gap: float = 2e-3, speed: float = 0.5, seed: int = 2, jitter: float = 0.0,
                iters: int = 20, steps: int = 100, cloth_mass: float = 1e-3,
                r: float = 2e-3, xi: float = 1e-3, plane_capacity: int = 1024,
                velocity: str = "iid") -> Scene:
    """Self-colliding stack of parallel cloth layers.

    Defaults: 4 layers of 256x256 vertices at 4 mm, 2 mm apart in y, every
    velocity component drawn iid from U(-speed, speed); r = 2 mm, xi = 1 mm,
    20 iterations, no obstacle.  velocity="smooth": the field of
    smooth_velocity (4 sinusoids per component, wavelengths 0.25-1 m, scaled
    to +-speed) instead of iid draws.
    """
    rng = np.random.default_rng(seed)
    ps, ts, es = [], [], []
    for k in range(layers):
        p = _cloth_grid(n_side, spacing, (0.0, k * gap, 0.0), rng, jitter)
        t = _grid_tris(n_side, n_side)
        ps.append(p)
        ts.append(t)
        es.append(edges_of_tris(t))
    n = sum(len(p) for p in ps)
    if velocity == "smooth":
        vel = smooth_velocity(np.concatenate(ps), speed, rng)
    elif velocity == "iid":
        vel = rng.uniform(-speed, speed, size=(n, 3))
    else:
        raise ValueError(f"velocity must be 'iid' or 'smooth', not {velocity!r}")
    params = default_params(r, xi, iters=iters, steps=steps, plane_capacity=plane_capacity)
    return _assemble("cloth_stack", ps, [np.full(len(p), 1.0 / cloth_mass) for p in ps],
                     ts, es, params, v=vel)


def wires(n_grid: int = 128, n_seg: int = 64, seg_len: float = 2e-3, axis_pitch: float = 0.02,
          seed: int = 3, grate: bool = True, grate_pitch: float = 0.01,
          iters: int = 10, steps: int = 50, strand_mass: float = 1e-4,
          plane_capacity: int = 128) -> Scene:
    """Helical polyline strands above a static grate of rods (edge-edge only).

    Defaults: 128x128 = 16,384 strands of 64 segments of 2 mm, helix radius
    U(2, 8) mm, pitch U(3, 6) mm, random phase, vertical axes 20 mm apart,
    bottoms 2 cm above the grate; the grate has x-rods at y = 0 and z-rods at
    y = 2 mm, 1 cm apart, in 1 cm segments.  r = 1 mm, xi = 0.5 mm.
    """
    rng = np.random.default_rng(seed)
    ns = n_grid * n_grid
    rad = rng.uniform(2e-3, 8e-3, ns)
    pitch = rng.uniform(3e-3, 6e-3, ns)
    phase = rng.uniform(0.0, 2.0 * np.pi, ns)
    gi, gj = np.meshgrid(np.arange(n_grid), np.arange(n_grid), indexing="ij")
    ax = (gi.ravel() - (n_grid - 1) / 2.0) * axis_pitch
    az = (gj.ravel() - (n_grid - 1) / 2.0) * axis_pitch
    c = pitch / (2.0 * np.pi)
    dth = seg_len / np.sqrt(rad ** 2 + c ** 2)
    k = np.arange(n_seg + 1)
    th = phase[:, None] + k[None, :] * dth[:, None]
    y0 = 0.002 + 0.02
    P = np.zeros((ns, n_seg + 1, 3))
    P[..., 0] = ax[:, None] + rad[:, None] * np.cos(th)
    P[..., 1] = y0 + c[:, None] * (k[None, :] * dth[:, None])
    P[..., 2] = az[:, None] + rad[:, None] * np.sin(th)
    P = P.reshape(-1, 3)
    base = (np.arange(ns) * (n_seg + 1))[:, None] + np.arange(n_seg)[None, :]
    E = np.stack([base.ravel(), base.ravel() + 1], 1)
    parts_p, parts_w, parts_e = [P], [np.full(len(P), 1.0 / strand_mass)], [E]
    if grate:
        half = (n_grid - 1) / 2.0 * axis_pitch + 0.03
        m = int(np.ceil(2 * half / grate_pitch)) + 1
        coords = -half + grate_pitch * np.arange(m)
        # x-rods at y = 0 (run along x, one per z), z-rods at y = 2 mm
        gx = np.zeros((m, m, 3))
        gx[..., 0] = coords[None, :]
        gx[..., 2] = coords[:, None]
        gz = np.zeros((m, m, 3))
        gz[..., 0] = coords[:, None]
        gz[..., 1] = 0.002
        gz[..., 2] = coords[None, :]
        rb = (np.arange(m) * m)[:, None] + np.arange(m - 1)[None, :]
        re = np.stack([rb.ravel(), rb.ravel() + 1], 1)
        parts_p += [gx.reshape(-1, 3), gz.reshape(-1, 3)]
        parts_w += [np.zeros(m * m), np.zeros(m * m)]
        parts_e += [re, re]
    params = default_params(1e-3, 5e-4, iters=iters, steps=steps,
                            plane_capacity=plane_capacity)
    return _assemble("wires", parts_p, parts_w, [None] * len(parts_p), parts_e, params)


def particle_cloud(n: int, spacing: float = 3e-3, jitter: float = 4e-4, seed: int = 0,
                   sphere_radius: float = 0.05, lift: float = 0.01, mass: float = 5e-4,
                   iters: int = 10, steps: int = 20, plane_capacity: int = 64) -> Scene:
    """Isolated particles on a jittered cubic lattice above a static sphere.

    Particle radius 1 mm is expressed as xi = 2 mm (centre-to-centre offset);
    the lattice spacing 3 mm with jitter U(-0.4, 0.4) mm keeps every initial
    gap at least 1.5 xi.
    """
    rng = np.random.default_rng(seed)
    side = int(np.ceil(n ** (1.0 / 3.0)))
    i, j, k = np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij")
    p = np.stack([i.ravel(), j.ravel(), k.ravel()], 1)[:n].astype(np.float64) * spacing
    p -= p.mean(axis=0)
    p[:, 1] += sphere_radius + lift + (side - 1) * spacing / 2.0
    p += rng.uniform(-jitter, jitter, size=p.shape)
    sp, st = uv_sphere(sphere_radius, 50, 41)
    params = default_params(1e-3, 2e-3, iters=iters, steps=steps, plane_capacity=plane_capacity)
    return _assemble("particle_cloud", [p, sp], [np.full(len(p), 1.0 / mass), np.zeros(len(sp))],
                     [None, st], [None, edges_of_tris(st)], params)


def _tet_lattice(n: int, h: float, origin) -> tuple[np.ndarray, np.ndarray]:
    """n^3 vertex lattice of spacing h; every cube cell split into six
    tetrahedra around its main diagonal (the same diagonal in every cell, so
    shared faces match)."""
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    P = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(np.float64) * h + np.asarray(origin, np.float64)
    vid = lambda a, b, c: (a * n + b) * n + c  # noqa: E731
    a, b, c = np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()
    c000, c111 = vid(a, b, c), vid(a + 1, b + 1, c + 1)
    c100, c010, c001 = vid(a + 1, b, c), vid(a, b + 1, c), vid(a, b, c + 1)
    c110, c101, c011 = vid(a + 1, b + 1, c), vid(a + 1, b, c + 1), vid(a, b + 1, c + 1)
    tets = np.concatenate([np.stack(t, 1) for t in (
        (c000, c100, c110, c111), (c000, c100, c101, c111), (c000, c010, c110, c111),
        (c000, c010, c011, c111), (c000, c001, c101, c111), (c000, c001, c011, c111))], 0)
    return P, tets.astype(np.int32)


def _boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one tetrahedron (the volume's surface)."""
    f = np.concatenate([tets[:, [0, 1, 2]], tets[:, [0, 1, 3]], tets[:, [0, 2, 3]], tets[:, [1, 2, 3]]], 0)
    fs = np.sort(f, axis=1)
    _, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    return f[cnt[inv.ravel()] == 1].astype(np.int32)


def _hinge_links(tris: np.ndarray) -> np.ndarray:
    """For every edge shared by two triangles, the two vertices opposite it
    (the cloth's bending links)."""
    t = np.asarray(tris, np.int64)
    rows = []
    for a, b, o in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        e = np.sort(np.stack([t[:, a], t[:, b]], 1), axis=1)
        rows.append(np.concatenate([e, t[:, [o]]], 1))
    r = np.concatenate(rows, 0)
    order = np.lexsort((r[:, 1], r[:, 0]))
    r = r[order]
    same = (r[1:, 0] == r[:-1, 0]) & (r[1:, 1] == r[:-1, 1])
    pairs = np.stack([r[:-1][same, 2], r[1:][same, 2]], 1)
    return np.sort(pairs, axis=1).astype(np.int32)


def codimensional(rod_seg: int = 16, cube_n: int = 3, particle_layers: int = 1, seed: int = 6,
                  iters: int = 10, steps: int = 20, plane_capacity: int = 768, speed: float = 0.5,
                  cloth_bending: float = 1.0, rod_bending: float = 0.1, volume_compliance: float = 0.0) -> Scene:
    """Rods, soft volumes, a cloth and particles in one simulation (a synthetic
    stand-in for the paper's coupled codimensional scene, Sec. 5).

    Lattice spacing h = 4 mm, scene width W = rod_seg * h.  Two crossing layers
    of rods pinned at both ends (x-rods at y = 0, z-rods at y = 5 mm, 10 mm
    apart), each with bending links to every second neighbour; a grid of soft
    cubes (cube_n^3 lattice, six tetrahedra per cell, 8 mm apart) over the
    left half, whose boundary triangles are their collision surface, whose
    inner edges are links and whose tetrahedra carry volume constraints; a
    cloth over the same half with hinge bending links; particle layers over the
    whole width, so that half of them land on the cloth and half directly on
    the rods (point-edge pairs).  Every movable vertex starts falling at
    `speed`; positions are jittered by U(-0.2, 0.2) mm.  r = 2 mm, xi = 1 mm.
    """
    rng = np.random.default_rng(seed)
    h = 4e-3
    W = rod_seg * h
    parts_p, parts_w, parts_t, parts_e, links, lcomp, tets = [], [], [], [], [], [], []
    base = 0

    def add(P, w, t=None, e=None, lk=None, lc=0.0, tt=None):
        nonlocal base
        parts_p.append(P)
        parts_w.append(w)
        parts_t.append(t)
        parts_e.append(e)
        if lk is not None and len(lk):
            links.append(np.asarray(lk) + base)
            lcomp.append(np.full(len(lk), lc))
        if tt is not None and len(tt):
            tets.append(np.asarray(tt) + base)
        base += len(P)

    # rods: x-rods at y = 0 and z-rods at y = 5 mm, pinned at both ends
    n_rods = max(2, int(W / 0.01))
    zs = (np.arange(n_rods) - (n_rods - 1) / 2.0) * 0.01
    u = np.arange(rod_seg + 1) * h - W / 2.0
    for layer in range(2):
        for z in zs:
            P = np.zeros((rod_seg + 1, 3))
            if layer == 0:
                P[:, 0], P[:, 2] = u, z
            else:
                P[:, 0], P[:, 1], P[:, 2] = z, 5e-3, u
            w = np.full(rod_seg + 1, 1.0 / 2e-4)
            w[0] = w[-1] = 0.0
            k = np.arange(rod_seg)
            bend = np.stack([np.arange(rod_seg - 1), np.arange(rod_seg - 1) + 2], 1)
            add(P, w, None, np.stack([k, k + 1], 1), bend, rod_bending)
    # soft cubes over the left half
    side = (cube_n - 1) * h
    pitch = side + 8e-3
    ncx = max(1, int((W / 2.0) // pitch))
    ncz = max(1, int(W // pitch))
    y_cube = 0.015
    for a in range(ncx):
        for b in range(ncz):
            org = (-W / 2.0 + a * pitch + 4e-3, y_cube, -W / 2.0 + b * pitch + 4e-3)
            P, tt = _tet_lattice(cube_n, h, org)
            faces = _boundary_faces(tt)
            e_surf = edges_of_tris(faces)
            e_all = canonical_edges(np.concatenate([tt[:, [i, j]] for i in range(4) for j in range(i + 1, 4)], 0))
            surf = set(map(tuple, e_surf.tolist()))
            inner = np.array([e for e in e_all.tolist() if tuple(e) not in surf], np.int32).reshape(-1, 2)
            add(P, np.full(len(P), 1.0 / 5e-4), faces, e_surf, inner, 0.0, tt)
    # cloth over the left half
    y_cloth = y_cube + side + 8e-3
    nx, nz = rod_seg // 2 + 1, rod_seg + 1
    gi, gj = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
    P = np.zeros((nx * nz, 3))
    P[:, 0] = -W / 2.0 + gi.ravel() * h
    P[:, 1] = y_cloth
    P[:, 2] = -W / 2.0 + gj.ravel() * h
    ct = _grid_tris(nx, nz)
    add(P, np.full(len(P), 1.0 / 1e-4), ct, edges_of_tris(ct), _hinge_links(ct), cloth_bending)
    # particle layers over the whole width
    y_part = y_cloth + 8e-3
    pi, pk, pl = np.meshgrid(np.arange(rod_seg), np.arange(rod_seg), np.arange(particle_layers), indexing="ij")
    P = np.zeros((pi.size, 3))
    P[:, 0] = -W / 2.0 + (pi.ravel() + 0.5) * h
    P[:, 1] = y_part + pl.ravel() * h
    P[:, 2] = -W / 2.0 + (pk.ravel() + 0.5) * h
    add(P, np.full(len(P), 1.0 / 2e-4))

    params = default_params(2e-3, 1e-3, iters=iters, steps=steps, plane_capacity=plane_capacity)
    allp = np.concatenate(parts_p, 0)
    allw = np.concatenate(parts_w, 0)
    allp = allp + rng.uniform(-2e-4, 2e-4, size=allp.shape) * (allw > 0)[:, None]
    vel = np.zeros_like(allp)
    vel[:, 1] = -speed * (allw > 0)
    offs = np.cumsum([0] + [len(q) for q in parts_p])
    sc = _assemble("codimensional", [allp[offs[i]:offs[i + 1]] for i in range(len(parts_p))], parts_w,
                   parts_t, parts_e, params, v=vel)
    sc.links = np.concatenate(links, 0).astype(np.int32) if links else np.zeros((0, 2), np.int32)
    sc.link_compliance = np.concatenate(lcomp, 0).astype(np.float32) if lcomp else np.zeros(0, np.float32)
    sc.tets = np.concatenate(tets, 0).astype(np.int32) if tets else np.zeros((0, 4), np.int32)
    sc.volume_compliance = float(volume_compliance)
    return sc


def particles_on_rod(n_seg: int = 8, seg_len: float = 4e-3, n_particles: int = 12, height: float = 3e-3,
                     pinned_rod: bool = True, cloth_patch: bool = False, speed: float = 0.3, seed: int = 8,
                     iters: int = 10, steps: int = 20, plane_capacity: int = 64) -> Scene:
    """Particles dropped just above a rod along x (point-edge pairs only, plus
    point-point pairs between the particles).  The rod is pinned at both ends
    (or wholly static with pinned_rod=False); the particles sit `height` above
    it, spread along it with U(-1, 1) mm offsets in x and z.  cloth_patch adds
    a small static cloth of 1 mm spacing far away, whose short edges shrink the
    edge cell so that the rod's segments become oversized edges.
    r = 2 mm, xi = 1 mm."""
    rng = np.random.default_rng(seed)
    L = n_seg * seg_len
    P = np.zeros((n_seg + 1, 3))
    P[:, 0] = np.arange(n_seg + 1) * seg_len - L / 2.0
    w = np.full(n_seg + 1, 1.0 / 2e-4) if pinned_rod else np.zeros(n_seg + 1)
    w[0] = w[-1] = 0.0
    k = np.arange(n_seg)
    parts_p, parts_w, parts_t, parts_e = [P], [w], [None], [np.stack([k, k + 1], 1)]
    bend = np.stack([np.arange(n_seg - 1), np.arange(n_seg - 1) + 2], 1) if pinned_rod else np.zeros((0, 2))
    Q = np.zeros((n_particles, 3))
    Q[:, 0] = (np.arange(n_particles) + 0.5) / n_particles * L - L / 2.0 + rng.uniform(-1e-3, 1e-3, n_particles)
    Q[:, 1] = height + 4e-3 * (np.arange(n_particles) % 2)
    Q[:, 2] = rng.uniform(-1e-3, 1e-3, n_particles)
    parts_p.append(Q)
    parts_w.append(np.full(n_particles, 1.0 / 2e-4))
    parts_t.append(None)
    parts_e.append(None)
    if cloth_patch:
        C = _cloth_grid(12, 1e-3, (0.0, 0.05, 0.05), rng, 0.0)
        ct = _grid_tris(12, 12)
        parts_p.append(C)
        parts_w.append(np.zeros(len(C)))
        parts_t.append(ct)
        parts_e.append(edges_of_tris(ct))
    params = default_params(2e-3, 1e-3, iters=iters, steps=steps, plane_capacity=plane_capacity)
    vel = np.zeros((sum(len(q) for q in parts_p), 3))
    vel[n_seg + 1:n_seg + 1 + n_particles, 1] = -speed
    sc = _assemble("particles_on_rod", parts_p, parts_w, parts_t, parts_e, params, v=vel)
    sc.links = np.asarray(bend, np.int32).reshape(-1, 2)
    sc.link_compliance = np.full(len(sc.links), 0.1, np.float32)
    return sc


def batch(n_scenes: int = 512, seed: int = 4, min_verts: int = 1024, max_verts: int = 65536,
          median_verts: int = 8192, particle_frac: float = 0.2, iters: int = 10, steps: int = 20,
          plane_capacity: int = 256, sphere_slices: int = 50, sphere_stacks: int = 41) -> list:
    """Independent scenes of uneven sizes for the batched step.

    Sizes N ~ lognormal(ln median, ln 2) clipped to [min, max].  80% are
    square cloths of side round(sqrt(N)) at 1 cm (+-1 mm jitter) dropped on a
    static UV sphere of radius 0.3 x the cloth side; 20% are particle clouds of
    N points (3 mm lattice, +-0.4 mm jitter) above a static sphere.  Cloth:
    r = 5 mm, xi = 1 mm; particles: r = 1 mm, xi = 2 mm; 10 iterations.
    """
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.exp(rng.normal(np.log(median_verts), np.log(2.0), n_scenes)), min_verts, max_verts)
    kinds = rng.uniform(size=n_scenes) < particle_frac
    out = []
    for k in range(n_scenes):
        n = int(sizes[k])
        sub = int(rng.integers(1 << 30))
        if kinds[k]:
            side_m = np.ceil(n ** (1.0 / 3.0)) * 3e-3
            sc = particle_cloud(n, seed=sub, sphere_radius=max(0.02, 0.3 * side_m), iters=iters, steps=steps,
                                plane_capacity=plane_capacity)
        else:
            side = max(4, int(round(np.sqrt(n))))
            sc = cloth_on_sphere(n_side=side, radius=0.3 * side * 0.01, slices=sphere_slices, stacks=sphere_stacks,
                                 seed=sub, iters=iters, steps=steps, plane_capacity=plane_capacity)
        sc.name = f"batch{k}_{sc.name}"
        out.append(sc)
    return out


def config(k: int, seed: int | None = None) -> Scene:
    """Scene of configuration k (1-based) at its full size."""
    if k == 1:
        return cloth_on_sphere(seed=1 if seed is None else seed)
    if k == 2:
        return cloth_stack(seed=2 if seed is None else seed)
    if k == 3:
        return wires(seed=3 if seed is None else seed)
    raise ValueError(f"no single-scene configuration {k}")


# --------------------------------------------------------------------------
# Small scenes for the tests
# --------------------------------------------------------------------------

def large_triangle(kind: str = "point", size: float = 0.1, height: float = 3e-3,
                   r: float = 5e-3, xi: float = 1e-3, speed: float = -1.0) -> Scene:
    """A point (or short edge) under the middle of one large static triangle.

    Every triangle vertex is much farther than 2r + xi from the point, so
    only a closest-point (not a vertex-distance) search can catch the pair
    (the paper's large-triangle test, Sec. 4.2).
    """
    tri_p = np.array([[-size, height, -size], [size, height, -size], [0.0, height, size]])
    if kind == "point":
        q = np.array([[0.0, 0.0, 0.0]])
        qe = None
    else:
        q = np.array([[-0.002, 0.0, 0.0], [0.002, 0.0, 0.0]])
        qe = np.array([[0, 1]])
    params = default_params(r, xi, iters=10, steps=10)
    params["gravity"] = (0.0, 0.0, 0.0)
    vel = np.zeros((len(q) + 3, 3))
    vel[: len(q), 1] = -speed
    return _assemble("large_triangle_" + kind, [q, tri_p], [np.full(len(q), 1e3), np.zeros(3)],
                     [None, np.array([[0, 1, 2]])], [qe, np.array([[0, 1], [1, 2], [0, 2]])],
                     params, v=vel)


def two_particles(dist: float = 0.01, speed: float = 1.0, xi: float = 2e-3, r: float = 1e-3,
                  w=(2e3, 2e3)) -> Scene:
    """Two isolated particles closing head-on along x."""
    p = np.array([[-dist / 2, 0.0, 0.0], [dist / 2, 0.0, 0.0]])
    vel = np.array([[speed, 0.0, 0.0], [-speed, 0.0, 0.0]])
    params = default_params(r, xi, iters=10, steps=10)
    params["gravity"] = (0.0, 0.0, 0.0)
    return _assemble("two_particles", [p], [np.asarray(w, float)], [None], [None], params, v=vel)


def particle_over_floor(height: float = 0.004, size: float = 0.05, r: float = 1e-3,
                        xi: float = 1e-3, iters: int = 10, steps: int = 30, delta: float = 0.0,
                        k_resp: float = 0.0, mu_s: float = 0.0, mu_k: float = 0.0,
                        v0=(0.0, 0.0, 0.0)) -> Scene:
    """One particle (mass 1 g) above a static two-triangle floor at y = 0,
    optionally with the contact response and an initial velocity."""
    q = np.array([[0.02, height, -0.01]])
    f = np.array([[-size, 0, -size], [size, 0, -size], [size, 0, size], [-size, 0, size]])
    params = default_params(r, xi, iters=iters, steps=steps, delta=delta, k_resp=k_resp, mu_s=mu_s,
                            mu_k=mu_k)
    vel = np.zeros((5, 3))
    vel[0] = v0
    return _assemble("particle_over_floor", [q, f], [np.full(1, 1e3), np.zeros(4)],
                     [None, np.array([[0, 1, 2], [0, 2, 3]])],
                     [None, edges_of_tris(np.array([[0, 1, 2], [0, 2, 3]]))], params, v=vel)


def card_stack(n_cards: int = 52, xi: float = 1e-3, size: float = 0.06, gap_factor: float = 1.5,
               r: float = 5e-4, floor: bool = True, iters: int = 10, steps: int = 10) -> Scene:
    """Stacked square cards (two triangles each), exactly parallel and aligned.

    Aligned cards give many identical or dependent planes per vertex (the
    paper's degeneration test, Sec. 4.2).
    """
    ps, ws, ts, es = [], [], [], []
    quad_t = np.array([[0, 1, 2], [0, 2, 3]])
    for k in range(n_cards):
        y = (k + 1) * gap_factor * xi
        ps.append(np.array([[-size, y, -size], [size, y, -size], [size, y, size], [-size, y, size]]))
        ws.append(np.full(4, 1.0 / 2.5e-4))
        ts.append(quad_t)
        es.append(edges_of_tris(quad_t))
    if floor:
        f = 2 * size
        ps.append(np.array([[-f, 0, -f], [f, 0, -f], [f, 0, f], [-f, 0, f]]))
        ws.append(np.zeros(4))
        ts.append(quad_t)
        es.append(edges_of_tris(quad_t))
    params = default_params(r, xi, iters=iters, steps=steps)
    return _assemble("card_stack", ps, ws, ts, es, params)


def triangle_soup(n_tris: int = 60, box: float = 0.05, size: float = 0.01, seed: int = 0,
                  static_frac: float = 0.2, r: float = 2e-3, xi: float = 1e-3,
                  n_points: int = 0) -> Scene:
    """Disjoint random small triangles (and optional isolated points) in a box.

    Triangles may lie close to each other or intersect; the scene exercises
    the candidate predicate, not the dynamics.
    """
    rng = np.random.default_rng(seed)
    c = rng.uniform(-box, box, size=(n_tris, 1, 3))
    p = (c + rng.uniform(-size, size, size=(n_tris, 3, 3))).reshape(-1, 3)
    t = np.arange(3 * n_tris).reshape(n_tris, 3)
    w = np.where(rng.uniform(size=n_tris) < static_frac, 0.0, 1e3).repeat(3)
    parts_p, parts_w, parts_t, parts_e = [p], [w], [t], [edges_of_tris(t)]
    if n_points:
        q = rng.uniform(-box, box, size=(n_points, 3))
        parts_p.append(q)
        parts_w.append(np.where(rng.uniform(size=n_points) < static_frac, 0.0, 1e3))
        parts_t.append(None)
        parts_e.append(None)
    params = default_params(r, xi)
    return _assemble("triangle_soup", parts_p, parts_w, parts_t, parts_e, params)


def isolated_points(x: np.ndarray, edges: np.ndarray, links=None, tets=None) -> np.ndarray:
    """Indices of vertices that belong to no edge, link or tetrahedron (the
    point primitives)."""
    used = np.zeros(len(x), bool)
    for a in (edges, links, tets):
        if a is not None and len(a):
            used[np.asarray(a).ravel()] = True
    return np.nonzero(~used)[0].astype(np.int32)
