"""Exact Euclidean projection onto a vertex's convex collision-free region.

TEST INFRASTRUCTURE ONLY: a report-only diagnostic beside Alg. 2.

The region of Sec. 3.1 is the intersection of the half-spaces
rho_k(y) = n_k . y + d_k >= 0 (y = x' - x, Eq. 2-3 in the form of Alg. 2).
Sec. 3.2 states the goal of the projection as the closest point of that
region; Alg. 2 reaches a point of it incrementally (Plesnik's projection onto
the intersection of an order-chosen set of violated planes, with retractions,
passes and a halt), which in general is not the closest point.  This module
computes the closest point itself, so that the tests can report how often and
by how much the two differ.  Nothing here is compared with the GPU.

Method: the dual active-set algorithm of Goldfarb and Idnani (Math.
Programming 27, 1983) for min 1/2 |y - y0|^2 subject to n_k . y >= -d_k,
which starts at the unconstrained minimum y0 and adds the most violated
constraint until none is violated, dropping constraints whose multipliers
would turn negative.  With the identity Hessian its steps reduce to
projections onto the span of the active normals.  ``brute_force`` enumerates
every active set of at most three planes (the optimum in 3-D has at most three
independent active constraints) and is the reference the first is pinned to.
"""
from __future__ import annotations

import itertools

import numpy as np


def _project_affine(y0, N, b):
    """Closest point to y0 on {y : N y = b} (rows independent)."""
    return y0 + N.T @ np.linalg.solve(N @ N.T, b - N @ y0)


def project(y0, normals, d, tol: float = 1e-15, max_iter: int = 10000):
    """Closest point of {y : normals @ y + d >= 0} to y0, and its multipliers.

    Returns (y, active, u): the optimum, the active plane indices and their
    multipliers (y = y0 + sum u_i n_i, u_i >= 0).  Returns (None, None, None)
    when the region is empty.
    """
    y0 = np.asarray(y0, np.float64)
    Nall = np.asarray(normals, np.float64).reshape(-1, 3)
    b = -np.asarray(d, np.float64).reshape(-1)
    y = y0.copy()
    act: list[int] = []
    u = np.zeros(0)
    for _ in range(max_iter):
        s = Nall @ y - b
        if len(s) == 0:
            return y, [], np.zeros(0)
        s_act = s.copy()
        s_act[act] = np.inf
        p = int(np.argmin(s_act))
        if not (s_act[p] < -tol):
            return y, act, u
        up = 0.0
        while True:
            npv = Nall[p]
            if act:
                N = Nall[act]
                r = np.linalg.solve(N @ N.T, N @ npv)
                z = npv - N.T @ r
            else:
                r = np.zeros(0)
                z = npv
            t1, l = np.inf, -1
            for j in range(len(act)):
                if r[j] > 0 and u[j] / r[j] < t1:
                    t1, l = u[j] / r[j], j
            zz = float(z @ npv)
            if zz <= 1e-14 * float(npv @ npv):
                if not np.isfinite(t1):
                    return None, None, None
                u = u - t1 * r
                up += t1
                del act[l]
                u = np.delete(u, l)
                continue
            t2 = -(float(npv @ y) - b[p]) / zz
            t = min(t1, t2)
            y = y + t * z
            u = u - t * r
            up += t
            if t2 <= t1:
                act.append(p)
                u = np.append(u, up)
                break
            del act[l]
            u = np.delete(u, l)
    raise RuntimeError("dual active-set method did not terminate")


def brute_force(y0, normals, d, tol: float = 1e-12):
    """Closest feasible point by enumerating active sets of at most 3 planes."""
    y0 = np.asarray(y0, np.float64)
    N = np.asarray(normals, np.float64).reshape(-1, 3)
    b = -np.asarray(d, np.float64).reshape(-1)
    best, best_d = None, np.inf
    cands = [y0]
    for k in (1, 2, 3):
        for S in itertools.combinations(range(len(N)), k):
            NS = N[list(S)]
            if np.linalg.matrix_rank(NS, tol=1e-9) < k:
                continue
            cands.append(_project_affine(y0, NS, b[list(S)]))
    for y in cands:
        if np.all(N @ y - b >= -tol):
            dist = float(np.linalg.norm(y - y0))
            if dist < best_d:
                best, best_d = y, dist
    return best
