"""How many of a vertex's planes are copies (CPU only, FP64 oracle).

One geometric contact (two vertices close together, a vertex near an edge)
is reached through every vertex-face and edge-edge pair that shares its
closest features, and each of those pairs stores a plane for it (Alg. 3).
This script builds the regions of the cloth stack with the oracle at the
start and after each of a few substeps and counts, per receiving vertex:

  - stored: the planes Alg. 3 stores;
  - distinct (bits): planes that differ in some bit of (n, d);
  - distinct (1e-9): planes that differ by more than 1e-9 in a normal
    component or 1e-12 m in the offset (rounded to those grids).

The ratio stored / distinct is the factor by which an emission that stores
each contact once would shorten the plane lists.

TEST INFRASTRUCTURE ONLY: a study of the method's inputs on the oracle.

Usage: python -m oracle.duplicate_study [--side 48] [--layers 4] [--steps 3] [--iters 3]
"""
from __future__ import annotations

import argparse
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_2607_26901_b300 import scenes as S  # noqa: E402


def count_distinct(offs, planes, tol_n=1e-9, tol_d=1e-12):
    """(stored, distinct by bits, distinct on the rounding grid) over all vertices."""
    bits = near = 0
    for i in range(len(offs) - 1):
        p = planes[offs[i]:offs[i + 1]]
        if len(p) == 0:
            continue
        bits += len(np.unique(np.ascontiguousarray(p).view(np.uint64).reshape(-1, 4), axis=0))
        grid = np.column_stack([np.round(p[:, :3] / tol_n), np.round(p[:, 3] / tol_d)]).astype(np.int64)
        near += len(np.unique(grid, axis=0))
    return int(offs[-1]), bits, near


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=48)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--iters", type=int, default=3)
    a = ap.parse_args(argv)
    sc = S.cloth_stack(n_side=a.side, layers=a.layers, iters=a.iters)
    P = O.make_params(sc.params, iters=a.iters, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = O.rest_lengths(x, sc.edges)
    print(f"| stack {a.layers}x{a.side}x{a.side} | planes per vertex | stored / distinct (bits) "
          f"| stored / distinct (1e-9) | most planes of a vertex |")
    print("|---|---:|---:|---:|---:|")
    for step in range(a.steps + 1):
        x4 = np.concatenate([x.astype(np.float32), sc.x[:, 3:4]], axis=1)
        R = O.build_regions(x, x4, sc.edges, sc.tris, P)
        stored, bits, near = count_distinct(R["offs"], R["planes"])
        cnt = np.diff(R["offs"])
        print(f"| after {step} substeps | {stored / max((cnt > 0).sum(), 1):.0f} | {stored / max(bits, 1):.2f} "
              f"| {stored / max(near, 1):.2f} | {cnt.max()} |", flush=True)
        if step < a.steps:
            x, v, _, _ = O.step(x, v, x4, sc.edges, sc.tris, rest, P)


if __name__ == "__main__":
    main()
