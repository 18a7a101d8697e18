"""Halting study on the FP64 oracle (CPU only).

Why do so many vertices halt on the cloth stack?  Alg. 2 halts a vertex
(x* = x) when its last pass still meets a violated plane (Sec. 3.2); the paper
reports that consecutive halting events stayed at or below 3% of the collision
points in its particle scene (Sec. 5, halting events).  This script steps the
oracle on the test-size scenes under the readings in question and prints one
markdown table row per (scene, variant):

  - halts / violated: halted vertex-iterations over vertex-iterations with a
    violated plane at the XPBD iterate (the "collision points" that Alg. 2
    has to move);
  - consecutive: vertex-iterations that halted in the iteration before as
    well (within the substep or across the substep boundary), over the same
    denominator;
  - halts / movable: halted vertex-iterations over movable vertex-iterations.

Variants: the pass budget n_max (reading R6 runs n_max + 1 passes); the
dependence tolerance eps_dep of Alg. 1 (reading R8); the retraction after
every Alg. 1 call, where Alg. 2's listing places it, instead of once per
pass (reading R9, from the wording of Sec. 3.2); near-duplicate planes merged
(a violated plane whose normal and offset equal those of a plane visited
before it, within 1e-9 and 1e-12 m, is skipped).  The last two are compiled
copies of the oracle with the change applied (oracle/variants.py).

Usage: python -m oracle.halt_study [--steps 2]
"""
from __future__ import annotations

import argparse
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from oracle import variants  # noqa: E402
from paper_2607_26901_b300 import scenes as S  # noqa: E402

RETRACT_ONCE_PER_PASS = """        }
        /* R9: the pass result (the projected boundary position) is retracted
         * once by eps towards the build position x, or reset to x when it is
         * closer to x than eps (Sec. 3.2) */
        if (nv > 0) {
            double dn[3];
            sub3(xt, x, dn);
            double L = norm3(dn);
            if (fabs(L - P->eps) <= P->band) *band = 1;
            if (L > P->eps) {
                for (int i = 0; i < 3; ++i) xt[i] = x[i] + (L - P->eps) * dn[i] / L;
            } else {
                for (int i = 0; i < 3; ++i) xt[i] = x[i];
            }
        }
        if (pass == 0) *nviol = nv;"""
RETRACT_EACH_CALL = """            double dn[3];
            sub3(xt, x, dn);
            double L = norm3(dn);
            if (L > P->eps) {
                for (int i = 0; i < 3; ++i) xt[i] = x[i] + (L - P->eps) * dn[i] / L;
            } else {
                for (int i = 0; i < 3; ++i) xt[i] = x[i];
            }
        }
        if (pass == 0) *nviol = nv;"""
SKIP_VIOLATED = """            if (rho >= 0.0) continue;"""
SKIP_VIOLATED_OR_DUPLICATE = """            if (rho >= 0.0) continue;
            int dup = 0;
            for (long o = 0; o < s && !dup; ++o) {
                const double *q = planes4 + 4 * ord[o].idx;
                dup = fabs(q[0] - pl[0]) <= 1e-9 && fabs(q[1] - pl[1]) <= 1e-9 && fabs(q[2] - pl[2]) <= 1e-9 &&
                      fabs(q[3] - pl[3]) <= 1e-12;
            }
            if (dup) continue;"""

SCENES = {
    "stack 4x24x24 (iid velocities)": lambda: S.cloth_stack(n_side=24, layers=4, seed=2),
    "stack 4x24x24 (smooth field)": lambda: S.cloth_stack(n_side=24, layers=4, seed=2, velocity="smooth"),
    "wires 6x6x32": lambda: S.wires(n_grid=6, n_seg=32, seed=3),
    "cloth on sphere 32x32": lambda: S.config(1),
    "particles 512 onto a sphere": lambda: S.particle_cloud(512, seed=13),
}

VARIANTS = [
    ("once per pass, n_max 1 (the build's reading R9)", "once", 1, 1e-6),
    ("once per pass, n_max 2", "once", 2, 1e-6),
    ("once per pass, n_max 4", "once", 4, 1e-6),
    ("once per pass, n_max 1, eps_dep 1e-9", "once", 1, 1e-9),
    ("once per pass, n_max 1, eps_dep 1e-12", "once", 1, 1e-12),
    ("once per pass, n_max 1, duplicates merged", "merge", 1, 1e-6),
    ("after every Alg. 1 call (the listing), n_max 1", "call", 1, 1e-6),
    ("after every Alg. 1 call, n_max 2", "call", 2, 1e-6),
    ("after every Alg. 1 call, n_max 4", "call", 4, 1e-6),
]


def libraries():
    return {
        "once": O,
        "call": variants.load("retract_each_call", [(RETRACT_ONCE_PER_PASS, RETRACT_EACH_CALL)]),
        "merge": variants.load("merge_dup", [(SKIP_VIOLATED, SKIP_VIOLATED_OR_DUPLICATE)]),
    }


def run(orc, sc, n_max, eps_dep, steps):
    p = dict(sc.params)
    p["n_max"] = n_max
    P = orc.make_params(p, capacity=0, eps_dep=eps_dep)
    x3 = sc.x[:, :3].astype(np.float64)
    v3 = sc.v[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x3, sc.edges)
    ex = None
    if len(sc.links) or len(sc.tets):
        ex = orc.Extra(x3, sc.links, sc.link_compliance, sc.tets, sc.volume_compliance)
    halts = viol = consec = its = 0
    prev = np.zeros(len(x3), np.uint8)
    for _ in range(steps):
        x3, v3, info, _, hist = orc.step(x3, v3, sc.x, sc.edges, sc.tris, rest, P, extra=ex, halt_history=True)
        halts += info.halts
        viol += info.violated
        its += info.iters_run
        for h in hist:
            consec += int(np.count_nonzero(h & prev))
            prev = h
    return halts, viol, consec, its


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--scenes", nargs="*", default=None)
    a = ap.parse_args(argv)
    libs = libraries()
    print("| scene | variant | halts / violated | consecutive / violated | halts / movable |")
    print("|---|---|---:|---:|---:|")
    for sname, make in SCENES.items():
        if a.scenes and not any(s in sname for s in a.scenes):
            continue
        sc = make()
        for vname, lib, n_max, eps_dep in VARIANTS:
            t0 = time.time()
            h, v, c, its = run(libs[lib], sc, n_max, eps_dep, a.steps)
            print(f"| {sname} | {vname} | {h / max(v, 1):.3f} | {c / max(v, 1):.3f} | "
                  f"{h / max(its * sc.n_movable, 1):.3f} |", flush=True)
            print(f"  ({h} halts, {v} violated, {its} iterations, {time.time() - t0:.1f} s)", file=sys.stderr)


if __name__ == "__main__":
    main()
