"""Timing of the FP64 oracle on the host cores, for a CPU baseline of each
configuration: the 1,024-vertex cloth on the sphere in full (20 substeps
of 10 iterations), the 262,144-vertex stack and the 1.2 M-vertex wires for a
bounded number of iterations, and 16 of the 512 batched scenes for a bounded
number of substeps.  At every host core (OpenMP) and at one core (the large
scenes at one core for one iteration); microseconds per vertex-iteration of
the whole substep (region build, projection, XPBD).  Bounded samples are
labelled with what they ran; per vertex-iteration figures extrapolate.

TEST INFRASTRUCTURE ONLY: the oracle is the correctness reference; these are
the reference arm's figures, not a tuned CPU implementation.

Usage: python -m oracle.cpu_report [--iters 2] [--threads 0 1]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_2607_26901_b300 import scenes as S  # noqa: E402


def time_scene(sc, steps, iters):
    P = O.make_params(sc.params, iters=iters, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = O.rest_lengths(x, sc.edges)
    t0 = time.perf_counter()
    for _ in range(steps):
        x, v, info, _ = O.step(x, v, sc.x, sc.edges, sc.tris, rest, P)
    return time.perf_counter() - t0, sc.n_movable * steps * iters


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=2, help="iterations of the large scenes (one substep)")
    ap.add_argument("--threads", type=int, nargs="*", default=[0, 1])
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=1, help="substeps of the 16 batched scenes")
    a = ap.parse_args(argv)
    batch16 = S.batch(seed=4)[:16]
    out = {"host_cores": os.cpu_count(), "unit": "us per vertex-iteration", "cases": []}
    for th in a.threads:
        used = O.set_threads(th)
        iters = a.iters if used > 1 else 1
        cases = [("C1 cloth on sphere 32x32, 20 substeps x 10 iterations", lambda: S.config(1), 20, None)]
        if not a.skip_large:
            cases += [(f"C2 stack 4x256x256, 1 substep x {iters} iterations", lambda: S.config(2), 1, iters),
                      (f"C3 wires 128x128x64, 1 substep x {iters} iterations", lambda: S.config(3), 1, iters)]
        for name, make, steps, it in cases:
            sc = make()
            it = sc.params["iters"] if it is None else it
            secs, units = time_scene(sc, steps, it)
            out["cases"].append({"case": name, "threads": used, "seconds": round(secs, 2),
                                 "us_per_vertex_iter": round(1e6 * secs / units, 3)})
            print(json.dumps(out["cases"][-1]), flush=True)
        secs = units = 0
        for sc in batch16:
            s, u = time_scene(sc, a.batch_steps, sc.params["iters"])
            secs += s
            units += u
        out["cases"].append({"case": f"C4 16 of the 512 batched scenes, {a.batch_steps} substeps x 10 iterations",
                             "threads": used, "seconds": round(secs, 2),
                             "us_per_vertex_iter": round(1e6 * secs / units, 3)})
        print(json.dumps(out["cases"][-1]), flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
