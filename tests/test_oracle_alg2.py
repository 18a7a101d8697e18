"""Pins of projectOntoConvexRegion (Alg. 2) beyond one plane, and the checks
that those pins catch plausible mistakes.

- Hand-derived multi-plane cases (tests/golden/alg2_multiplane.json): the
  corner point of Alg. 1 followed by one retraction per pass, the visiting
  order (ascending rho at the input), the n_max + 1 pass budget, the halt when
  a fourth violated plane meets three stored lines, and the return of an
  unviolated candidate unchanged.
- Three mutually perpendicular planes: the result is the corner point of
  Alg. 1 (the exact closest point of the region, Sec. 3.2) moved by at most a
  few retractions of eps, inside every plane.
- Mutations: each plausible mistake in a copy of the oracle's Alg. 2 / Alg. 1
  (descending sort, a retraction after every Alg. 1 call, n_max passes, no
  halt fallback, retraction measured from the pass input, the sort key taken
  at the build position, Alg. 1's first dependence measure on the first
  stored line) makes at least one pin fail.
"""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import qp
from oracle import variants
from paper_2607_26901_b300 import scenes as S

GOLDEN = Path(__file__).resolve().parent / "golden"


def _project_one(orc, planes, candidate, n_max, eps=1e-6, eps_dep=1e-6):
    p = S.default_params(0.005, 0.001)
    p["n_max"], p["eps"], p["eps_dep"] = n_max, eps, eps_dep
    P = orc.make_params(p, capacity=0)
    planes = np.asarray(planes, np.float64).reshape(-1, 4)
    out, halt, band, nviol = orc.project(np.zeros((1, 3)), np.asarray([candidate], np.float64), np.ones(1),
                                         np.array([0, len(planes)]), planes,
                                         np.arange(1, len(planes) + 1, dtype=np.uint64), None, P)
    return out[0], int(halt[0]), int(nviol[0])


def check_golden_multiplane(orc):
    cases = json.loads((GOLDEN / "alg2_multiplane.json").read_text())["cases"]
    for c in cases:
        got, halt, nviol = _project_one(orc, c["planes"], c["candidate"], c["n_max"], c["eps"], c["eps_dep"])
        assert halt == c["halt"], c["name"]
        assert nviol == c["nviol"], c["name"]
        np.testing.assert_allclose(got, c["projected"], rtol=0, atol=1e-15, err_msg=c["name"])


CORNER_D = (0.002, 0.0015, 0.001)
CORNER_CANDIDATES = [(-0.003, -0.004, -0.005), (-0.005, -0.004, -0.003), (-0.006, -0.0025, -0.004),
                     (-0.0041, -0.0052, -0.0033)]
# three planes at oblique angles, and candidates x' = vertex - N^T lambda
# (lambda > 0: inside the normal cone of the vertex, whose closest point
# in the region is the vertex itself)
SKEW_N = np.array([[1.0, 0.0, 0.0], [0.6, 0.8, 0.0], [0.0, 0.6, 0.8]])
SKEW_D = np.array([0.002, 0.0015, 0.001])
SKEW_LAMBDA = [(0.002, 0.001, 0.0015), (0.001, 0.003, 0.001), (0.0005, 0.0005, 0.004)]


def check_three_plane_corner(orc):
    """A candidate pushed into the corner of three planes: with enough passes
    the result is the corner point of Alg. 1 (the intersection of the three
    planes, which is here the exact closest point of the region), moved by the
    retractions only, each of length eps (at most one per Alg. 1 call and
    pass: 3 + 3 here), and every plane holds with rho in [0, 6 eps].  First
    x >= -a1, y >= -a2, z >= -a3, then three oblique planes."""
    eps = 1e-6
    planes = np.array([[1, 0, 0, CORNER_D[0]], [0, 1, 0, CORNER_D[1]], [0, 0, 1, CORNER_D[2]]], np.float64)
    cases = [(planes, np.array(c), -np.array(CORNER_D)) for c in CORNER_CANDIDATES]
    vert = -np.array([SKEW_D[0], (SKEW_D[1] - 0.6 * SKEW_D[0]) / 0.8, 0.0])
    vert[2] = (-SKEW_D[2] - 0.6 * vert[1]) / 0.8
    skew = np.c_[SKEW_N, SKEW_D]
    cases += [(skew, vert - SKEW_N.T @ np.array(lam), vert) for lam in SKEW_LAMBDA]
    for pl, cand, corner in cases:
        np.testing.assert_allclose(pl[:, :3] @ corner + pl[:, 3], 0.0, atol=1e-18)
        ref, _, _ = qp.project(cand, pl[:, :3], pl[:, 3])
        np.testing.assert_allclose(ref, corner, atol=1e-17)
        got, halt, nviol = _project_one(orc, pl, cand, n_max=3, eps=eps)
        assert halt == 0 and nviol == 3
        assert np.abs(got - corner).max() <= 6 * eps
        rho = pl[:, :3] @ got + pl[:, 3]
        assert np.all(rho >= 0) and np.all(rho <= 6 * eps)


def _pins():
    from tests import test_oracle_projection as T
    return [
        ("golden multi-plane cases", check_golden_multiplane),
        ("three-plane corner", check_three_plane_corner),
        ("single violated plane, closed form", T.test_alg2_single_plane_closed_form),
        ("worked examples", T.test_worked_examples_golden),
    ]


def test_alg2_golden_multiplane(orc):
    check_golden_multiplane(orc)


def test_alg2_three_plane_corner(orc):
    check_three_plane_corner(orc)


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

MUTATIONS = {
    "sort descending": [("    if (p->rho < q->rho) return -1;\n    if (p->rho > q->rho) return 1;",
                         "    if (p->rho > q->rho) return -1;\n    if (p->rho < q->rho) return 1;")],
    "retraction after every Alg. 1 call": [(RETRACT_ONCE_PER_PASS, RETRACT_EACH_CALL)],
    "n_max passes": [("pass < P->n_max + 1; ++pass", "pass < P->n_max; ++pass")],
    "no halt fallback": [("    if (halted) { xp[0] = x[0]; xp[1] = x[1]; xp[2] = x[2]; }", "")],
    "retraction from the pass input": [(RETRACT_ONCE_PER_PASS, RETRACT_ONCE_PER_PASS.replace(
        "sub3(xt, x, dn);", "sub3(xt, x0, dn);").replace("xt[i] = x[i] + (L", "xt[i] = x0[i] + (L").replace(
        "for (int i = 0; i < 3; ++i) xt[i] = x[i];", "for (int i = 0; i < 3; ++i) xt[i] = x0[i];"))],
    "sort key at the build position": [("ord[k].rho = dot3(y, planes4 + 4 * k) + planes4[4 * k + 3];",
                                        "ord[k].rho = planes4[4 * k + 3];")],
    "Alg. 1 beta_u on the first line": [("double beta_u = dot3(dn, S->V[m - 1]);",
                                         "double beta_u = dot3(dn, S->V[0]);")],
}


def test_pins_pass_on_the_oracle(orc):
    for name, pin in _pins():
        pin(orc)


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_pins_catch_mutation(mutation):
    """The mistake is planted in a compiled copy of the oracle (CPU only);
    at least one Alg. 2 pin must fail on it."""
    bad = variants.load("mut_" + "".join(ch if ch.isalnum() else "_" for ch in mutation), MUTATIONS[mutation])
    caught = []
    for name, pin in _pins():
        try:
            pin(bad)
        except AssertionError:
            caught.append(name)
    assert caught, f"no pin catches the mutation {mutation!r}"


def _without_exact_copies(R):
    """The regions with every plane that repeats an earlier plane of the same
    vertex bit for bit (n and d) removed; each list keeps its key order."""
    offs, planes, keys = R["offs"], R["planes"], R["key"]
    keep = np.zeros(len(planes), bool)
    for v in range(len(offs) - 1):
        a, b = offs[v], offs[v + 1]
        if a < b:
            bits = np.ascontiguousarray(planes[a:b]).view(np.uint64).reshape(-1, 4)
            keep[a + np.unique(bits, axis=0, return_index=True)[1]] = True
    vert = np.repeat(np.arange(len(offs) - 1), np.diff(offs))
    noffs = np.concatenate([[0], np.cumsum(np.bincount(vert[keep], minlength=len(offs) - 1))])
    return noffs, planes[keep], keys[keep]


@pytest.mark.parametrize("make,step_first", [
    (lambda: S.cloth_stack(n_side=12, layers=4, speed=0.5, seed=5, iters=3), True),
    (lambda: S.card_stack(n_cards=8), False),
])
def test_alg2_unchanged_by_exact_copies_of_planes(orc, make, step_first):
    """A plane that repeats one of the vertex's planes bit for bit (one
    contact reached through several pairs) changes nothing in Alg. 2: the copy
    has the same rho as the original at every iterate, so it is violated
    exactly when the original is, and once Alg. 1 holds the original its copy
    is dependent (beta = 0).  Results and halts are bitwise those of the lists
    without copies; only the count of violated planes differs."""
    sc = make()
    P = orc.make_params(sc.params, capacity=0)
    x3 = sc.x[:, :3].astype(np.float64)
    if step_first:                       # leave the exactly parallel start
        rest = orc.rest_lengths(x3, sc.edges)
        x3, _, _, _ = orc.step(x3, sc.v[:, :3].astype(np.float64), sc.x, sc.edges, sc.tris, rest, P)
    x4 = sc.x.copy()
    x4[:, :3] = x3
    R = orc.build_regions(x3, x4, sc.edges, sc.tris, P)
    noffs, nplanes, nkeys = _without_exact_copies(R)
    assert len(nplanes) < len(R["planes"])
    for seed in range(3):
        xp = x3 + np.random.default_rng(seed).normal(scale=2e-3, size=x3.shape)
        a = orc.project(x3, xp, sc.x[:, 3], R["offs"], R["planes"], R["key"], None, P)
        b = orc.project(x3, xp, sc.x[:, 3], noffs, nplanes, nkeys, None, P)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        assert a[1].sum() > 0 or not step_first
