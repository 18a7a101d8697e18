"""Mutation checks of the oracle beyond Alg. 2: a plausible mistake planted
in a compiled copy of the oracle (CPU only, oracle/variants.py) must make at
least one of the pins of the part it touches fail.

The parts and what each mutation plants:
- candidate predicate (Sec. 4.1, Alg. 3 exclusions): the pad dropped from the
  boxes, a shared-vertex or own-triangle exclusion dropped, the sweep's lower
  bound without the largest item extent;
- closest points (the Voronoi-region and clamped-segment rules named in the
  oracle): a wrong edge-region parameter, a sign in the segment parameter, an
  unclamped point-segment parameter;
- planes of a pair (Alg. 3, Eq. 1-3, readings R1-R4): the gap without xi, the
  acceptance threshold r instead of 2r, the two sides' shares swapped, side B
  given +n, the unweighted generalized inverse mass, the edge-edge closest
  point with its barycentric weights swapped;
- Alg. 1 and the overflow rule (R7, R16): the first stored offset negated, a
  stored line's offset with the wrong sign, a step along the first stored
  direction instead of the last, the overflow bound taken as the largest
  offset;
- the step (Alg. 4, R12-R15, X2): gravity dropped from the prediction, the
  XPBD multiplier's sign flipped, the iterate not restarted from the
  prediction, the regions built at the prediction, the max-step clamp
  dropped, the velocity update multiplied by dt, the first colour starting at
  1, the volume gradient of one corner negated;
- mixed scenes (X1, X2, X4, X5): volume-interior vertices colliding,
  point-edge pairs with triangle edges, the links' compliance or the volume
  compliance ignored;
- the contact response (Sec. 3.3, F1-F5): the gap taken at the build position,
  static friction against mu_k, a wrong smoothstep, the compliance without the
  visibility weight.

Every pin is first run on the oracle itself through the same harness, so a
pin that cannot run (wrong arguments) fails there instead of counting as a
catch; only an AssertionError counts as a catch.
"""
import itertools

import pytest

from oracle import variants
from tests import test_oracle_broad as TB
from tests import test_oracle_geometry as TG
from tests import test_oracle_mixed as TM
from tests import test_oracle_projection as TP
from tests import test_oracle_response as TR
from tests import test_oracle_step as TS


def _calls(fn):
    """fn's parameter sets from its parametrize marks (cartesian product)."""
    axes = []
    for mark in getattr(fn, "pytestmark", []):
        if mark.name != "parametrize":
            continue
        names = mark.args[0]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        sets = []
        for val in mark.args[1]:
            vals = val.values if hasattr(val, "values") else ((val,) if len(names) == 1 else tuple(val))
            sets.append(dict(zip(names, vals)))
        axes.append(sets)
    if not axes:
        return [{}]
    return [dict(kv for d in combo for kv in d.items()) for combo in itertools.product(*axes)]


PINS = {
    "candidates": [TB.test_candidates_match_definition, TB.test_candidates_superset_of_close_pairs,
                   TM.test_point_edge_candidates_match_definition, TM.test_no_point_edge_pairs_with_triangle_edges],
    "geometry": [TG.test_closest_point_triangle_regions, TG.test_closest_point_triangle_vs_sampling,
                 TG.test_closest_segments_parallel_and_crossing, TG.test_closest_segments_vs_sampling,
                 TM.test_closest_point_segment_brute_force, TG.test_distance_helpers_and_intersections],
    "planes": [TP.test_worked_examples_golden, TP.test_large_triangle_caught_by_closest_point,
               TP.test_regions_contain_current_configuration, TM.test_point_edge_plane_worked_example],
    "projection": [TP.test_alg1_equals_least_norm_projection, TP.test_alg1_skips_dependent_and_duplicate_planes,
                   TP.test_worked_examples_golden, TP.test_alg2_single_plane_closed_form,
                   TP.test_overflow_rule_is_safe, TP.test_alg2_result_is_feasible_or_halted],
    "step": [TS.test_free_fall_closed_form, TS.test_early_exit_when_converged, TS.test_particle_rests_on_floor,
             TS.test_two_particles_head_on, TS.test_edge_colours_valid_and_first_fit,
             TS.test_xpbd_sweep_satisfies_last_colour, TM.test_volume_constraint_is_a_linearised_projection,
             TM.test_link_compliance_limits, TS.test_card_stack_stays_static,
             TS.test_trajectory_is_penetration_free],
    "mixed": [TM.test_volume_interior_takes_no_part_in_collision, TM.test_no_point_edge_pairs_with_triangle_edges,
              TM.test_point_edge_candidates_match_definition, TM.test_point_edge_plane_worked_example,
              TM.test_link_compliance_limits, TM.test_volume_constraint_is_a_linearised_projection,
              TM.test_volume_compliance_halves_the_first_order_correction],
    "response": [TR.test_rest_gap_is_force_balance, TR.test_no_response_outside_band_and_delta_zero,
                 TR.test_kinetic_friction_decelerates_at_mu_g, TR.test_static_friction_stops_sliding,
                 TR.test_response_is_along_the_normal_and_occlusion_silences_farther_contacts,
                 TR.test_partly_occluded_contact_acts_with_its_visibility_weight],
}

MUTATIONS = {
    # candidate predicate
    "boxes without the pad": ("candidates", [
        ("volatile float lo = mn - pad, hi = mx + pad;", "volatile float lo = mn, hi = mx;")]),
    "vertex-face pair with the triangle's own vertex": ("candidates", [
        ("    if (v == T[0] || v == T[1] || v == T[2]) return 0;\n", "")]),
    "edge-edge pair sharing a vertex": ("candidates", [
        ("    if (A[0] == B[0] || A[0] == B[1] || A[1] == B[0] || A[1] == B[1]) return 0;\n", "")]),
    "sweep from the query's lower bound": ("candidates", [
        ("double from = (double)q.lo[0] - maxext;", "double from = (double)q.lo[0];")]),
    # closest points
    "triangle edge bc parameter": ("geometry", [
        ("double s = (d4 - d3) / ((d4 - d3) + (d5 - d6));", "double s = (d4 - d3) / ((d4 - d3) - (d5 - d6));")]),
    "segment parameter sign": ("geometry", [
        ("            t = (b * s + f) / e;", "            t = (b * s - f) / e;")]),
    "point-segment parameter unclamped": ("geometry", [
        ("return l2 > 0.0 ? clamp01(dot3(ap, ab) / l2) : 0.0;", "return l2 > 0.0 ? dot3(ap, ab) / l2 : 0.0;")]),
    # planes of a pair
    "gap without xi": ("planes", [("    double phi = dist - P->xi;", "    double phi = dist;")]),
    "acceptance below r": ("planes", [("if (!(phi < 2.0 * P->r)) return 0;", "if (!(phi < P->r)) return 0;")]),
    "shares swapped": ("planes", [
        ("if (w[va[i]] > 0) plv_push(out, va[i], n, (wa / W) * phi, phi, key);",
         "if (w[va[i]] > 0) plv_push(out, va[i], n, (wb / W) * phi, phi, key);"),
        ("if (w[vb[i]] > 0) plv_push(out, vb[i], mn, (wb / W) * phi, phi, key);",
         "if (w[vb[i]] > 0) plv_push(out, vb[i], mn, (wa / W) * phi, phi, key);")]),
    "side B with +n": ("planes", [
        ("if (w[vb[i]] > 0) plv_push(out, vb[i], mn, (wb / W) * phi, phi, key);",
         "if (w[vb[i]] > 0) plv_push(out, vb[i], n, (wb / W) * phi, phi, key);")]),
    "unweighted inverse mass": ("planes", [
        ("for (int i = 0; i < nb; ++i) wb += bb[i] * w[vb[i]];", "for (int i = 0; i < nb; ++i) wb += w[vb[i]];")]),
    "edge-edge point with swapped weights": ("planes", [
        ("pa[i] = (1 - s) * x3[3 * A[0] + i] + s * x3[3 * A[1] + i];",
         "pa[i] = s * x3[3 * A[0] + i] + (1 - s) * x3[3 * A[1] + i];")]),
    # Alg. 1 and the overflow rule
    "Alg. 1 first offset negated": ("projection", [("        S->B[0] = b;\n", "        S->B[0] = -b;\n")]),
    "Alg. 1 offset of a stored line with the wrong sign": ("projection", [
        ("double alpha_w = bj - b0 - dot3(dnj, wv);", "double alpha_w = bj + b0 - dot3(dnj, wv);")]),
    "Alg. 1 step along the first stored direction": ("projection", [
        ("u[i] = xt[i] + (alpha_u / beta_u) * S->V[m - 1][i];", "u[i] = xt[i] + (alpha_u / beta_u) * S->V[0][i];")]),
    "overflow bound is the largest offset": ("projection", [
        ("if (R->p[k].d < m) m = R->p[k].d;", "if (!(R->p[k].d < m) || m == INFINITY) m = R->p[k].d;")]),
    # the step
    "prediction without gravity": ("step", [
        ("x3[3 * i + a] + dt * v3[3 * i + a] + dt * dt * P->g[a]", "x3[3 * i + a] + dt * v3[3 * i + a]")]),
    "XPBD multiplier sign": ("step", [
        ("double dl = (-C - at * lambda[e]) / wsum;", "double dl = (C - at * lambda[e]) / wsum;")]),
    "iterate not restarted from the prediction": ("step", [
        ("        memcpy(xs, xt, N3);\n", "        memcpy(xs, it == 0 ? xt : xc, N3);\n")]),
    "regions built at the prediction": ("step", [
        ("orc_regions *R = build_regions(xc, w, &t, P);", "orc_regions *R = build_regions(xt, w, &t, P);")]),
    "no max-step clamp": ("step", [("            clamp_len(x, y, P->r);   /* max-step clamp", "            /* max-step clamp")]),
    "velocity times dt": ("step", [
        ("v3[3 * i + a] = (xc[3 * i + a] - xn[3 * i + a]) / dt;", "v3[3 * i + a] = (xc[3 * i + a] - xn[3 * i + a]) * dt;")]),
    "colours from 1": ("step", [
        ("        u64 m = used[a] | used[b];\n        int c = 0;", "        u64 m = used[a] | used[b];\n        int c = 1;")]),
    "volume gradient of corner 0 negated": ("step", [
        ("for (int k = 0; k < 3; ++k) g[0][k] = -(g[1][k] + g[2][k] + g[3][k]);",
         "for (int k = 0; k < 3; ++k) g[0][k] = g[1][k] + g[2][k] + g[3][k];")]),
    # mixed scenes
    "interior volume vertices collide (X5)": ("mixed", [
        ("t->collides[i] = used[i] != 2;", "t->collides[i] = 1;")]),
    "point-edge pairs with triangle edges (X4)": ("mixed", [("    if (!t->free_edge[e]) return 0;\n", "")]),
    "links take the edges' compliance (X1)": ("mixed", [
        ("dcomp[ne + l] = ex->link_compliance[l];", "dcomp[ne + l] = P->compliance;")]),
    "volume compliance ignored (X2)": ("mixed", [
        ("double atv = ex ? ex->volume_compliance / (dt * dt) : 0.0;", "double atv = 0.0;")]),
    # the contact response
    "response gap at the build position": ("response", [
        ("double C = P->delta - (phi[all[a].k] + dot3(n, d));", "double C = P->delta - phi[all[a].k];")]),
    "static friction against mu_k": ("response", [
        ("double f = (tl < P->mu_s * depth[a])", "double f = (tl < P->mu_k * depth[a])")]),
    "smoothstep 3t^2 - t^3": ("response", [("return t * t * (3.0 - 2.0 * t);", "return t * t * (3.0 - t);")]),
    "compliance without the visibility weight": ("response", [
        ("double at = 1.0 / (P->k_resp * wt[a] * P->dt * P->dt);", "double at = 1.0 / (P->k_resp * P->dt * P->dt);")]),
}


def _run_part(orc, part, stop_at_first_catch):
    caught = []
    for fn in PINS[part]:
        for kw in _calls(fn):
            try:
                fn(orc, **kw)
            except AssertionError:
                caught.append(fn.__name__)
                if stop_at_first_catch:
                    return caught
                break
    return caught


@pytest.mark.parametrize("part", sorted(PINS))
def test_pins_pass_on_the_oracle(orc, part):
    assert _run_part(orc, part, stop_at_first_catch=False) == []


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_pins_catch_mutation(mutation):
    part, repl = MUTATIONS[mutation]
    bad = variants.load("mut_" + "".join(ch if ch.isalnum() else "_" for ch in mutation), repl)
    assert _run_part(bad, part, stop_at_first_catch=True), f"no pin of {part!r} catches {mutation!r}"
