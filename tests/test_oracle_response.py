"""Pins of the oracle's contact response and friction (Sec. 3.3, readings
F1-F7) against physics and invariants that do not restate its formulas:

- a particle resting on a static floor inside the repulsion band settles where
  the spring force balances gravity: gap xi + delta - m g / k;
- kinetic friction decelerates a sliding particle at mu_k g (Coulomb);
- static friction with mu_s above the sliding ratio stops it at once;
- the response acts only inside the band, only along the contact normal, and
  a contact occluded by a closer one (gap difference >= delta_v) changes
  nothing;
- delta = 0 leaves the step unchanged."""
import numpy as np
import pytest

from paper_2607_26901_b300 import scenes as S

G = 9.81


def run(orc, sc, steps):
    P = orc.make_params(sc.params, capacity=0)
    x = sc.x[:, :3].astype(np.float64)
    v = sc.v[:, :3].astype(np.float64)
    rest = orc.rest_lengths(x, sc.edges)
    xs, vs = [], []
    for _ in range(steps):
        x, v, info, _ = orc.step(x, v, sc.x, sc.edges, sc.tris, rest, P)
        xs.append(x.copy())
        vs.append(v.copy())
    return np.array(xs), np.array(vs)


@pytest.mark.parametrize("delta,gap_k", [(1e-3, 4e-4), (2e-3, 1.5e-3), (5e-4, 1e-4)])
def test_rest_gap_is_force_balance(orc, delta, gap_k):
    """m g = k (delta - g_beyond_xi): the XPBD soft constraint with compliance
    1/k reaches the static equilibrium of the penalty energy."""
    m = 1e-3                                   # particle_over_floor: inverse mass 1e3
    k = m * G / gap_k
    xi = 1e-3
    sc = S.particle_over_floor(height=0.004, r=2e-3, xi=xi, iters=10, delta=delta, k_resp=k)
    xs, vs = run(orc, sc, 600)
    h = xs[:, 0, 1]
    assert h.min() >= xi - 1e-12                                  # never inside the offset
    np.testing.assert_allclose(h[-1], xi + delta - gap_k, rtol=0, atol=1e-9)
    assert abs(vs[-1, 0, 1]) < 1e-6


def test_no_response_outside_band_and_delta_zero(orc):
    base = S.particle_over_floor(height=0.012, r=1e-3, xi=1e-3, iters=10)
    resp = S.particle_over_floor(height=0.012, r=1e-3, xi=1e-3, iters=10, delta=1e-3, k_resp=50.0)
    xb, _ = run(orc, base, 2)
    xr, _ = run(orc, resp, 2)
    # the first substeps keep the particle above xi + delta: identical trajectories
    assert xb[:, 0, 1].min() > 2e-3
    np.testing.assert_array_equal(xb, xr)
    # delta = 0 with a stiffness set is still no response
    off = S.particle_over_floor(height=0.004, r=1e-3, xi=1e-3, iters=10, delta=0.0, k_resp=50.0)
    xo, _ = run(orc, off, 40)
    xb2, _ = run(orc, S.particle_over_floor(height=0.004, r=1e-3, xi=1e-3, iters=10), 40)
    np.testing.assert_array_equal(xo, xb2)


def settled_slider(orc, mu_s, mu_k, vx, steps):
    """A particle put at its rest gap with horizontal velocity vx."""
    m, delta, xi = 1e-3, 1e-3, 1e-3
    k = m * G / 4e-4
    sc = S.particle_over_floor(height=xi + delta - 4e-4, size=1.0, r=2e-3, xi=xi, iters=10, delta=delta,
                               k_resp=k, mu_s=mu_s, mu_k=mu_k, v0=(vx, 0.0, 0.0))
    return run(orc, sc, steps)


def test_kinetic_friction_decelerates_at_mu_g(orc):
    mu_k, vx = 0.2, 0.5
    dt = 1.0 / 60.0
    xs, vs = settled_slider(orc, 0.0, mu_k, vx, 12)
    vel = vs[:, 0, 0]
    assert np.all(vel > 0)
    # Coulomb: dv = -mu_k g dt per substep while sliding (normal force m g)
    np.testing.assert_allclose(np.diff(vel), -mu_k * G * dt, rtol=1e-6, atol=1e-9)


def test_static_friction_stops_sliding(orc):
    # tangential motion per substep vx dt = 1.7 mm < mu_s x (normal correction g dt^2 = 2.7 mm)
    xs, vs = settled_slider(orc, 1.0, 0.5, 0.1, 5)
    np.testing.assert_allclose(vs[:, 0, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(xs[:, 0, 0], 0.02, atol=1e-12)


def test_response_is_along_the_normal_and_occlusion_silences_farther_contacts(orc):
    rng = np.random.default_rng(3)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    x = np.zeros(3)
    y = 1e-4 * rng.normal(size=3)
    params = S.default_params(2e-3, 1e-3, delta=1e-3, k_resp=30.0, delta_v=2e-4)
    P = orc.make_params(params, capacity=0)
    w = 1e3
    g_near = 2e-4
    phi_near = g_near - n @ (y - x)
    one = np.array([[*n, 0.0]])
    y1, b1 = orc.response(y, x, x, one, [phi_near], [1], w, P)
    # along the normal only, outward, and only inside the band
    d = y1 - y
    assert np.allclose(np.cross(d, n), 0.0, atol=1e-15) and d @ n > 0 and b1 == 0
    out, _ = orc.response(y, x, x, one, [phi_near + 1e-3], [1], w, P)
    np.testing.assert_array_equal(out, y)
    # a second contact with the same normal, farther by >= delta_v: fully occluded
    two = np.array([[*n, 0.0], [*n, 0.0]])
    y2, _ = orc.response(y, x, x, two, [phi_near, phi_near + 3e-4], [1, 2], w, P)
    np.testing.assert_allclose(y2, y1, rtol=0, atol=1e-18)
    # farther by less than delta_v: partly visible, moves the vertex further out
    y3, _ = orc.response(y, x, x, two, [phi_near, phi_near + 1e-4], [1, 2], w, P)
    assert (y3 - y1) @ n >= 0.0


# the cubic smoothstep 3t^2 - 2t^3 at t = 1/4, 1/2, 3/4 (textbook values:
# S(1/2) = 1/2 and S(t) + S(1 - t) = 1)
SMOOTHSTEP_AT = {0.25: 0.15625, 0.5: 0.5, 0.75: 0.84375}


@pytest.mark.parametrize("t", sorted(SMOOTHSTEP_AT))
def test_partly_occluded_contact_acts_with_its_visibility_weight(orc, t):
    """Two contacts with the same normal, the farther one t * delta_v behind
    the nearer (F2): the nearer is fully visible and acts first (F4); the
    farther acts after it as a lone contact whose stiffness is k times its
    visibility 1 - S(t), S the cubic smoothstep (F2, F3: compliance
    1 / (k w_c))."""
    rng = np.random.default_rng(5)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    x = np.zeros(3)
    y = 1e-4 * rng.normal(size=3)
    k, dv = 3.0, 2e-4
    P = orc.make_params(S.default_params(2e-3, 1e-3, delta=1e-3, k_resp=k, delta_v=dv), capacity=0)
    w = 1e3
    phi_a = 1e-4 - n @ (y - x)
    phi_b = phi_a + t * dv
    two = np.array([[*n, 0.0], [*n, 0.0]])
    got, _ = orc.response(y, x, x, two, [phi_a, phi_b], [1, 2], w, P)
    y_a, _ = orc.response(y, x, x, two[:1], [phi_a], [1], w, P)
    Pw = orc.make_params(S.default_params(2e-3, 1e-3, delta=1e-3, k_resp=k * (1.0 - SMOOTHSTEP_AT[t]),
                                          delta_v=dv), capacity=0)
    want, _ = orc.response(y_a, x, x, two[1:], [phi_b], [2], w, Pw)
    assert (want - y_a) @ n > 1e-7          # the farther contact still acts
    np.testing.assert_allclose(got - y, want - y, rtol=1e-9, atol=0.0)
