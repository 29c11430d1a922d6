"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one stage by a closed form, an invariant, a textbook special
case or brute force, so that a dropped term, a wrong sign or a transposed
operand anywhere in the oracle fails at least one of them:

  free fall            discrete closed form of semi-implicit Euler
  pendulum             discrete frequency (2/dt) asin(w dt / 2) of semi-implicit Euler
  two-link arm         textbook closed forms of M(q) and the gravity torques
  ABA == CRBA          Featherstone's two algorithms agree on random trees
  implicit PD          one-step closed form of the stable-PD recurrence
  energy drift         O(dt) drift of an undamped chain (ratio ~2 under dt halving)
  elastic pair         1-D elastic collision closed form, momentum conservation
  narrowphase          sphere closed forms, box-plane vertex enumeration, box-box
                       15-axis SAT restated in numpy + sampled distances
  broadphase           all-pairs AABB overlap restated in numpy
  colouring            greedy first fit in unit order checked pairwise, serial
                       overflow colour past 64 units on one node
  PGS                  LCP solution by active-set enumeration; static friction
                       sum = m g dt; incline stick / slide a = g (sin - mu cos)
  sleep                exact sleep step; wake step predicted from free fall; the
                       counter restarts after a fast step (apex of a vertical throw)
  orientation          spinning body: q_n = (cos n b, 0, 0, sin n b), b = atan(w dt / 2)
  joint limit          reached exactly in the crossing step, never passed; a violated
                       limit recovers the fraction beta (Baumgarte) in one step
  training targets     a new resting contact's target is 1 unit of m_eff,n |g| dt
  friction warm start  static friction on an incline is carried to the next step
  warm-start match     a contact moving beyond the match distance starts from zero
  covariance           a rotated frictionless scene gives the rotated result
  residual             sweeps to the relative 1e-6 target do not depend on the mass scale
  MLP                  GELU values from math.erf; gradients by finite differences;
                       warm start from the output limited to +-10, non-finite -> prior frame;
                       contact features of a resting sphere (2m/7 rolling mass, m g dt prior)
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import scenegen as sg

DT = 1.0 / 120.0
G = 9.81


def qrot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def params(**kw):
    p = sg.SimParams()
    p.sleep_enabled = 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------------------- integration
def test_free_fall_closed_form():
    x0, v0 = np.array([0.5, -0.2, 10.0]), np.array([0.3, 0.1, 1.0])
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.1, mass=1.0, pos=x0, vel=v0)], plane=False)])
    o = O.Oracle(b, params())
    for n in range(1, 101):
        o.step(1)
        s = o.get_state()
        z = x0[2] + n * DT * v0[2] - G * DT * DT * n * (n + 1) / 2
        assert abs(s["obj_pos"][0, 2] - z) < 1e-12
        assert abs(s["obj_vel"][0, 2] - (v0[2] - n * G * DT)) < 1e-12
        assert np.allclose(s["obj_pos"][0, :2], x0[:2] + n * DT * v0[:2], atol=1e-12)


def _pendulum(d=0.3, m=1.3, hw=0.02, theta0=0.01, dt=DT):
    j = dict(parent=-1, type=0, axis=(0, 1, 0), com=(0, 0, -d), half=(hw, hw, d), mass=m, q0=theta0)
    return sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 5), joints=[j])], plane=False)])


@pytest.mark.parametrize("dt", [1.0 / 30.0, 1.0 / 120.0])
def test_pendulum_discrete_frequency(dt):
    d, m, hw, th0 = 0.3, 1.3, 0.02, 0.01
    o = O.Oracle(_pendulum(d, m, hw, th0), params(dt=dt))
    steps = int(round(20.0 / dt))
    q = np.zeros(steps + 1)
    q[0] = th0
    for n in range(steps):
        o.step(1)
        q[n + 1] = o.get_state()["joint_q"][0]
    I_pivot = m * (hw * hw + d * d) / 3 + m * d * d
    w = math.sqrt(m * G * d / I_pivot)
    w_disc = 2 / dt * math.asin(w * dt / 2)
    cross = [k + q[k] / (q[k] - q[k + 1]) for k in range(steps) if q[k] > 0 >= q[k + 1]]
    T_meas = (cross[-1] - cross[0]) / (len(cross) - 1) * dt
    assert len(cross) > 10
    assert abs(T_meas - 2 * math.pi / w_disc) / T_meas < 1e-4
    if dt > 1.0 / 60.0:
        # the continuous-time period differs by far more than the tolerance at this dt
        assert abs(2 * math.pi / w - 2 * math.pi / w_disc) / T_meas > 5e-4


# ----------------------------------------------------------------------------- articulated dynamics
def _two_link(q1, q2, l1=0.5, l2=0.4, m1=2.0, m2=1.5, w=0.03):
    js = [dict(parent=-1, type=0, axis=(0, 1, 0), com=(l1 / 2, 0, 0), half=(l1 / 2, w, w), mass=m1, q0=q1),
          dict(parent=0, type=0, axis=(0, 1, 0), origin_pos=(l1, 0, 0), com=(l2 / 2, 0, 0), half=(l2 / 2, w, w),
               mass=m2, q0=q2)]
    return sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 2), joints=js)], plane=False)])


def test_two_link_mass_matrix_and_gravity_closed_form():
    l1, l2, m1, m2, w = 0.5, 0.4, 2.0, 1.5, 0.03
    for q1, q2 in ((0.3, -0.7), (1.1, 0.4), (-2.0, 2.5)):
        o = O.Oracle(_two_link(q1, q2, l1, l2, m1, m2, w), params())
        _, bias, M = o.dynamics_check(0, 0, np.zeros(2), np.zeros(2))
        lc1, lc2 = l1 / 2, l2 / 2
        I1 = m1 * ((l1 / 2) ** 2 + w * w) / 3
        I2 = m2 * ((l2 / 2) ** 2 + w * w) / 3
        M11 = m1 * lc1 ** 2 + I1 + m2 * (l1 ** 2 + lc2 ** 2 + 2 * l1 * lc2 * math.cos(q2)) + I2
        M12 = m2 * (lc2 ** 2 + l1 * lc2 * math.cos(q2)) + I2
        M22 = m2 * lc2 ** 2 + I2
        assert np.allclose(M, [[M11, M12], [M12, M22]], atol=1e-12)
        # rotation about +y takes +x towards -z: z_com1 = -lc1 sin q1, ...
        G1 = -G * (m1 * lc1 + m2 * l1) * math.cos(q1) - m2 * G * lc2 * math.cos(q1 + q2)
        G2 = -m2 * G * lc2 * math.cos(q1 + q2)
        assert np.allclose(bias, [G1, G2], atol=1e-12)


def _random_tree(rng, n):
    js = []
    for i in range(n):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        h = rng.uniform(0.02, 0.2, 3)
        js.append(dict(parent=int(rng.integers(-1, i)) if i else -1, type=int(rng.integers(0, 2)), axis=ax,
                       origin_pos=rng.uniform(-0.3, 0.3, 3), origin_quat=rand_quat(rng),
                       com=rng.uniform(-0.2, 0.2, 3), half=h, mass=rng.uniform(0.2, 3.0),
                       q0=rng.uniform(-1, 1), qd0=rng.uniform(-2, 2)))
    return js


def test_aba_equals_crba_dense_solve():
    rng = np.random.default_rng(1)
    envs = [dict(arts=[dict(base_pos=rng.uniform(-1, 1, 3), base_quat=rand_quat(rng),
                            joints=_random_tree(rng, n))], plane=False) for n in range(1, 10) for _ in range(3)]
    b = sg.custom_batch(envs)
    o = O.Oracle(b, params())
    for e, env in enumerate(envs):
        n = len(env["arts"][0]["joints"])
        tau = rng.normal(size=n) * 5
        qdd, bias, M = o.dynamics_check(e, 0, tau, np.zeros(n))
        assert np.allclose(M, M.T, atol=1e-12)
        assert np.all(np.linalg.eigvalsh(M) > 0)
        ref = np.linalg.solve(M, tau - bias)
        assert np.allclose(qdd, ref, rtol=1e-10, atol=1e-10)
        _, tau_back, _ = o.dynamics_check(e, 0, tau, qdd)
        assert np.allclose(tau_back, tau, rtol=1e-10, atol=1e-10)


def test_joint_space_inverse_inverts_the_mass_matrix():
    """The joint-space inverse M^-1 that the contact and limit rows use (a dense
    Cholesky inverse of the mass matrix) satisfies M M^-1 = M^-1 M = I, for random
    trees of 1 to 9 revolute and prismatic joints."""
    rng = np.random.default_rng(4)
    envs = [dict(arts=[dict(base_pos=rng.uniform(-1, 1, 3), base_quat=rand_quat(rng),
                            joints=_random_tree(rng, n))], plane=False) for n in range(2, 10) for _ in range(2)]
    b = sg.custom_batch(envs)
    o = O.Oracle(b, params())
    o.step(1)
    for e, env in enumerate(envs):
        a = o.articulation(e, 0)
        n = len(env["arts"][0]["joints"])
        assert a["n"] == n
        assert np.allclose(a["M"] @ a["Minv"], np.eye(n), atol=1e-9)
        assert np.allclose(a["Minv"] @ a["M"], np.eye(n), atol=1e-9)


def test_prismatic_slider_free_fall_along_its_axis():
    """One prismatic joint on a fixed, rotated base (joint frame rotated too), no
    motor, no limit: the joint accelerates at g . a, a the axis in world axes, and
    the link's centre of mass moves along a, whatever the link's mass and inertia;
    semi-implicit Euler gives qd_n = (g . a) dt n, q_n = (g . a) dt^2 n (n + 1) / 2."""
    rng = np.random.default_rng(5)
    qb, qo = rand_quat(rng), rand_quat(rng)
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    j = dict(parent=-1, type=1, axis=tuple(axis), origin_pos=(0.1, -0.2, 0.3), origin_quat=tuple(qo),
             com=(0.05, 0.02, -0.1), half=(0.1, 0.05, 0.2), mass=2.5)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 1.0), base_quat=tuple(qb), joints=[j])], plane=False)])
    o = O.Oracle(b, params())
    a_world = qrot(qb) @ qrot(qo) @ axis
    acc = -G * a_world[2]
    assert abs(acc) > 1.0
    o.step(1)
    c1 = o.articulation(0, 0)["com"][0].copy()
    q1 = acc * DT * DT
    for n in range(2, 31):
        o.step(1)
        st = o.get_state()
        assert abs(st["joint_qd"][0] - acc * DT * n) < 1e-12, n
        qn = acc * DT * DT * n * (n + 1) / 2
        assert abs(st["joint_q"][0] - qn) < 1e-12, n
    c = o.articulation(0, 0)["com"][0]  # the link's pose at q_30, measured from q_1's
    assert np.allclose(c - c1, a_world * (acc * DT * DT * 30 * 31 / 2 - q1), rtol=0, atol=1e-12)


def test_slider_pressed_into_the_floor_gets_no_normal_impulse():
    """A link on a horizontal prismatic joint, its box pressed 1 mm into the floor: no
    joint motion changes the contacts' normal velocity (the joint axis is
    horizontal), so each normal row's inverse effective mass is zero -- a degenerate
    row, which gets no impulse -- and with no normal impulse the friction bound is
    zero too.  The slider keeps its rate exactly (gravity has no component along its
    axis) and the state stays finite."""
    qd0 = 0.5
    j = dict(parent=-1, type=1, axis=(1, 0, 0), origin_pos=(0, 0, 0), origin_quat=(1, 0, 0, 0),
             com=(0, 0, 0), half=(0.1, 0.05, 0.05), mass=2.0, qd0=qd0)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 0.049), joints=[j])], plane=True)])
    o = O.Oracle(b, params())
    for n in range(1, 11):
        o.step(1)
        st = o.get_state()
        assert o.stats()["n_contacts"][0] >= 1
        assert st["joint_qd"][0] == qd0, (n, st["joint_qd"][0])
        assert abs(st["joint_q"][0] - qd0 * DT * n) < 1e-12
        assert o.stats()["status"][0] == 0


def test_implicit_pd_one_step_closed_form():
    """Single joint about the vertical axis (no gravity torque): the stable-PD step
    I q̈ = kp (q̄ - q - dt q̇) - kd q̇ - (dt kd + dt² kp) q̈."""
    m, hx, hw, kp, kd, q0, qd0, tgt = 0.8, 0.15, 0.03, 100.0, 10.0, 0.2, -0.5, 0.9
    j = dict(parent=-1, type=0, axis=(0, 0, 1), com=(hx, 0, 0), half=(hx, hw, hw), mass=m, kp=kp, kd=kd,
             q0=q0, qd0=qd0, target=tgt)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 1), joints=[j])], plane=False)])
    o = O.Oracle(b, params())
    I = m * (hx * hx + hw * hw) / 3 + m * hx * hx
    q, qd = q0, qd0
    for _ in range(50):
        qdd = (kp * (tgt - q - DT * qd) - kd * qd) / (I + DT * kd + DT * DT * kp)
        qd = qd + DT * qdd
        q = q + DT * qd
        o.step(1)
        s = o.get_state()
        assert abs(s["joint_qd"][0] - qd) < 1e-12 and abs(s["joint_q"][0] - q) < 1e-12
    art = o.articulation(0, 0)
    _, _, M0 = o.dynamics_check(0, 0, np.zeros(1), np.zeros(1))
    assert abs(art["M"][0, 0] - M0[0, 0] - (DT * kd + DT * DT * kp)) < 1e-12


def _energy_run(dt, T=2.0):
    rng = np.random.default_rng(7)
    js = []
    for i in range(3):
        js.append(dict(parent=i - 1, type=0, axis=(0, 1, 0) if i != 1 else (1, 0, 0),
                       origin_pos=(0.3 if i else 0.0, 0, 0), com=(0.15, 0, 0), half=(0.15, 0.03, 0.03),
                       mass=1.0 + i, q0=0.4 - 0.3 * i, qd0=0.5))
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 3), joints=js)], plane=False)])
    p = params(dt=dt)
    o = O.Oracle(b, p)
    masses = np.array([1.0, 2.0, 3.0])

    def energy():
        a = o.articulation(0, 0)
        qd = o.get_state()["joint_qd"]
        return 0.5 * qd @ a["M"] @ qd + G * masses @ a["com"][:, 2]

    e0 = energy()
    drift = 0.0
    for _ in range(int(round(T / dt))):
        o.step(1)
        drift = max(drift, abs(energy() - e0))
    return drift


def test_energy_drift_first_order():
    d1 = _energy_run(1 / 120)
    d2 = _energy_run(1 / 240)
    assert d1 > 0
    assert 1.6 < d1 / d2 < 2.6


# ----------------------------------------------------------------------------- contacts: restitution
@pytest.mark.parametrize("m1,m2", [(1.0, 1.0), (1.0, 3.0), (2.5, 0.7)])
def test_elastic_pair_closed_form(m1, m2):
    v1, v2, r = 1.5, -0.8, 0.1
    gap = -0.0004  # inside the slop band: no position correction
    objs = [dict(shape=0, half=r, mass=m1, mu=0.0, rest=1.0, pos=(-r - gap / 2, 0, 5), vel=(v1, 0, 0)),
            dict(shape=0, half=r, mass=m2, mu=0.0, rest=1.0, pos=(r + gap / 2, 0, 5), vel=(v2, 0, 0))]
    b = sg.custom_batch([dict(objects=objs, plane=False)])
    o = O.Oracle(b, params(gravity=(0.0, 0.0, 0.0), rest_thresh=0.0, pgs_iters=20))
    o.step(1)
    v = o.get_state()["obj_vel"][:, 0]
    e1 = ((m1 - m2) * v1 + 2 * m2 * v2) / (m1 + m2)
    e2 = ((m2 - m1) * v2 + 2 * m1 * v1) / (m1 + m2)
    assert abs(v[0] - e1) < 1e-12 and abs(v[1] - e2) < 1e-12
    assert abs(m1 * v[0] + m2 * v[1] - (m1 * v1 + m2 * v2)) < 1e-12


def test_sphere_hitting_a_pivoted_lever_conserves_angular_momentum():
    """No gravity, no friction: a sphere (restitution 1) falls onto a lever that turns
    freely about a horizontal axis through one end.  The impact is elastic in the
    normal direction and the angular momentum about the pivot is conserved, which
    fixes both outcomes: with d the lever arm of the contact and I_p the lever's
    moment of inertia about the pivot, the normal impulse is
    lambda = 2 v / (1/m + d^2 / I_p), the sphere leaves at -v + lambda / m and the
    lever turns at lambda d / I_p."""
    m, r, v, d = 0.7, 0.05, 1.2, 0.4
    M, hx, hy, hz = 3.0, 0.25, 0.05, 0.01
    lever = dict(parent=-1, type=0, axis=(0, 1, 0), origin_pos=(0, 0, 0), origin_quat=(1, 0, 0, 0),
                 com=(hx, 0, 0), half=(hx, hy, hz), mass=M, mu=0.0)
    gap = -0.0004  # inside the slop band
    sphere = dict(shape=0, half=r, mass=m, mu=0.0, rest=1.0, pos=(d, 0, hz + r + gap), vel=(0, 0, -v))
    b = sg.custom_batch([dict(objects=[sphere], arts=[dict(base_pos=(0, 0, 0), joints=[lever])], plane=False)])
    o = O.Oracle(b, params(gravity=(0.0, 0.0, 0.0), rest_thresh=0.0, pgs_iters=20))
    o.step(1)
    st = o.get_state()
    Ip = M / 3 * (hx * hx + hz * hz) + M * hx * hx
    lam = 2 * v / (1 / m + d * d / Ip)
    assert abs(st["obj_vel"][0][2] - (-v + lam / m)) < 1e-10
    assert abs(st["joint_qd"][0] - lam * d / Ip) < 1e-10
    assert abs(Ip * st["joint_qd"][0] - m * d * st["obj_vel"][0][2] - m * d * v) < 1e-10  # L about the pivot


@pytest.mark.parametrize("rests", [(0.5, 0.0), (0.0, 0.5)])
def test_restitution_of_a_pair_is_the_larger_coefficient(rests):
    """Newton's law of restitution for a head-on pair, with the pair's coefficient
    the larger of the two bodies' (the reading of an unspecified combination rule):
    the bodies separate at e times their approach speed and momentum is conserved,
    whichever body carries the restitution."""
    m1, m2, v1, v2, r = 1.0, 3.0, 1.5, -0.8, 0.1
    gap = -0.0004  # inside the slop band: no position correction
    objs = [dict(shape=0, half=r, mass=m1, mu=0.0, rest=rests[0], pos=(-r - gap / 2, 0, 5), vel=(v1, 0, 0)),
            dict(shape=0, half=r, mass=m2, mu=0.0, rest=rests[1], pos=(r + gap / 2, 0, 5), vel=(v2, 0, 0))]
    b = sg.custom_batch([dict(objects=objs, plane=False)])
    o = O.Oracle(b, params(gravity=(0.0, 0.0, 0.0), rest_thresh=0.0, pgs_iters=20))
    o.step(1)
    v = o.get_state()["obj_vel"][:, 0]
    e, M = max(rests), m1 + m2
    assert abs(v[0] - (m1 * v1 + m2 * v2 - m2 * e * (v1 - v2)) / M) < 1e-12
    assert abs(v[1] - (m1 * v1 + m2 * v2 + m1 * e * (v1 - v2)) / M) < 1e-12


# ----------------------------------------------------------------------------- narrowphase
def test_sphere_contacts_closed_form():
    c = O.narrowphase(0, (0.3, -0.2, 0.07), (1, 0, 0, 0), (0.08, 0, 0), 2)
    assert len(c["sep"]) == 1
    assert np.allclose(c["n"][0], [0, 0, 1]) and abs(c["sep"][0] + 0.01) < 1e-15
    assert np.allclose(c["p"][0], [0.3, -0.2, -0.005])
    # sphere-sphere: A is the first collider, normal from B to A
    c = O.narrowphase(0, (0, 0, 0), (1, 0, 0, 0), (0.1, 0, 0), 0, (0.15, 0.05, 0), None, (0.05, 0, 0))
    d = np.array([-0.15, -0.05, 0])
    dist = np.linalg.norm(d)
    assert np.allclose(c["n"][0], d / dist) and abs(c["sep"][0] - (dist - 0.15)) < 1e-15
    # sphere-box, closest point outside, and inside (push out through the nearest face)
    c = O.narrowphase(0, (1.49, 0.2, 0.3), (1, 0, 0, 0), (0.48, 0, 0), 1, (0, 0, 0), (1, 0, 0, 0), (1, 2, 3))
    assert np.allclose(c["n"][0], [1, 0, 0]) and abs(c["sep"][0] - 0.01) < 1e-12
    assert np.allclose(c["p"][0], [1.005, 0.2, 0.3])
    c = O.narrowphase(0, (0.1, 0.1, 2.9), (1, 0, 0, 0), (0.05, 0, 0), 1, (0, 0, 0), (1, 0, 0, 0), (1, 2, 3))
    assert np.allclose(c["n"][0], [0, 0, 1]) and abs(c["sep"][0] + 0.15) < 1e-12
    # rotated box: same answer in the box frame
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rand_quat(rng)
        R = qrot(q)
        xb = rng.uniform(-1, 1, 3)
        h = rng.uniform(0.1, 0.5, 3)
        loc = np.array([h[0] + 0.005, rng.uniform(-h[1], h[1]), rng.uniform(-h[2], h[2])])
        c = O.narrowphase(0, xb + R @ loc, (1, 0, 0, 0), (0.003, 0, 0), 1, xb, q, h)
        assert np.allclose(c["n"][0], R[:, 0], atol=1e-12) and abs(c["sep"][0] - 0.002) < 1e-12


def _vertices(x, R, h):
    out = []
    for k in range(8):
        l = np.array([h[0] if k & 1 else -h[0], h[1] if k & 2 else -h[1], h[2] if k & 4 else -h[2]])
        out.append(x + R @ l)
    return np.array(out)


def test_box_plane_vertex_enumeration():
    rng = np.random.default_rng(4)
    n_checked = 0
    for _ in range(300):
        q = rand_quat(rng)
        h = rng.uniform(0.03, 0.15, 3)
        x = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.0, 0.3)])
        V = _vertices(x, qrot(q), h)
        c = O.narrowphase(1, x, q, h, 2)
        expect = [k for k in range(8) if V[k, 2] <= 0.02]
        if len(expect) > 4:
            continue
        n_checked += 1
        assert list(c["feat"]) == expect
        for i, k in enumerate(expect):
            assert np.allclose(c["p"][i], [V[k, 0], V[k, 1], V[k, 2] / 2], atol=1e-14)
            assert abs(c["sep"][i] - V[k, 2]) < 1e-14
    assert n_checked > 50
    # thin plate lying flat: all 8 vertices within the margin -> reduced to 4, deepest kept
    h = np.array([0.2, 0.1, 0.004])
    q = np.array([math.cos(0.01), math.sin(0.01), 0, 0])
    x = np.array([0, 0, 0.005])
    V = _vertices(x, qrot(q), h)
    c = O.narrowphase(1, x, q, h, 2)
    assert len(c["sep"]) == 4
    assert int(np.argmin(V[:, 2])) in list(c["feat"])


def _sat_axes(xa, Ra, ha, xb, Rb, hb):
    faces = [Rb[:, k] for k in range(3)] + [Ra[:, k] for k in range(3)]
    edges = []
    for i in range(3):
        for j in range(3):
            u = np.cross(Ra[:, i], Rb[:, j])
            edges.append(u / np.linalg.norm(u) if np.linalg.norm(u) >= 1e-3 else None)

    def sep(u):
        ra = sum(ha[k] * abs(u @ Ra[:, k]) for k in range(3))
        rb = sum(hb[k] * abs(u @ Rb[:, k]) for k in range(3))
        return abs(u @ (xa - xb)) - ra - rb

    return faces, [sep(u) for u in faces], edges, [sep(u) if u is not None else -np.inf for u in edges]


def _surface_samples(x, R, h, k=9):
    g = np.linspace(-1, 1, k)
    pts = []
    for ax in range(3):
        for s in (-1, 1):
            for a in g:
                for bb in g:
                    l = np.zeros(3)
                    l[ax] = s
                    o = [i for i in range(3) if i != ax]
                    l[o[0]], l[o[1]] = a, bb
                    pts.append(x + R @ (l * h))
    return np.array(pts)


def test_box_box_against_sat_brute_force():
    rng = np.random.default_rng(5)
    n_face = n_edge = n_none = 0
    for it in range(600):
        qa, qb = rand_quat(rng), rand_quat(rng)
        Ra, Rb = qrot(qa), qrot(qb)
        ha, hb = rng.uniform(0.03, 0.3, 3), rng.uniform(0.03, 0.3, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xb = rng.uniform(-1, 1, 3)
        xa = xb + d * rng.uniform(0.0, 1.0) * (np.linalg.norm(ha) + np.linalg.norm(hb))
        faces, fs, edges, es = _sat_axes(xa, Ra, ha, xb, Rb, hb)
        c = O.narrowphase(1, xa, qa, ha, 1, xb, qb, hb, margin=0.02)
        fmax, emax = max(fs), max(es)
        if emax > fmax + 1e-3:
            if emax > 0.02:
                assert len(c["sep"]) == 0
                n_none += 1
                continue
            n_edge += 1
            assert len(c["sep"]) == 1 and abs(c["sep"][0] - emax) < 1e-4
            k = next(i for i in range(9) if es[i] >= emax - 1e-4)
            assert c["feat"][0] == 1024 + k
            assert abs(abs(c["n"][0] @ edges[k]) - 1) < 1e-12 and c["n"][0] @ (xa - xb) >= 0
            continue
        if fmax > 0.02:
            assert len(c["sep"]) == 0
            n_none += 1
            # a separated pair never has sampled surface points closer than the SAT gap
            pa, pb = _surface_samples(xa, Ra, ha), _surface_samples(xb, Rb, hb)
            dmin = np.sqrt(((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1).min())
            assert dmin >= fmax - 1e-9
            continue
        k = next(i for i in range(6) if fs[i] >= fmax - 1e-4)
        u = faces[k]
        ref_is_b = k < 3
        n_face += 1
        assert 1 <= len(c["sep"]) <= 4
        xr, Rr, hr = (xb, Rb, hb) if ref_is_b else (xa, Ra, ha)
        xi = xa if ref_is_b else xb
        nref = u if u @ (xi - xr) >= 0 else -u
        exp_n = nref if ref_is_b else -nref
        fc = xr + nref * hr[k % 3]
        for i in range(len(c["sep"])):
            assert np.allclose(c["n"][i], exp_n, atol=1e-12)
            assert c["sep"][i] <= 0.02 + 1e-12
            # the incident point (contact point + half the separation along nref) lies on the
            # reference face's side of every clip plane and at distance sep from its plane
            pi = c["p"][i] + nref * c["sep"][i] / 2
            assert abs(nref @ (pi - fc) - c["sep"][i]) < 1e-10
            for t in [j for j in range(3) if j != k % 3]:
                assert abs(Rr[:, t] @ (pi - fc)) <= hr[t] + 1e-10
            assert c["feat"][i] // 64 == (0 if ref_is_b else 6) + 2 * (k % 3) + (0 if nref @ u > 0 else 1)
        # contacts carry the deepest clipped point: no point of the reduced set is deeper
        # than the reference-axis overlap
        assert min(c["sep"]) >= fs[k] - 1e-9
    assert n_face > 100 and n_edge > 10 and n_none > 50


def test_edge_contact_point_midway_between_the_edges_closest_points():
    """Edge-edge contacts over 3000 random box pairs: the supporting edge of each box
    along the contact normal (of A's four edges parallel to its axis i the one
    deepest towards B, of B's the one deepest towards A, found here by enumeration),
    the closest points of the two edges' lines (solved here as a 2 x 2 system), each
    clamped to its edge, and the contact point midway between them.  Some pairs need
    the clamp."""
    rng = np.random.default_rng(5)
    n_edge = n_clamped = 0
    for it in range(3000):
        qa, qb = rand_quat(rng), rand_quat(rng)
        Ra, Rb = qrot(qa), qrot(qb)
        ha, hb = rng.uniform(0.03, 0.3, 3), rng.uniform(0.03, 0.3, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        xb = rng.uniform(-1, 1, 3)
        xa = xb + d * rng.uniform(0.0, 1.0) * (np.linalg.norm(ha) + np.linalg.norm(hb))
        _, fs, _, es = _sat_axes(xa, Ra, ha, xb, Rb, hb)
        if not (max(es) > max(fs) + 1e-3 and max(es) <= 0.02):
            continue
        c = O.narrowphase(1, xa, qa, ha, 1, xb, qb, hb, margin=0.02)
        k = int(c["feat"][0]) - 1024
        i, j, L = k // 3, k % 3, c["n"][0]
        ua, ub = Ra[:, i], Rb[:, j]

        def mids(x, R, h, axis):
            others = [t for t in range(3) if t != axis]
            return [x + s0 * h[others[0]] * R[:, others[0]] + s1 * h[others[1]] * R[:, others[1]]
                    for s0, s1 in itertools.product((-1, 1), repeat=2)]

        ma = min(mids(xa, Ra, ha, i), key=lambda m: L @ m)
        mb = max(mids(xb, Rb, hb, j), key=lambda m: L @ m)
        A = np.array([[ua @ ua, -(ua @ ub)], [ua @ ub, -(ub @ ub)]])
        s_, t_ = np.linalg.solve(A, [-(ua @ (ma - mb)), -(ub @ (ma - mb))])
        n_clamped += abs(s_) > ha[i] or abs(t_) > hb[j]
        want = (ma + np.clip(s_, -ha[i], ha[i]) * ua + mb + np.clip(t_, -hb[j], hb[j]) * ub) / 2
        assert np.linalg.norm(c["p"][0] - want) < 1e-10, (it, c["p"][0], want)
        n_edge += 1
    assert n_edge > 500 and n_clamped >= 1, (n_edge, n_clamped)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _qaxis(ax, ang):
    ax = np.asarray(ax, float) / np.linalg.norm(ax)
    return np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)])


def test_face_manifold_reduced_to_deepest_farthest_and_largest_areas():
    """A box turned 0.5 rad and tilted 0.02 rad, pressed into a larger box's top face:
    its bottom face, clipped to the top face's four side planes (textbook
    Sutherland-Hodgman, here), has six vertices at six depths.  The manifold keeps
    four, picked in turn: the deepest; the one farthest from it; the one spanning the
    largest triangle with those two; the one spanning the largest quadrilateral with
    those three (the sum of the three triangles it forms with their sides).  Each pick
    is unique here by a clear margin, so the tie rule does not enter."""
    hb, xb = np.array([0.3, 0.2, 0.1]), np.zeros(3)
    ha = np.array([0.25, 0.15, 0.05])
    qa = _qmul(_qaxis((1, 0.3, 0), 0.02), _qaxis((0, 0, 1), 0.5))
    Ra = qrot(qa)
    quad = [Ra @ np.array([sx * ha[0], sy * ha[1], -ha[2]]) for sx, sy in [(-1, -1), (1, -1), (1, 1), (-1, 1)]]
    xa = np.array([0.0, 0.0, hb[2] - min(c[2] for c in quad) - 0.004])
    poly = [xa + c for c in quad]
    for axis, lim in ((0, hb[0]), (0, -hb[0]), (1, hb[1]), (1, -hb[1])):  # keep s * (P[axis] - lim) <= 0
        sgn = 1.0 if lim > 0 else -1.0
        dist = lambda P: sgn * (P[axis] - lim)
        out = []
        for i in range(len(poly)):
            P, Q = poly[i], poly[(i + 1) % len(poly)]
            if dist(P) <= 0:
                out.append(P)
            if (dist(P) <= 0) != (dist(Q) <= 0):
                out.append(P + (Q - P) * (dist(P) / (dist(P) - dist(Q))))
        poly = out
    assert len(poly) == 6
    seps = np.array([P[2] - hb[2] for P in poly])
    pts = np.array([P - np.array([0, 0, 1.0]) * sp / 2 for P, sp in zip(poly, seps)])  # contact points: midway

    def pick(vals, taken, biggest):
        order = sorted((v, i) for i, v in enumerate(vals) if i not in taken)
        best, runner = (order[-1], order[-2]) if biggest else (order[0], order[1])
        assert abs(best[0] - runner[0]) > 1e-4  # unique: no tie to break
        return best[1]

    i1 = pick(seps, set(), False)
    i2 = pick([np.linalg.norm(q - pts[i1]) for q in pts], {i1}, True)
    p1, p2 = pts[i1], pts[i2]
    i3 = pick([np.linalg.norm(np.cross(p2 - p1, q - p1)) for q in pts], {i1, i2}, True)
    p3 = pts[i3]
    i4 = pick([np.linalg.norm(np.cross(q - p1, p2 - p1)) + np.linalg.norm(np.cross(q - p2, p3 - p2)) +
               np.linalg.norm(np.cross(q - p3, p1 - p3)) for q in pts], {i1, i2, i3}, True)
    c = O.narrowphase(1, xa, qa, ha, 1, xb, (1, 0, 0, 0), hb)
    assert len(c["sep"]) == 4
    np.testing.assert_allclose(c["n"], np.tile([0, 0, 1.0], (4, 1)), atol=1e-12)
    np.testing.assert_allclose(sorted(c["sep"]), sorted(seps[[i1, i2, i3, i4]]), rtol=0, atol=1e-12)
    want = pts[[i1, i2, i3, i4]]
    for q in c["p"]:
        assert np.min(np.linalg.norm(want - q, axis=1)) < 1e-12


def test_box_stack_contacts_closed_form():
    # A (half 0.1) resting 5 mm into B (half 0.3, 0.3, 0.2): four corners of A's bottom face
    c = O.narrowphase(1, (0.05, 0, 0.295), (1, 0, 0, 0), (0.1, 0.1, 0.1), 1, (0, 0, 0), (1, 0, 0, 0),
                      (0.3, 0.3, 0.2))
    assert len(c["sep"]) == 4
    assert np.allclose(c["n"], [[0, 0, 1]] * 4)
    assert np.allclose(c["sep"], -0.005)
    assert list(c["feat"]) == [256, 257, 258, 259]
    assert np.allclose(sorted(map(tuple, c["p"][:, :2].round(12))), sorted([(-0.05, -0.1), (0.15, -0.1),
                                                                             (0.15, 0.1), (-0.05, 0.1)]))
    assert np.allclose(c["p"][:, 2], 0.1975)
    # overhanging by 5 cm over the +x side: two original vertices, two clipped on the x = 0.3 plane
    c = O.narrowphase(1, (0.25, 0, 0.295), (1, 0, 0, 0), (0.1, 0.1, 0.1), 1, (0, 0, 0), (1, 0, 0, 0),
                      (0.3, 0.3, 0.2))
    xs = sorted(c["p"][:, 0].round(12))
    assert len(c["sep"]) == 4 and np.allclose(xs, [0.15, 0.15, 0.3, 0.3])


# ----------------------------------------------------------------------------- broadphase
def _aabb(shape, x, q, h):
    if shape == 0:
        return x - h[0], x + h[0]
    e = np.abs(qrot(q)) @ h
    return x - e, x + e


def test_broadphase_all_pairs():
    rng = np.random.default_rng(6)
    envs = []
    for _ in range(10):
        objs = []
        for i in range(12):
            shape = int(rng.integers(0, 2))
            objs.append(dict(shape=shape, half=rng.uniform(0.03, 0.15, 3) if shape else rng.uniform(0.03, 0.1),
                             mass=1.0, pos=rng.uniform([-0.6, -0.6, 0.0], [0.6, 0.6, 0.6]), quat=rand_quat(rng)))
        sts = [dict(pos=rng.uniform([-0.6, -0.6, 0.0], [0.6, 0.6, 0.3]), half=rng.uniform(0.1, 0.3, 3))
               for _ in range(4)]
        envs.append(dict(objects=objs, statics=sts, plane=True))
    b = sg.custom_batch(envs)
    o = O.Oracle(b, params())
    s0 = o.get_state()
    o.step(1)
    h = 0.01
    for e, env in enumerate(envs):
        boxes = []
        o0 = b["obj_off"][e]
        for i, ob in enumerate(env["objects"]):
            hh = np.full(3, ob["half"]) if ob["shape"] == 0 else np.asarray(ob["half"])
            boxes.append(_aabb(ob["shape"], s0["obj_pos"][o0 + i], s0["obj_quat"][o0 + i], hh))
        n_obj = len(boxes)
        for st in env["statics"]:
            boxes.append(_aabb(1, np.asarray(st["pos"]), np.array([1.0, 0, 0, 0]), np.asarray(st["half"])))
        expect = []
        nc = len(boxes) + 1
        for a in range(nc):
            for bb in range(a + 1, nc):
                if a >= n_obj and bb >= n_obj:
                    continue
                if bb == nc - 1:
                    ok = boxes[a][0][2] - h <= h
                else:
                    ok = np.all(boxes[a][0] - h <= boxes[bb][1] + h) and np.all(boxes[bb][0] - h <= boxes[a][1] + h)
                if ok:
                    expect.append(a * 4096 + bb)
        assert list(o.pairs(e)) == expect


# ----------------------------------------------------------------------------- PGS
def _lcp_enumerate(A, b):
    n = len(b)
    sols = []
    for mask in range(1 << n):
        S = [i for i in range(n) if mask >> i & 1]
        lam = np.zeros(n)
        if S:
            lam[S] = np.linalg.solve(A[np.ix_(S, S)], -b[S])
        w = A @ lam + b
        if np.all(lam >= -1e-12) and np.all(w >= -1e-12):
            sols.append(lam)
    return sols


def test_pgs_frictionless_equals_lcp_enumeration():
    r = 0.1
    objs = [dict(shape=0, half=r, mass=1.0, mu=0.0, pos=(0, 0, r - 0.004), vel=(0.1, 0, -0.3)),
            dict(shape=0, half=r, mass=2.0, mu=0.0, pos=(0.03, 0.0, 3 * r - 0.01), vel=(0, 0, -0.5)),
            dict(shape=0, half=0.08, mass=0.7, mu=0.0, pos=(0.03 + 0.17, 0.05, 3 * r + 0.03), vel=(-0.4, 0, 0))]
    b = sg.custom_batch([dict(objects=objs, plane=True)])
    p = params(plane_mu=0.0, pgs_tol=1e-14, pgs_max_iters=20000, warm_mode=0)
    o = O.Oracle(b, p)
    s0 = o.get_state()
    o.step(1)
    c = o.contacts(0)
    assert len(c["sep"]) == 3
    m = np.array([1.0, 2.0, 0.7])
    x0 = s0["obj_pos"]
    vstar = s0["obj_vel"] + np.array([0, 0, -G * DT])
    # J rows (linear part only: spheres' angular terms vanish for normals through the centre)
    J = np.zeros((3, 9))
    tgt = np.zeros(3)
    for k in range(3):
        a, bb = c["key"][k, 0], c["key"][k, 1]
        n = c["n"][k]
        J[k, 3 * a:3 * a + 3] = n
        if bb < 3:
            J[k, 3 * bb:3 * bb + 3] = -n
        sep = c["sep"][k]
        tgt[k] = -sep / DT if sep > 0 else (0.0 if sep > -0.001 else -0.2 * (sep + 0.001) / DT)
    Minv = np.diag(np.repeat(1 / m, 3))
    A = J @ Minv @ J.T
    bvec = J @ vstar.ravel() - tgt
    sols = _lcp_enumerate(A, bvec)
    assert len(sols) == 1
    assert np.allclose(c["lam"][:, 0], sols[0], atol=1e-9)
    v_exp = vstar.ravel() + Minv @ J.T @ sols[0]
    assert np.allclose(o.get_state()["obj_vel"].ravel(), v_exp, atol=1e-9)


def test_one_sweep_on_a_single_contact_is_sequential_projection():
    """One PGS sweep over a single contact unit, worked out here from the rigid-body
    quantities: the normal row first, then the two friction rows, each projected with
    the body velocity the rows before it left (Gauss-Seidel within the unit, the
    friction bound from the new normal impulse).  A box resting on one corner, away
    from below its centre of mass (the rows couple through r x d), sliding and
    spinning, one step with one sweep: the oracle's final velocities equal this to
    1e-12."""
    hs, m, mu = np.array([0.1, 0.07, 0.13]), 2.0, 0.5
    rng = np.random.default_rng(13)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    R = qrot(q)
    corners = [np.array(c) * hs for c in itertools.product((-1, 1), repeat=3)]
    zs = sorted((R @ c)[2] for c in corners)
    low = min(corners, key=lambda c: (R @ c)[2])
    p = params(pgs_iters=1)
    assert zs[1] - zs[0] > 2 * p.margin and p.plane_mu == mu  # one corner within the margin
    x = np.array([0.3, -0.1, 0.0])
    x[2] = -0.0004 - (R @ low)[2]  # the corner 0.4 mm deep: inside the slop band
    v0, w0 = np.array([0.5, 0.2, -0.3]), np.array([0.3, -0.4, 0.1])
    b = sg.custom_batch([dict(objects=[dict(shape=1, half=tuple(hs), mass=m, mu=mu, rest=0.0, pos=tuple(x),
                                            quat=tuple(q), vel=tuple(v0), omega=tuple(w0))], plane=True)])
    o = O.Oracle(b, p)
    o.step(1)
    assert o.stats()["n_contacts"][0] == 1
    st = o.get_state()
    # the predict, then the unit's three rows in order (plane: static, normal +z,
    # tangents t1 = n x e_x / |n x e_x| = +y and t2 = n x t1 = -x)
    v, w = v0 + np.array([0.0, 0.0, -G]) * DT, w0.copy()
    Ib = m / 3 * np.array([hs[1] ** 2 + hs[2] ** 2, hs[0] ** 2 + hs[2] ** 2, hs[0] ** 2 + hs[1] ** 2])  # solid box
    Iinv = R @ np.diag(1 / Ib) @ R.T
    corner = x + R @ low
    r = np.array([corner[0], corner[1], corner[2] * 0.5]) - x  # contact point midway to the plane
    n, t1 = np.array([0.0, 0.0, 1.0]), np.array([0.0, 1.0, 0.0])
    t2 = np.cross(n, t1)
    assert np.linalg.norm(np.cross(r, n)) > 0.05  # the normal row turns the box

    def row_vel(d):
        return d @ v + np.cross(r, d) @ w

    def row_meff(d):
        c = np.cross(r, d)
        return 1 / (1 / m + c @ Iinv @ c)

    ln = max(0.0, row_meff(n) * (0.0 - row_vel(n)))
    v, w = v + n * ln / m, w + Iinv @ np.cross(r, n) * ln
    for d in (t1, t2):
        lt = float(np.clip(-row_meff(d) * row_vel(d), -mu * ln, mu * ln))
        v, w = v + d * lt / m, w + Iinv @ np.cross(r, d) * lt
    assert ln > 0
    assert np.allclose(st["obj_vel"][0], v, rtol=0, atol=1e-12), (st["obj_vel"][0], v)
    assert np.allclose(st["obj_omega"][0], w, rtol=0, atol=1e-12), (st["obj_omega"][0], w)


def test_static_friction_box_on_plane():
    m, h = 0.7, np.array([0.1, 0.07, 0.05])
    b = sg.custom_batch([dict(objects=[dict(shape=1, half=h, mass=m, pos=(0, 0, h[2] - 0.0005))], plane=True)])
    o = O.Oracle(b, params(pgs_tol=1e-12, pgs_max_iters=5000))
    for _ in range(30):
        o.step(1)
        c = o.contacts(0)
        assert len(c["sep"]) == 4
        assert abs(c["lam"][:, 0].sum() - m * G * DT) < 1e-9
        assert np.abs(o.get_state()["obj_vel"][0, :2]).max() < 1e-9


@pytest.mark.parametrize("theta", [0.35, 0.6])
def test_incline_stick_and_slide(theta):
    mu = 0.5
    n = np.array([0, -math.sin(theta), math.cos(theta)])
    qs = (math.cos(theta / 2), math.sin(theta / 2), 0, 0)
    hb = 0.1
    x = n * (0.5 + hb - 0.0003)
    b = sg.custom_batch([dict(objects=[dict(shape=1, half=hb, mass=1.0, mu=mu, pos=x, quat=qs)],
                              statics=[dict(pos=(0, 0, 0), half=(2, 2, 0.5), quat=qs, mu=mu)], plane=False)])
    o = O.Oracle(b, params(pgs_tol=1e-13, pgs_max_iters=20000))
    down = np.array([0, -math.cos(theta), -math.sin(theta)])
    vs = []
    for _ in range(40):
        o.step(1)
        vs.append(o.get_state()["obj_vel"][0] @ down)
    vs = np.array(vs)
    if math.tan(theta) < mu:
        assert np.abs(vs).max() < 1e-8
    else:
        a = np.diff(vs[5:]) / DT
        assert np.allclose(a, G * (math.sin(theta) - mu * math.cos(theta)), rtol=1e-6)


def test_contact_capacity_keeps_the_first_contacts_in_order():
    """Eight boxes resting apart on the plane (four vertex contacts each, 32 in all)
    with a capacity of 10: exactly the first 10 contacts in (a, b, feature) order are
    kept -- those of an uncapped run -- and the environment is flagged as overflowed."""
    hb = 0.05
    objs = [dict(shape=1, half=hb, mass=1.0, pos=(0.3 * i, 0, hb)) for i in range(8)]
    b = sg.custom_batch([dict(objects=objs, plane=True)])
    keys = {}
    for cap in (64, 10):
        p = sg.SimParams()
        p.max_contacts = cap
        o = O.Oracle(b, p)
        o.step(1)
        keys[cap] = o.contacts(0)["key"]
        st = o.stats()
        if cap == 64:
            assert len(keys[64]) == 32 and st["status"][0] & 1 == 0
        else:
            assert st["n_contacts"][0] == 10 and st["status"][0] & 1
    assert np.array_equal(keys[10], keys[64][:10])


# ----------------------------------------------------------------------------- sleeping
def test_sleep_step_and_wake_from_free_fall():
    hb, r = 0.1, 0.05
    z0 = 1.0
    objs = [dict(shape=1, half=hb, mass=1.0, pos=(0, 0, hb)), dict(shape=0, half=r, mass=0.5, pos=(0, 0, 50.0))]
    b = sg.custom_batch([dict(objects=objs, plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 1
    o = O.Oracle(b, p)
    for n in range(1, p.sleep_steps + 1):
        o.step(1)
        awake = o.get_state()["obj_awake"][0]
        assert awake == (1 if n < p.sleep_steps else 0), n
    # drop the sphere from z0 above the sleeping box: the first step whose start-of-step
    # position has the fattened AABBs overlapping wakes the box (free fall closed form)
    s = o.get_state()
    s["obj_pos"][1] = (0, 0, z0)
    s["obj_vel"][1] = 0
    o.set_state(s)
    top = 2 * hb
    k_wake = next(k for k in range(1000) if z0 - G * DT * DT * k * (k + 1) / 2 - r <= top + p.margin)
    for k in range(k_wake + 1):
        o.step(1)
        awake = o.get_state()["obj_awake"][0]
        assert awake == (1 if k == k_wake else 0), (k, k_wake)


def test_wake_pass_runs_once_in_pair_order():
    """Sleeping (Sec. 4.1), as read here: one pass per step over the candidate pairs
    in (a, b) order, in which a sleeping object paired with an awake dynamic collider
    wakes -- so a wake travels forward along the pair order within a step, not back.
    Three boxes in a row on the plane, touching: with box 0 awake, pair (0, 1) wakes
    box 1 and then (1, 2) wakes box 2 in the same step; with box 2 awake, pair (0, 1)
    comes first while both are asleep, (1, 2) wakes box 1, and box 0 wakes one step
    later.  (A closure over the contact graph would wake all three at once in both.)"""
    hb = 0.1
    objs = [dict(shape=1, half=hb, mass=1.0, pos=(2 * hb * i, 0, hb)) for i in range(3)]
    b = sg.custom_batch([dict(objects=objs, plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 1
    for start, after1, after2 in (((1, 0, 0), (1, 1, 1), (1, 1, 1)), ((0, 0, 1), (0, 1, 1), (1, 1, 1))):
        o = O.Oracle(b, p)
        s = o.get_state()
        s["obj_awake"][:] = start
        s["obj_ctr"][:] = 0
        s["obj_vel"][:] = 0
        s["obj_omega"][:] = 0
        o.set_state(s)
        o.step(1)
        assert tuple(int(v) for v in o.get_state()["obj_awake"]) == after1, start
        if start[0]:  # every pair active: the order the pass takes, (a, b) ascending (plane = collider 3)
            assert [int(v) for v in o.pairs(0)] == [0 * 4096 + 1, 0 * 4096 + 3, 1 * 4096 + 2, 1 * 4096 + 3,
                                                     2 * 4096 + 3]
        o.step(1)
        assert tuple(int(v) for v in o.get_state()["obj_awake"]) == after2, start


def test_a_body_falls_asleep_at_rest():
    """A frictionless box sliding on the plane at 0.02 m/s, below the sleep threshold,
    counts slow steps and falls asleep after the sleep step count: from then on it is
    at rest -- zero velocity and angular velocity, its position unchanged by later
    steps -- although it was still sliding."""
    hb, v0 = 0.05, 0.02
    b = sg.custom_batch([dict(objects=[dict(shape=1, half=hb, mass=1.0, mu=0.0, pos=(0, 0, hb),
                                            vel=(v0, 0, 0))], plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 1
    o = O.Oracle(b, p)
    for n in range(1, p.sleep_steps + 1):
        o.step(1)
    st = o.get_state()
    assert st["obj_awake"][0] == 0
    assert np.all(st["obj_vel"][0] == 0) and np.all(st["obj_omega"][0] == 0)
    x = st["obj_pos"][0].copy()
    assert x[0] > 0.5 * v0 * p.sleep_steps * DT  # it was still moving when it fell asleep
    o.step(5)
    assert np.array_equal(o.get_state()["obj_pos"][0], x)


def test_an_articulation_link_wakes_a_sleeping_object():
    """Links always count as dynamic colliders in the wake rule: a sleeping box on the
    plane with a link hanging 1 cm above it (the fattened AABBs overlap), the link
    at rest on a vertical revolute axis, wakes at the first step."""
    box = dict(shape=1, half=(0.05, 0.05, 0.05), mass=1.0, pos=(0, 0, 0.05))
    link = dict(parent=-1, type=0, axis=(0, 0, 1), origin_pos=(0, 0, 0), origin_quat=(1, 0, 0, 0),
                com=(0, 0, 0), half=(0.05, 0.05, 0.01), mass=1.0)
    b = sg.custom_batch([dict(objects=[box], arts=[dict(base_pos=(0, 0, 0.12), joints=[link])], plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 1
    o = O.Oracle(b, p)
    s = o.get_state()
    s["obj_awake"][:] = 0
    s["obj_ctr"][:] = 0
    o.set_state(s)
    o.step(1)
    assert o.get_state()["obj_awake"][0] == 1
    assert 0 * 4096 + 1 in [int(v) for v in o.pairs(0)]  # the box-link pair


def test_sleep_counter_counts_consecutive_slow_steps_only():
    """A sphere thrown straight up with v0 = k g dt (no plane): semi-implicit Euler
    gives v_n = v0 - n g dt, so the speed is below the sleep threshold only at the
    apex step n = k (v is exactly 0 there, and +-g dt = +-0.082 m/s on either side,
    above the 0.05 m/s threshold).  The
    sleep counter reads 1 there and 0 at every other step: a slow step is counted,
    a fast one starts the count again."""
    k = 20
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.05, mass=1.0, pos=(0, 0, 5.0),
                                            vel=(0, 0, k * G * DT))], plane=False)])
    p = sg.SimParams()
    p.sleep_enabled = 1
    assert G * DT > p.sleep_lin
    o = O.Oracle(b, p)
    for n in range(1, 2 * k + 1):
        o.step(1)
        st = o.get_state()
        assert st["obj_ctr"][0] == (1 if n == k else 0), n
        assert st["obj_awake"][0] == 1


def test_spinning_body_orientation_recurrence():
    """A sphere spinning at w about z (no contacts; the sphere's inertia is isotropic,
    so w stays constant): the update q <- normalise(q + dt/2 (0, w) q) multiplies q by
    (1, w dt / 2), a rotation by 2 beta with beta = atan(w dt / 2), so from the
    identity q_n = (cos n beta, 0, 0, sin n beta)."""
    w = 7.0
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.05, mass=1.0, pos=(0, 0, 5.0),
                                            omega=(0, 0, w))], plane=False)])
    p = sg.SimParams()
    p.sleep_enabled = 0
    o = O.Oracle(b, p)
    beta = math.atan(w * DT / 2)
    for n in range(1, 121):
        o.step(1)
        q = o.get_state()["obj_quat"][0]
        np.testing.assert_allclose(q, [math.cos(n * beta), 0, 0, math.sin(n * beta)], atol=1e-12)
    np.testing.assert_allclose(o.get_state()["obj_omega"][0], [0, 0, w], atol=1e-12)


def test_joint_limit_is_reached_exactly_and_never_passed():
    """A pendulum released at 0.15 rad swings towards a lower limit at -0.1 rad.  The
    limit row's target (close the remaining gap within the step) puts the joint
    exactly on the limit in the step that would cross it, and never beyond."""
    d, m, hw, lo = 0.3, 1.3, 0.02, -0.1
    j = dict(parent=-1, type=0, axis=(0, 1, 0), com=(0, 0, -d), half=(hw, hw, d), mass=m, q0=0.15,
             lo=lo, hi=0.3, has_limit=1)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 5), joints=[j])], plane=False)])
    o = O.Oracle(b, params())
    q = []
    for _ in range(300):
        o.step(1)
        q.append(o.get_state()["joint_q"][0])
    q = np.array(q)
    assert q.min() >= lo - 1e-12
    assert abs(q.min() - lo) < 1e-12
    free_min = -0.15  # without the limit the swing would reach the mirror of the release angle
    assert lo > free_min + 0.04


def test_prior_frame_match_needs_the_contact_to_stay_close():
    """A sphere sliding at 3 m/s moves its contact point 2.5 cm per step, beyond the
    1 cm match distance: its contact never matches the previous frame, so the warm
    start of every step starts from zero (matched flag 0, prior impulses 0)."""
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.1, mass=1.0, pos=(0, 0, 0.1), vel=(3.0, 0, 0))],
                              plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 0
    assert 2.0 * DT > p.match_dist
    o = O.Oracle(b, p)
    for _ in range(6):
        _, X, _ = o.step_logged()
        assert len(X) == 1
        np.testing.assert_array_equal(X[0][23:27], [0, 0, 0, 0])
        assert o.get_state()["obj_vel"][0, 0] > 2.0


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _qmat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _axis_q(axis, angle):
    u = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * u])


def test_rotating_the_whole_frictionless_scene_rotates_the_result():
    """Rotational covariance: a tilted, anisotropic, spinning box dropped on a static
    floor box, and the same scene with everything (floor, box, velocities, gravity)
    rotated by Q.  After 40 steps with contacts, every result of the rotated scene
    is Q applied to the original one.  Friction is off (the pyramid's tangents are
    tied to the world axes); contacts, impulses, world inertias and integration
    must all transform as vectors and tensors."""
    def run(Rq):
        R = _qmat(Rq)
        q0 = _axis_q((1, 0.5, 0.2), 0.6)
        box = dict(shape=1, half=(0.3, 0.1, 0.05), mass=2.0, mu=0.0, pos=tuple(R @ [0, 0, 0.45]),
                   quat=tuple(_qmul(Rq, q0)), vel=tuple(R @ [0.2, 0, -1.0]), omega=tuple(R @ [0.5, -1.0, 2.0]))
        floor = dict(pos=tuple(R @ [0, 0, -0.5]), half=(2, 2, 0.5), quat=tuple(Rq), mu=0.0)
        b = sg.custom_batch([dict(objects=[box], statics=[floor], plane=False)])
        p = params()
        p.gravity = tuple(R @ [0, 0, -G])
        o = O.Oracle(b, p)
        contacts = 0
        for _ in range(40):
            o.step(1)
            contacts = max(contacts, o.stats()["n_contacts"][0])
        return o.get_state(), contacts
    Q = _axis_q((0.3, -1, 0.4), 1.1)
    R = _qmat(Q)
    a, na = run(np.array([1.0, 0, 0, 0]))
    b, nb = run(Q)
    assert na == nb >= 3
    for k in ("obj_pos", "obj_vel", "obj_omega"):
        np.testing.assert_allclose(b[k][0], R @ a[k][0], atol=1e-12)
    qa = _qmul(Q, a["obj_quat"][0])
    assert min(np.abs(b["obj_quat"][0] - qa).max(), np.abs(b["obj_quat"][0] + qa).max()) < 1e-12


def test_residual_sweeps_do_not_depend_on_the_mass_scale():
    """The residual target is relative (|d lambda| / |lambda|): scaling every mass by
    1000 scales every impulse by 1000 and leaves the sweeps to 1e-6 unchanged, and the
    velocities equal."""
    def run(k):
        boxes = [dict(shape=1, half=(0.2, 0.2, 0.1), mass=m * k, pos=(0.02 * i, 0, 0.1 + 0.2 * i))
                 for i, m in enumerate((3.0, 1.0, 2.0))]
        b = sg.custom_batch([dict(objects=boxes, plane=True)])
        p = params(pgs_tol=1e-6, pgs_max_iters=1000)
        o = O.Oracle(b, p)
        o.step(30)
        return o.stats()["iters"][0], o.get_state()
    (i1, s1), (i2, s2) = run(1.0), run(1000.0)
    assert 3 < i1 < 1000
    assert i1 == i2
    np.testing.assert_allclose(s2["obj_vel"], s1["obj_vel"], atol=1e-9)


def _two_box_stack(m):
    return sg.custom_batch([dict(objects=[dict(shape=1, half=(0.05, 0.05, 0.05), mass=m, pos=(0, 0, 0.05)),
                                          dict(shape=1, half=(0.05, 0.05, 0.05), mass=m, pos=(0.02, 0, 0.15))],
                                 plane=True)])


def test_residual_mode_flags_the_sweep_cap():
    """Residual mode stops at the relative residual target or at the sweep cap; a
    solve stopped by the cap is flagged (status bit 4) and reports the cap as its
    sweep count, one that met the target is not flagged."""
    o = O.Oracle(_two_box_stack(1.0), params(pgs_tol=1e-14, pgs_max_iters=3))
    o.step(1)
    st = o.stats()
    assert st["iters"][0] == 3 and st["status"][0] & 4 and st["resid"][0] > 1e-14
    o = O.Oracle(_two_box_stack(1.0), params(pgs_tol=1e-6, pgs_max_iters=1000))
    o.step(1)
    st = o.stats()
    assert st["iters"][0] < 1000 and st["status"][0] & 4 == 0 and st["resid"][0] <= 1e-6


def test_residual_floor_ends_solves_of_negligible_impulses():
    """The relative residual divides by max(|lambda|, lambda_floor): impulses far below
    the floor (a stack of two 1 mg boxes, whose impulses are 1e-9 of a 1 kg stack's)
    need only a few sweeps, where the same stack at 1 kg -- the same velocities, the
    same relative residual without the floor -- needs many."""
    sweeps = {}
    for m in (1.0, 1e-9):
        o = O.Oracle(_two_box_stack(m), params(pgs_tol=1e-6, pgs_max_iters=1000))
        o.step(1)
        st = o.stats()
        assert st["resid"][0] <= 1e-6 and st["status"][0] & 4 == 0
        sweeps[m] = int(st["iters"][0])
    assert sweeps[1.0] > 50 and sweeps[1e-9] <= 10, sweeps


def test_violated_joint_limit_recovers_at_the_baumgarte_rate():
    """A pendulum at rest 0.05 rad past its lower limit, with gravity pressing it further
    in: the active limit row sets the joint rate that removes the fraction beta of the
    violation in one step, q_1 - lo = (1 - beta)(q_0 - lo)."""
    d, m, hw, lo, q0 = 0.3, 1.3, 0.02, 0.1, 0.05
    j = dict(parent=-1, type=0, axis=(0, 1, 0), com=(0, 0, -d), half=(hw, hw, d), mass=m, q0=q0,
             lo=lo, hi=0.5, has_limit=1)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 5), joints=[j])], plane=False)])
    p = params()
    o = O.Oracle(b, p)
    o.step(1)
    assert abs((o.get_state()["joint_q"][0] - lo) - (1 - p.baumgarte) * (q0 - lo)) < 1e-12


def test_new_contact_training_target_in_units_of_the_support_impulse():
    """A sphere placed exactly on the plane, at rest, with an empty contact cache: its
    contact is new (prior 0) and converges to the support impulse m g dt.  The target's
    unit is m_eff,n (|g| dt + |v_rel|) with m_eff,n = m and the relative velocity
    before the solve the free-fall increment, |v_rel| = g dt, so the unit is 2 m g dt
    and the logged target is (1/2, 0, 0)."""
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.1, mass=2.0, pos=(0, 0, 0.1))], plane=True)])
    o = O.Oracle(b, params())
    _, X, T = o.step_logged()
    assert len(X) == 1 and X[0][26] == 0
    np.testing.assert_allclose(X[0][9:12], [-G * DT, 0, 0], atol=1e-12)
    np.testing.assert_allclose(T[0], [0.5, 0, 0], atol=1e-12)


def test_log_leaves_out_solves_that_missed_the_residual():
    """Training pairs are converged impulses: in residual mode a solve stopped by the
    sweep cap before the residual target logs nothing; the same step with a reachable
    target logs its contact."""
    b = sg.custom_batch([dict(objects=[dict(shape=1, half=(0.1, 0.1, 0.1), mass=1.0, pos=(0, 0, 0.1))],
                              plane=True)])
    for tol, cap, logged in ((1e-14, 1, 0), (1e-6, 1000, 4)):
        p = params()
        p.pgs_tol, p.pgs_max_iters = tol, cap
        o = O.Oracle(b, p)
        _, X, _ = o.step_logged()
        assert len(X) == logged, (tol, cap, len(X))


def test_static_friction_on_an_incline_is_carried_to_the_next_step():
    """A box at rest on an incline of 0.3 rad (mu 0.9 > tan 0.3) tilted about a diagonal
    axis: static friction carries m g sin(theta) dt down the slope.  The next step's
    prior-frame tangential impulses, summed over the box's matched contacts, have that
    magnitude, with both tangent components non-zero (the slope lies between them)."""
    th, m = 0.3, 2.0
    Q = _axis_q((1, 1, 0), th)
    R = _qmat(Q)
    floor = dict(pos=tuple(R @ [0, 0, -0.5]), half=(3, 3, 0.5), quat=tuple(Q), mu=0.9)
    box = dict(shape=1, half=(0.2, 0.2, 0.1), mass=m, mu=0.9, pos=tuple(R @ [0, 0, 0.1]), quat=tuple(Q))
    b = sg.custom_batch([dict(objects=[box], statics=[floor], plane=False)])
    o = O.Oracle(b, params())
    o.step(120)
    _, X, _ = o.step_logged()
    assert len(X) == 4 and np.all(X[:, 26] == 1)
    t = X[:, 24:26].sum(0)
    assert abs(np.linalg.norm(t) - m * G * math.sin(th) * DT) < 1e-9
    assert min(abs(t[0]), abs(t[1])) > 0.2 * np.linalg.norm(t)


# ----------------------------------------------------------------------------- learned warm start MLP
def test_mlp_gelu_values():
    P = np.zeros(O.mlp_nparam())
    off = [0, 128 * 32, 128 * 32 + 128]
    P[0] = 1.0                                  # W1[0][0]
    P[off[2]] = 1.0                             # W2[0][0]
    P[off[2] + 128 * 128 + 128] = 1.0           # W3[0][0]
    w4 = off[2] + 2 * (128 * 128 + 128)
    P[w4] = 1.0                                 # W4[0][0]
    P[w4 + 3 * 128 + 1] = 0.25                  # b4[1]
    gelu = lambda x: 0.5 * x * (1 + math.erf(x / math.sqrt(2)))
    for x0 in (-2.0, -0.3, 0.0, 0.7, 1.0, 3.0):
        X = np.zeros((1, 32))
        X[0, 0] = x0
        Y = O.mlp_forward(P, X)
        assert abs(Y[0, 0] - gelu(gelu(gelu(x0)))) < 1e-15
        assert Y[0, 1] == 0.25 and Y[0, 2] == 0.0


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(8)
    P = sg.mlp_init(3)
    P[128 * 32:128 * 32 + 128] = rng.normal(0, 0.1, 128)
    X = rng.normal(size=(5, 32))
    T = rng.normal(size=(5, 3))
    loss, grad = O.mlp_loss_grad(P, X, T)
    assert loss > 0
    idx = np.concatenate([rng.choice(np.arange(a, b), min(12, b - a), replace=False) for a, b in
                          ((0, 4096), (4096, 4224), (4224, 20608), (20608, 20736), (20736, 37120),
                           (37120, 37248), (37248, 37632), (37632, 37635))])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (O.mlp_loss_grad(Pp, X, T)[0] - O.mlp_loss_grad(Pm, X, T)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def _constant_output_step(s0, batch, c, iters=0, mode=2):
    """One step from s0 with a network whose output is the constant c (W4 = 0, b4 = c);
    with no sweeps the applied impulses are the warm start itself."""
    p = sg.params_for(2)
    p.warm_mode = mode
    p.pgs_iters = iters
    P = np.zeros(O.mlp_nparam())
    P[-3:] = c
    o = O.Oracle(batch, p)
    o.set_mlp(P)
    o.set_state(s0)
    o.step(1)
    return o.get_state()


def test_warm_start_output_limit_and_fallback():
    """The learned warm start uses the network's output limited to the training-target
    range +-10 (units of m_eff,n |g| dt): a constant output beyond it starts the solve
    exactly where the limit does, one inside it does not; a non-finite output falls
    back to the prior-frame impulse, which is zero for contacts without a match."""
    b = sg.make_batch(2, 8)
    o = O.Oracle(b, sg.params_for(2))
    o.step(40)
    s0 = o.get_state()
    s0["cache_count"][:] = 0  # every contact is new
    at_limit = _constant_output_step(s0, b, [10.0, -10.0, 10.0])
    beyond = _constant_output_step(s0, b, [25.0, -30.0, 40.0])
    inside = _constant_output_step(s0, b, [5.0, -5.0, 5.0])
    for k in ("obj_vel", "obj_omega", "joint_qd"):
        assert np.array_equal(at_limit[k], beyond[k]), k
    assert np.abs(inside["obj_vel"] - at_limit["obj_vel"]).max() > 1e-2
    prior = _constant_output_step(s0, b, [0.0, 0.0, 0.0], mode=1)
    nan = _constant_output_step(s0, b, [np.nan, 0.0, 0.0])
    for k in ("obj_vel", "obj_omega", "joint_qd"):
        assert np.array_equal(prior[k], nan[k]), k


def test_contact_features_of_a_resting_sphere():
    """The learned warm start's 32 contact features for a sphere resting on the plane,
    from closed forms: normal +z; lever arms along the normal (the contact point is
    midway between the sphere's lowest point and the plane); the row velocity before
    the solve is the free-fall increment -g dt; effective masses m along the normal
    and m / (1 + 5 |r_a|^2 / (2 r^2)) = 2m/7 along the tangents (solid sphere,
    I = 2/5 m r^2); friction sqrt(mu_a mu_b); prior impulse m g dt (static support,
    matched); pair type sphere-plane; a zero correction target."""
    r, m, dt = 0.1, 2.0, 1.0 / 120.0
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=r, mass=m, mu=0.8, pos=(0.3, -0.2, r + 0.002))],
                              plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 0
    p.plane_mu = 0.5
    o = O.Oracle(b, p)
    o.step(60)
    _, X, T = o.step_logged()
    assert len(X) == 1
    f, g = X[0], 9.81
    z = o.get_state()["obj_pos"][0, 2]
    assert abs(z - r) < 1e-9
    np.testing.assert_allclose(f[0:3], [0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(f[3:6], [0, 0, -(z + r) / 2], atol=1e-9)
    np.testing.assert_allclose(f[6:9], [0, 0, (z - r) / 2], atol=1e-9)
    np.testing.assert_allclose(f[9:12], [-g * dt, 0, 0], atol=1e-9)
    np.testing.assert_allclose(f[12:15], 0, atol=1e-12)
    assert abs(f[15]) < 1e-9
    assert f[16] == 1 / m and f[17] == 0
    ra2 = ((z + r) / 2) ** 2
    mt = m / (1 + 2.5 * ra2 / r ** 2)
    np.testing.assert_allclose(f[18:21], [m, mt, mt], rtol=1e-9)
    assert abs(f[19] - 2 * m / 7) < 1e-6
    assert abs(f[21] - math.sqrt(0.8 * 0.5)) < 1e-12
    assert abs(f[22] + g * dt) < 1e-12
    np.testing.assert_allclose(f[23:26], [m * g * dt, 0, 0], atol=1e-9)
    assert f[26] == 1
    np.testing.assert_array_equal(f[27:32], [0, 1, 0, 0, 0])
    np.testing.assert_allclose(T[0], 0, atol=1e-9)


def test_contact_features_of_spinning_spheres_pressed_into_a_box_and_the_plane():
    """The features at the first step of two spinning spheres pressed 4 mm into a
    static box and into the plane, from closed forms: the lever arms to the contact
    point midway between the surfaces (to the box's centre for the box; to the
    contact point's foot on the plane, i.e. along the normal, for the plane); the
    relative angular velocity, sphere minus the (static) other side; separation
    -4 mm; no prior impulse; pair types sphere-box and sphere-plane."""
    r, m, pen = 0.1, 2.0, 0.004
    bx, bh = np.array([0.0, 0.0, 0.5]), np.array([0.2, 0.2, 0.05])
    top = bx[2] + bh[2]
    s0, w0 = np.array([0.03, -0.02, top + r - pen]), np.array([0.0, 0.0, 3.0])
    s1, w1 = np.array([0.3, 0.1, r - pen]), np.array([0.0, 0.0, -2.0])
    envs = [dict(objects=[dict(shape=0, half=r, mass=m, mu=0.8, pos=tuple(s0), omega=tuple(w0))],
                 statics=[dict(pos=tuple(bx), half=tuple(bh), mu=0.5)], plane=False),
            dict(objects=[dict(shape=0, half=r, mass=m, mu=0.8, pos=tuple(s1), omega=tuple(w1))], plane=True)]
    b = sg.custom_batch(envs)
    p = params(plane_mu=0.5)
    o = O.Oracle(b, p)
    _, X, _ = o.step_logged()
    assert len(X) == 2
    for f, s, w, other, onehot in ((X[0], s0, w0, bx, [0, 0, 1, 0, 0]),
                                   (X[1], s1, w1, None, [0, 1, 0, 0, 0])):
        pz = s[2] - r + pen / 2  # midway between the sphere's lowest point and the surface
        cp = np.array([s[0], s[1], pz])
        np.testing.assert_allclose(f[0:3], [0, 0, 1], atol=1e-12)
        np.testing.assert_allclose(f[3:6], cp - s, atol=1e-12)
        rb = cp - other if other is not None else np.array([0.0, 0.0, pz])
        np.testing.assert_allclose(f[6:9], rb, atol=1e-12)
        np.testing.assert_allclose(f[12:15], w, atol=1e-12)
        assert abs(f[15] + pen) < 1e-12
        assert f[16] == 1 / m and f[17] == 0
        np.testing.assert_allclose(f[23:27], 0, atol=0)
        np.testing.assert_array_equal(f[27:32], onehot)


def test_sphere_comes_to_rest_on_a_turned_robot_base_box():
    """A robot base turned 90 degrees about z carries its collider box at an offset
    fixed in the base frame: the box sits at base_pos + R off.  A sphere released 1 mm
    above that box's top face comes to rest on it (its height settles at the top plus
    its radius, within the slop band), 0.5 m from where the unturned offset would put
    the box."""
    yaw = (math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4))
    base, off, bh = np.array([0.0, 0.0, 0.5]), np.array([0.5, 0.0, 0.2]), 0.1
    box_c = base + qrot(yaw) @ off
    assert np.allclose(box_c, [0.0, 0.5, 0.7])
    top, r = box_c[2] + bh, 0.05
    link = dict(parent=-1, type=0, axis=(0, 0, 1), origin_pos=(-1.0, -1.0, 0.0), origin_quat=(1, 0, 0, 0),
                com=(0, 0, 0), half=(0.05, 0.05, 0.05), mass=1.0)
    arts = [dict(base_pos=tuple(base), base_quat=yaw, base_coll=(tuple(off), (bh, bh, bh)), kinematic=1,
                 joints=[link])]
    sphere = dict(shape=0, half=r, mass=1.0, pos=(box_c[0], box_c[1], top + r + 0.001))
    b = sg.custom_batch([dict(objects=[sphere], arts=arts, plane=False)])
    o = O.Oracle(b, params())
    o.step(60)
    z = o.get_state()["obj_pos"][0][2]
    assert top + r - 0.0011 < z < top + r + 1e-6, z - (top + r)


def _check_first_fit(col, na, nb):
    """A colouring against its definition, pairwise: units that share a colouring
    node never share a colour below the serial overflow colour 64, and each unit
    takes the smallest colour left by the earlier units it shares a node with
    (64 once all 64 are taken)."""
    n = len(col)
    nodes = [{x for x in (na[i], nb[i]) if x >= 0} for i in range(n)]
    for j in range(n):
        taken = {col[i] for i in range(j) if nodes[i] & nodes[j] and col[i] < 64}
        want = next((c for c in range(64) if c not in taken), 64)
        assert col[j] == want, (j, col[j], want)
        for i in range(j):
            if nodes[i] & nodes[j]:
                assert col[i] != col[j] or col[j] == 64, (i, j)


@pytest.mark.parametrize("config,n,warm", [(2, 8, 40), (3, 8, 40)])
def test_colouring_is_greedy_first_fit_in_unit_order(config, n, warm):
    b = sg.make_batch(config, n)
    o = O.Oracle(b, sg.params_for(config))
    o.step(warm)
    multi = 0
    for e in range(n):
        c = o.colouring(e)
        col = list(c["colour"])
        _check_first_fit(col, c["node_a"], c["node_b"])
        assert o.stats()["n_colours"][e] == (max(col) + 1 if col else 0)
        multi += max(col, default=0) >= 1
    assert multi >= n // 2  # most environments need more than one colour


def test_limit_rows_of_one_articulation_take_distinct_colours():
    """Units in one colour touch disjoint bodies, and every joint-limit row acts on
    its whole articulation: three joints of one chain held at zero-width limits and
    started moving give three limit rows, which must fall in three colours."""
    js = [dict(parent=i - 1, type=0, axis=(0, 0, 1), origin_pos=(0.2 if i else 0.0, 0, 0), origin_quat=(1, 0, 0, 0),
               com=(0.1, 0, 0), half=(0.1, 0.02, 0.02), mass=1.0, lo=0.0, hi=0.0, has_limit=1, qd0=1.0 + i)
          for i in range(3)]
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0, 0, 1.0), joints=js)], plane=False)])
    o = O.Oracle(b, params())
    o.step(1)
    st = o.stats()
    assert st["n_limit_rows"][0] == 3 and st["n_contacts"][0] == 0
    col = list(o.colouring(0)["colour"])
    assert len(col) == 3 and sorted(col) == [0, 1, 2], col


def test_colouring_overflows_into_the_serial_colour():
    """70 spheres resting on one dynamic box put more than 64 units on the box's
    node: colours 0..63 go to the first 64, the rest to the serial colour 64."""
    k, r = 10, 0.04
    spheres = [dict(shape=0, half=r, mass=0.1, pos=(-0.9 + 0.2 * (i % k), -0.6 + 0.2 * (i // k), 0.2 + r))
               for i in range(70)]
    box = dict(shape=1, half=(1.0, 0.7, 0.1), mass=50.0, pos=(0, 0, 0.1))
    b = sg.custom_batch([dict(objects=[box] + spheres, plane=True)])
    p = sg.SimParams()
    p.sleep_enabled = 0
    p.max_contacts = 256
    o = O.Oracle(b, p)
    o.step(3)
    c = o.colouring(0)
    col = list(c["colour"])
    _check_first_fit(col, c["node_a"], c["node_b"])
    on_box = [i for i in range(len(col)) if 0 in (c["node_a"][i], c["node_b"][i])]
    assert len(on_box) > 64
    assert sorted(col[i] for i in on_box[:64]) == list(range(64))
    assert all(col[i] == 64 for i in on_box[64:])
    assert o.stats()["n_colours"][0] == 65


def test_learned_warm_start_scale_and_pyramid():
    """With no sweeps the warm start is the whole impulse.  A sphere placed exactly on
    the plane with an empty cache (its contact is new, relative velocity -g dt along
    the normal): a network output of (1/2, 0, 0), half a unit of m_eff,n (|g| dt +
    |v_rel|) = 2 m g dt, is exactly the support impulse, so the velocity stays 0; an
    output of (0, 5, -5) has no normal impulse, so the friction pyramid clamps the
    tangential impulses to 0 and only the free-fall increment -g dt remains."""
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.1, mass=2.0, pos=(0, 0, 0.1))], plane=True)])
    s0 = O.Oracle(b, sg.params_for(2)).get_state()
    v = _constant_output_step(s0, b, [0.5, 0.0, 0.0])["obj_vel"][0]
    np.testing.assert_allclose(v, [0, 0, 0], atol=1e-12)
    v = _constant_output_step(s0, b, [0.0, 5.0, -5.0])["obj_vel"][0]
    np.testing.assert_allclose(v, [0, 0, -G * DT], atol=1e-12)


def test_learned_gate_serves_fast_matched_contacts_only():
    """The network starts a matched contact only when the contact's relative velocity
    exceeds 4 |g| dt.  With no sweeps and a constant output (y, 0, 0):
    - a sphere resting on the plane (matched, |v_rel| = g dt) keeps its prior-frame
      impulse, so the step equals the prior-frame warm start's exactly;
    - a sphere sliding at 1 m/s (matched, |v_rel| > 4 g dt) gets the normal impulse
      prior + y m (g dt + |v_rel|), so its vertical velocity rises by exactly
      y (g dt + |v_rel|) over the prior-frame start's (a sphere's normal impulse acts
      through its centre)."""
    r, m, y = 0.1, 2.0, 0.75
    for vx, served in ((0.0, False), (1.0, True)):
        b = sg.custom_batch([dict(objects=[dict(shape=0, half=r, mass=m, pos=(0, 0, r), vel=(vx, 0, 0))],
                                  plane=True)])
        p = sg.params_for(2)
        p.sleep_enabled = 0
        o = O.Oracle(b, p)
        o.step(1)  # the contact is cached: matched from here on
        s0 = o.get_state()
        prior = _constant_output_step(s0, b, [0.0, 0.0, 0.0], mode=1)
        learned = _constant_output_step(s0, b, [y, 0.0, 0.0])
        q = sg.params_for(2)
        q.sleep_enabled, q.pgs_iters = 0, 0
        o2 = O.Oracle(b, q)
        o2.set_state(s0)
        _, X, _ = o2.step_logged()
        assert len(X) == 1 and X[0][26] == 1
        vrel = float(np.linalg.norm(X[0][9:12]))
        assert (vrel > 4 * G * DT) == served
        dz = learned["obj_vel"][0, 2] - prior["obj_vel"][0, 2]
        if served:
            assert abs(dz - y * (G * DT + vrel)) < 1e-12, (dz, y * (G * DT + vrel))
        else:
            for k in ("obj_vel", "obj_omega", "obj_pos"):
                assert np.array_equal(learned[k], prior[k]), k


def test_learned_start_keeps_each_rows_prior_and_never_pulls():
    """A sphere sliding at 1 m/s on the plane (matched, served by the network), with no
    sweeps, so that the applied impulses are the warm start itself:
    - a zero output starts every row at its own prior-frame impulse -- the normal row
      at the normal's, each friction row at its own tangent's (the cached friction
      lies along t2 here) -- so the step equals the prior-frame start exactly;
    - an output of -20 (limited to -10 units) drives the normal impulse below zero,
      where it stops at zero: no support and no friction, so the sphere leaves the
      step in free fall, v = v0 - g dt e_z, its spin unchanged."""
    r, m = 0.1, 2.0
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=r, mass=m, pos=(0, 0, r), vel=(1.0, 0, 0))], plane=True)])
    p = sg.params_for(2)
    p.sleep_enabled = 0
    o = O.Oracle(b, p)
    o.step(1)
    s0 = o.get_state()
    q = sg.params_for(2)
    q.sleep_enabled, q.pgs_iters = 0, 0
    o2 = O.Oracle(b, q)
    o2.set_state(s0)
    _, X, _ = o2.step_logged()
    assert len(X) == 1 and X[0][26] == 1 and abs(X[0][25]) > 1e-3 and abs(X[0][24]) < 1e-12
    prior = _constant_output_step(s0, b, [0.0, 0.0, 0.0], mode=1)
    zero = _constant_output_step(s0, b, [0.0, 0.0, 0.0])
    for k in ("obj_vel", "obj_omega", "obj_pos"):
        assert np.array_equal(zero[k], prior[k]), k
    pulled = _constant_output_step(s0, b, [-20.0, 0.0, 0.0])
    np.testing.assert_allclose(pulled["obj_vel"][0], s0["obj_vel"][0] + np.array([0, 0, -G * DT]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(pulled["obj_omega"][0], s0["obj_omega"][0], rtol=0, atol=1e-12)


def test_param_count():
    assert O.mlp_nparam() == 32 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 3 + 3 == len(sg.mlp_init(0))


def _box_on_robot_base(mass=0.7):
    """A box resting on the kinematic robot's base box; the robot's one link is far above."""
    link = dict(parent=-1, type=0, axis=(0.0, 0.0, 1.0), origin_pos=(0.0, 0.0, 1.5), com=(0.0, 0.0, 0.1),
                half=(0.03, 0.03, 0.1), mass=1.0, kp=100.0, kd=10.0)
    robot = dict(base_pos=(0.0, 0.0, 0.0), base_coll=((0.0, 0.0, 0.2), (0.25, 0.25, 0.2)), kinematic=1,
                 joints=[link])
    box = dict(shape=1, half=(0.05, 0.05, 0.05), mass=mass, pos=(0.05, -0.03, 0.4499))
    cabinet = dict(robot, kinematic=0)  # the same articulation, not the robot
    return sg.custom_batch([dict(objects=[box], arts=[robot]), dict(objects=[box]),
                            dict(objects=[box], arts=[cabinet])])


def test_robot_contact_force_equals_supported_weight():
    """At rest on the robot's base the box's normal impulses per step sum to m g dt, so the
    robot's contact force is m g; it accumulates by m g per step from a reset and flags the
    env once past the limit.  An env without a robot has none, and neither has a box
    resting on another articulation's base."""
    m = 0.7
    b = _box_on_robot_base(m)
    p = sg.SimParams()
    p.sleep_enabled = 0
    p.pgs_tol = 1e-10
    p.force_limit = 0.0
    orc = O.Oracle(b, p)
    orc.step(240)
    step, acc = orc.robot_force()
    w = m * 9.81
    assert abs(step[0] - w) < 1e-6 * w, (step[0], w)
    assert step[1] == 0.0 and acc[1] == 0.0
    # resting on a base box that is not the robot's: contacts, but no robot force
    assert orc.stats()["n_contacts"][2] > 0 and step[2] == 0.0 and acc[2] == 0.0
    orc.reset_robot_force([0])
    p.force_limit = 3.5 * w
    orc.set_params(p)
    for k in range(4):
        orc.step(1)
        assert (orc.stats()["status"][0] & 8) == (8 if (k + 1) * w > p.force_limit * (1 + 1e-9) else 0)
    _, acc = orc.robot_force()
    assert abs(acc[0] - 4 * w) < 4e-6 * w


def _motor_link(target, half=(0.5, 0.1, 0.05), mass=6.0):
    """One revolute link about z on a kinematic base, COM on the axis (gravity exerts no
    torque about z), nothing to touch."""
    link = dict(parent=-1, type=0, axis=(0.0, 0.0, 1.0), origin_pos=(0.0, 0.0, 1.0), com=(0.0, 0.0, 0.0),
                half=half, mass=mass, kp=100.0, kd=10.0, target=target)
    return sg.custom_batch([dict(arts=[dict(base_pos=(0.0, 0.0, 0.0), kinematic=1, joints=[link])], plane=False)])


def test_motor_row_closes_kp_of_the_error_per_step():
    """Motor mode: one row on q̇ with target rate kp (q̄ - q)/dt; unsaturated, the error
    shrinks by (1 - kp) per step exactly (the implicit PD is off)."""
    p = sg.SimParams()
    p.motor_mode = 1
    q_bar = 0.01
    orc = O.Oracle(_motor_link(q_bar), p)
    for k in range(1, 8):
        orc.step(1)
        q = orc.get_state()["joint_q"][0]
        assert abs(q - (q_bar - (1 - p.motor_kp) ** k * q_bar)) < 1e-12, (k, q)


def test_motor_impulse_is_capped():
    """A large error saturates the row: one step adds exactly max_impulse / I_zz to q̇
    (I_zz = m (hx² + hy²) / 3 about the COM axis; no armature in motor mode)."""
    p = sg.SimParams()
    p.motor_mode = 1
    half, m = (0.5, 0.1, 0.05), 6.0
    orc = O.Oracle(_motor_link(2.0, half, m), p)
    orc.step(1)
    i_zz = m * (half[0] ** 2 + half[1] ** 2) / 3
    qd = orc.get_state()["joint_qd"][0]
    assert abs(qd - p.motor_max_impulse / i_zz) < 1e-9 * qd, (qd, p.motor_max_impulse / i_zz)
    assert abs(orc.get_state()["joint_motor_lambda"][0] - p.motor_max_impulse) < 1e-12
