"""GPU (CUDA, FP32) against the FP64 oracle, element by element, through the C ABI.

Tolerances (stated by the method's accuracy contract): from an identical state,
one step agrees within 1e-4 absolute in metres, radians and metres/second;
100 contact-free steps of the 7-DoF arms agree within 1e-3.  Environments whose
discrete decisions differ (contact keys, awake flags, active joint limits,
colour count, residual-driven sweep count) are counted as decision flips and
compared only up to the flip; they must stay rare.
"""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from parity import (decision_flips, env_errors, gpu_to_oracle, identical_start, input_ulp_sensitivity, state_errors,
                    step_both_and_compare)

pytestmark = pytest.mark.gpu

TOL = 1e-4       # m, rad, m/s (and quaternion components)
RATE_TOL = 1e-3  # rad/s (free-body omega, revolute joint rates): see test_tolerance_derivation.py
TOLS = {"obj_pos": TOL, "obj_vel": TOL, "obj_quat": TOL, "joint_q": TOL, "joint_qd_prismatic": TOL,
        "joint_qd_revolute": RATE_TOL, "obj_omega": RATE_TOL}


def _engine(batch, params, **kw):
    from paper_2106_14405_gb300 import Sim
    return Sim(batch, params, **kw)


def _assert_errors(err):
    for k, v in err.items():
        assert v <= TOLS[k], (k, v, err)


# ----------------------------------------------------------------------------- articulations
def test_config1_per_step_and_free_run():
    b = sg.make_batch(1)  # 64 fixed 7-DoF arms, contact-free
    p = sg.params_for(1)
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    worst = 0.0
    for _ in range(100):
        err, flips, _, _ = step_both_and_compare(b, sim, orc)
        assert not flips.any()
        worst = max(worst, err["joint_q"], err["joint_qd_revolute"])
    assert worst <= TOL
    # free run from the initial state, no re-synchronisation
    sim2 = _engine(b, p)
    orc2 = O.Oracle(b, p)
    sim2.step(100)
    orc2.step(100)
    gs, os_ = sim2.get_state(), orc2.get_state()
    err = state_errors(b, gs, os_, np.arange(b.n_envs))
    assert err["joint_q"] <= 1e-3 and err["joint_qd_revolute"] <= 1e-3, err


@pytest.mark.parametrize("config,n", [(2, 32), (3, 32)])
def test_aba_crba_inverse_stage(config, n):
    b = sg.make_batch(config, n)
    p = sg.params_for(config)
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(7)
    identical_start(sim, orc)
    sim.step(1)  # ABA outputs of this step are at the state just set
    a = sim.articulation()
    jo = b["joint_off"]
    for e in range(b.n_envs):
        for k in range(b["art_off"][e], b["art_off"][e + 1]):
            r = orc.articulation(e, k - b["art_off"][e])
            j0, nj = jo[k], r["n"]
            assert np.abs(a["com"][j0:j0 + nj] - r["com"]).max() < 1e-5
            assert np.abs(a["rot"][j0:j0 + nj] - r["rot"]).max() < 1e-5
            assert np.abs(a["qdd"][j0:j0 + nj] - r["qdd"]).max() * p.dt < TOL
            rel = np.abs(a["minv"][k, :nj, :nj] - r["Minv"]).max() / np.abs(r["Minv"]).max()
            assert rel < 1e-4


def test_fp64_inverse_path():
    b = sg.make_batch(2, 16)
    p = sg.params_for(2)
    p.fp64_cond = 1.0  # every articulation counts as ill-conditioned
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(3)
    identical_start(sim, orc)
    sim.step(1)
    assert (sim.stats()["fp64_used"] == 1).all()
    a = sim.articulation()
    for e in range(b.n_envs):
        r = orc.articulation(e, 0)
        rel = np.abs(a["minv"][b["art_off"][e], :9, :9] - r["Minv"]).max() / np.abs(r["Minv"]).max()
        assert rel < 1e-5


# ----------------------------------------------------------------------------- collision
def _collision_stage(b, p, warms):
    """From identical states after each warm-up, one step on both sides: the pair lists
    and contact keys exactly, the contact values within TOL.  Returns the number of
    environments checked, of decision flips and the largest active pair count seen."""
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    checked = flips = most = 0
    for i, warm in enumerate(warms):
        sim.step(warm)
        identical_start(sim, orc)
        sim.step(1)
        orc.step(1)
        cnt, pairs = sim.pairs(1024)
        gc = sim.contacts()
        for e in range(b.n_envs):
            most = max(most, int(cnt[e]))
            op = orc.pairs(e)
            oc = orc.contacts(e)
            n = gc["count"][e]
            if not np.array_equal(pairs[e, :cnt[e]], op) or n != len(oc["sep"]) or \
                    not np.array_equal(gc["key"][e, :n], oc["key"]):
                flips += 1
                continue
            checked += 1
            if n:
                assert np.abs(gc["p"][e, :n] - oc["p"]).max() < TOL
                assert np.abs(gc["n"][e, :n] - oc["n"]).max() < TOL
                assert np.abs(gc["sep"][e, :n] - oc["sep"]).max() < TOL
    return checked, flips, most


def test_collision_stage_pairs_and_contacts():
    checked, flips, _ = _collision_stage(sg.make_batch(2, 64), sg.params_for(2), (20, 5, 5))
    assert checked > 0
    assert flips <= 0.05 * (checked + flips), (flips, checked)


def test_collision_stage_more_pairs_than_lanes():
    """Scenes whose active pairs take more than one round of 32 lanes (the prefix sum
    of contact counts carried across rounds): the 30-object scene inside its timed
    window, and environments of 64 mixed spheres and boxes (box-box, box-plane and
    sphere pairs together), the latter also with a contact capacity they overflow (the
    first capacity-many contacts in pair order are kept)."""
    checked, flips, most = _collision_stage(sg.make_batch(5, 32), sg.params_for(5), (70, 15))
    assert most > 32, most
    assert checked > 0 and flips <= 0.1 * (checked + flips), (flips, checked)
    envs = []
    for seed in range(6):
        rng = np.random.default_rng(seed)
        envs.append(dict(objects=[dict(shape=int(i % 2), half=(0.05, 0.05, 0.05) if i % 2 else 0.05, mass=0.5,
                                       pos=(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 0.05 + 0.11 * (i // 16)))
                                  for i in range(64)]))
    b = sg.custom_batch(envs)
    for cap in (256, 40):
        p = sg.SimParams()
        p.max_contacts = cap
        checked, flips, most = _collision_stage(b, p, (1, 3))
        assert most > 32, most
        assert checked > 0, (flips, checked)


def _rand_quat(rng):
    q = rng.normal(size=4)
    return q / np.linalg.norm(q)


def test_box_box_contacts_random_poses():
    """Box-box narrowphase over 2048 random relative poses in contact (face-face,
    face-edge, edge-edge; half extents U(0.03, 0.15)): the GPU's contacts -- keys,
    points, normals, separations -- against the oracle's 15-axis SAT with
    Sutherland-Hodgman clipping of the incident face.  The GPU enumerates the clipped
    polygon's vertices directly with the same labels, so keys must agree exactly;
    near-ties of the axis choice (within rounding of the 1e-4 m tolerance) may flip a
    few cases."""
    rng = np.random.default_rng(31)
    envs, ref = [], []
    while len(envs) < 2048:
        ha, hb = rng.uniform(0.03, 0.15, 3), rng.uniform(0.03, 0.15, 3)
        qa, qb = _rand_quat(rng), _rand_quat(rng)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dist = rng.uniform(0.3, 1.0) * (np.linalg.norm(ha) + np.linalg.norm(hb))
        xb = np.array([0.0, 0.0, 1.0])
        xa = xb + d * dist
        c = O.narrowphase(1, xa, qa, ha, 1, xb, qb, hb, margin=0.02)
        if len(c["sep"]) == 0:
            continue
        ref.append(c)
        envs.append(dict(objects=[dict(shape=1, half=tuple(ha), mass=1.0, pos=tuple(xa), quat=tuple(qa)),
                                  dict(shape=1, half=tuple(hb), mass=1.0, pos=tuple(xb), quat=tuple(qb))],
                         plane=False))
    b = sg.custom_batch(envs)
    p = sg.params_for(2)
    p.gravity = (0.0, 0.0, 0.0)
    sim = _engine(b, p)
    sim.step(1)
    gc = sim.contacts()
    flips = checked = 0
    kinds = set()
    for e, c in enumerate(ref):
        n = gc["count"][e]
        keys = gc["key"][e, :n]
        if n != len(c["sep"]) or not (np.all(keys[:, :2] == [0, 1]) and np.array_equal(keys[:, 2], c["feat"])):
            flips += 1
            continue
        checked += 1
        kinds.add("edge" if c["feat"][0] >= 1024 else "face")
        assert np.abs(gc["p"][e, :n] - c["p"]).max() < TOL, e
        assert np.abs(gc["n"][e, :n] - c["n"]).max() < TOL, e
        assert np.abs(gc["sep"][e, :n] - c["sep"]).max() < TOL, e
    assert kinds == {"edge", "face"}
    assert flips <= 0.02 * len(ref), (flips, checked)


# ----------------------------------------------------------------------------- full step
@pytest.mark.parametrize("config,n,warm", [(2, 64, 12), (2, 64, 40), (2, 64, 150), (3, 48, 30), (5, 24, 40)])
def test_full_step_parity(config, n, warm):
    b = sg.make_batch(config, n)
    p = sg.params_for(config)
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(warm)
    err, flips, gs, os_ = step_both_and_compare(b, sim, orc)
    assert flips.mean() <= 0.05, flips.sum()
    _assert_errors(err)
    # final impulses of the contacts of unflipped envs
    gc = sim.contacts()
    for e in np.nonzero(~flips)[0]:
        oc = orc.contacts(e)
        m = len(oc["sep"])
        if m:
            assert np.abs(gc["lam"][e, :m] - oc["lam"]).max() < 1e-3 * max(1.0, np.abs(oc["lam"]).max())


@pytest.mark.parametrize("config,warm", [(2, 150), (3, 60)])
def test_robot_contact_force_parity(config, warm):
    """Per-env contact force on the robot (normal impulses of its contacts / dt) and the
    force-limit flag against the oracle from an identical state; the force tolerance is
    the impulse tolerance of the full-step test summed over the env's robot contacts."""
    b = sg.make_batch(config, 64)
    p = sg.params_for(config)
    p.force_limit = 20.0
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(warm)
    sim.sync()
    sim.reset_robot_force()
    orc.reset_robot_force()
    identical_start(sim, orc)
    sim.step(1)
    orc.step(1)
    st_g, st_o = sim.stats()["status"], orc.stats()["status"]  # before any sync clears the GPU bits
    flips = decision_flips(b, sim, orc, sim.get_state(), orc.get_state())
    g_step, g_acc = sim.robot_force()
    o_step, o_acc = orc.robot_force()
    checked = 0
    for e in np.nonzero(~flips)[0]:
        oc = orc.contacts(e)
        m = len(oc["sep"])
        tol = 1e-3 * max(1.0, np.abs(oc["lam"]).max() if m else 0.0) * max(m, 1) / p.dt
        assert abs(g_step[e] - o_step[e]) <= tol, (e, g_step[e], o_step[e], tol)
        assert g_acc[e] == g_step[e]
        if abs(o_acc[e] - p.force_limit) > tol:
            assert (st_g[e] & 8) == (st_o[e] & 8), (e, g_acc[e], o_acc[e])
        checked += o_step[e] > 0
    assert checked > 0  # some arm is in contact
    sim.reset_robot_force([int(np.argmax(g_acc))])
    assert sim.robot_force()[1].max() <= np.sort(g_acc)[-2] + 1e-6


@pytest.mark.parametrize("config,warm", [(2, 40), (2, 150), (3, 30)])
def test_motor_mode_parity(config, warm):
    """The paper's impulse-capped joint motors (motor mode) against the oracle: full-step
    state parity from an identical state, and the motor impulses of unflipped envs."""
    b = sg.make_batch(config, 64)
    p = sg.params_for(config)
    p.motor_mode = 1
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(warm)
    err, flips, gs, os_ = step_both_and_compare(b, sim, orc)
    assert flips.mean() <= 0.05, flips.sum()
    _assert_errors(err)
    lam_g, lam_o = gs["joint_motor_lambda"], os_["joint_motor_lambda"]
    assert np.abs(lam_o).max() > 0  # the motors act
    jo = b.arrays["joint_off"][b.arrays["art_off"]]
    for e in np.nonzero(~flips)[0]:
        g, o = lam_g[jo[e]:jo[e + 1]], lam_o[jo[e]:jo[e + 1]]
        assert np.abs(g - o).max() <= 1e-3 * max(1.0, np.abs(o).max()), (e, g, o)


def test_motor_closed_form_on_gpu():
    """One motor-driven link with no gravity torque: the error shrinks by (1 - kp) per step."""
    link = dict(parent=-1, type=0, axis=(0.0, 0.0, 1.0), origin_pos=(0.0, 0.0, 1.0), com=(0.0, 0.0, 0.0),
                half=(0.5, 0.1, 0.05), mass=6.0, kp=100.0, kd=10.0, target=0.01)
    b = sg.custom_batch([dict(arts=[dict(base_pos=(0.0, 0.0, 0.0), kinematic=1, joints=[link])], plane=False)] * 4)
    p = sg.SimParams()
    p.motor_mode = 1
    sim = _engine(b, p)
    for k in range(1, 8):
        sim.step(1)
        q = sim.get_state()["joint_q"]
        want = 0.01 - (1 - p.motor_kp) ** k * 0.01
        assert np.abs(q - want).max() < 1e-6, (k, q, want)


@pytest.mark.parametrize("warm_mode", [0, 1])
def test_residual_mode_parity(warm_mode):
    b = sg.make_batch(4, 48)
    p = sg.params_for(4)
    p.warm_mode = warm_mode
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(30)
    err, flips, _, _ = step_both_and_compare(b, sim, orc, compare_iters=False)
    assert flips.mean() <= 0.05
    _assert_errors(err)
    gst, ost = sim.stats(), orc.stats()
    ok = ~flips & (ost["n_rows"] > 0)
    # the sweep count to 1e-6 agrees up to the FP32 rounding of the residual
    assert np.abs(gst["iters"][ok] - ost["iters"][ok]).max() <= max(3, 0.1 * ost["iters"][ok].max())


@pytest.mark.parametrize("config,warm,tune,learned", [(2, 30, False, False), (2, 150, True, False),
                                                     (3, 60, True, False), (5, 40, True, False), (5, 40, True, True)])
def test_full_size_sampled_parity_bench_config(config, warm, tune, learned):
    """Full-size workloads (4096 / 16384 / 65536 environments) in the benchmark's
    launch configuration: CUDA graph, and with `tune` the autotuner's shape chosen on
    the live batch as the benchmark does; 64 sampled environments, always including
    the one with the most colours (the longest Gauss-Seidel chain, swept on one
    lane), checked against the oracle one step later.

    With `learned` the step uses the learned warm start.  Its BF16 network starts
    new contacts a little away from the oracle's FP64 forward, so a fixed sweep
    count would not give the same impulses; both sides therefore iterate to the
    1e-6 relative residual, where the solution no longer depends on the start."""
    b = sg.make_batch(config)
    p = sg.params_for(config)
    P = None
    if learned:
        p.warm_mode, p.pgs_tol, p.pgs_max_iters = 2, 1e-6, 1000
        P = sg.mlp_init(5) * 0.1
    sim = _engine(b, p, use_graph=True)
    if P is not None:
        sim.set_mlp(P)
    sim.step(warm)
    if tune:
        sim.autotune(steps_per_trial=1, rounds=2)
        sim.step(2)
    rc, acc, _ = sim.sync()
    assert acc & 2 == 0
    heaviest = int(np.argmax(sim.stats()["n_colours"]))
    gs = sim.get_state()
    gs["obj_pos_comp"][:] = 0
    gs["joint_q_comp"][:] = 0
    sim.set_state({"obj_pos_comp": gs["obj_pos_comp"], "joint_q_comp": gs["joint_q_comp"]})
    rng = np.random.default_rng(0)
    envs = np.unique(np.concatenate([rng.choice(b.n_envs, 63, replace=False), [heaviest]]))
    sub = b.subset(envs)
    orc = O.Oracle(sub, p)
    if P is not None:
        orc.set_mlp(P)
    oo, jo = b["obj_off"], b["joint_off"][b["art_off"]]
    oi = np.concatenate([np.arange(oo[e], oo[e + 1]) for e in envs])
    ji = np.concatenate([np.arange(jo[e], jo[e + 1]) for e in envs])
    ai = np.concatenate([np.arange(b["art_off"][e], b["art_off"][e + 1]) for e in envs])
    s_sub = {}
    for k in ("obj_pos", "obj_quat", "obj_vel", "obj_omega", "obj_awake", "obj_ctr"):
        s_sub[k] = gs[k][oi]
    for k in ("joint_q", "joint_qd", "joint_target", "joint_lim_lambda", "joint_lim_side", "joint_motor_lambda"):
        s_sub[k] = gs[k][ji]
    for k in ("art_base_pos", "art_base_quat"):
        s_sub[k] = gs[k][ai]
    for k in ("cache_count", "cache_key", "cache_p", "cache_lambda"):
        s_sub[k] = gs[k].reshape((b.n_envs, -1) + gs[k].shape[1:])[envs].reshape((-1,) + gs[k].shape[1:]) \
            if k != "cache_count" else gs[k][envs]
    start = gpu_to_oracle(s_sub)
    orc.set_state(start)
    sim.step(1)
    sim.sync()
    orc.step(1)
    g2 = sim.get_state()
    o2 = orc.get_state()
    gc = sim.contacts()
    flips = 0
    over = {}  # env -> its errors, where one exceeds the fixed tolerance
    for i, e in enumerate(envs):
        oc = orc.contacts(i)
        n = gc["count"][e]
        if n != len(oc["sep"]) or not np.array_equal(gc["key"][e, :n], oc["key"]):
            flips += 1
            continue
        so = np.arange(sub["obj_off"][i], sub["obj_off"][i + 1])
        go = np.arange(oo[e], oo[e + 1])
        if not np.array_equal(g2["obj_awake"][go], o2["obj_awake"][so]):
            flips += 1
            continue
        err = env_errors(sub, g2, o2, i, go=go, gj=np.arange(jo[e], jo[e + 1]))
        if any(v >= TOLS[k] for k, v in err.items()):
            over[i] = err
    assert flips <= 4
    # An env over the fixed tolerance passes only where the state itself is
    # ill-conditioned: one FP32 ulp of input must move the FP64 result by at least
    # a third of the tolerance, and the GPU must stay within the tolerance plus
    # three times that movement.  Such states are rare (at most 2 of 64).
    assert len(over) <= 2, over
    if over:
        floor = input_ulp_sensitivity(sub, p, start, mlp=P)
        for i, err in over.items():
            for k, v in err.items():
                if v >= TOLS[k]:
                    assert floor[i][k] >= TOLS[k] / 3 and v < TOLS[k] + 3 * floor[i][k], (envs[i], k, v, floor[i])


def test_overflow_colour_runs_serially_between_parallel_colours():
    """More than 64 units on one node (17 small boxes resting on one dynamic box, four
    contact points each, and the box's own four on the plane) send the surplus to the
    serial overflow colour 64; 7 more boxes on the plane keep the environment on the
    colour-parallel path (more than 1.5 units per colour), so colour 64 runs on one
    lane after 64 parallel colours.  One step from an identical state matches the
    oracle, with 65 colours on both sides."""
    h = 0.05
    on_box = [dict(shape=1, half=h, mass=0.2, pos=(-0.8 + 0.25 * (i % 6), -0.5 + 0.3 * (i // 6), 0.2 + h))
              for i in range(17)]
    on_plane = [dict(shape=1, half=h, mass=0.2, pos=(-1.5 + 0.3 * i, 1.3, h)) for i in range(7)]
    box = dict(shape=1, half=(1.0, 0.7, 0.1), mass=50.0, pos=(0, 0, 0.1))
    scene = dict(objects=[box] + on_box + on_plane, plane=True)
    b = sg.custom_batch([scene, scene])
    p = sg.SimParams()
    p.sleep_enabled = 0
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    sim.step(3)
    err, flips, _, _ = step_both_and_compare(b, sim, orc)
    assert not flips.any()
    _assert_errors(err)
    assert sim.stats()["n_colours"].tolist() == orc.stats()["n_colours"].tolist() == [65, 65]
    assert sim.sync()[1] & 3 == 0


# ----------------------------------------------------------------------------- closed forms on the GPU
def test_gpu_free_fall_and_elastic_pair():
    x0 = np.array([0.5, -0.2, 10.0])
    b = sg.custom_batch([dict(objects=[dict(shape=0, half=0.1, mass=1.0, pos=x0)], plane=False),
                         dict(objects=[dict(shape=0, half=0.1, mass=1.0, rest=1.0, mu=0.0, pos=(-0.1002, 0, 5),
                                            vel=(1.5, 0, 0)),
                                       dict(shape=0, half=0.1, mass=3.0, rest=1.0, mu=0.0, pos=(0.1002, 0, 5),
                                            vel=(-0.8, 0, 0))], plane=False)])
    p = sg.SimParams()
    p.sleep_enabled = 0
    p.rest_thresh = 0.0
    sim = _engine(b, p)
    sim.step(1)
    s = sim.get_state()
    v = s["obj_vel"]
    g = 9.81 * p.dt
    assert abs(v[0, 2] + g) < 1e-6
    m1, m2, v1, v2 = 1.0, 3.0, 1.5, -0.8
    e1 = ((m1 - m2) * v1 + 2 * m2 * v2) / (m1 + m2)
    e2 = ((m2 - m1) * v2 + 2 * m1 * v1) / (m1 + m2)
    assert abs(v[1, 0] - e1) < 1e-5 and abs(v[2, 0] - e2) < 1e-5
    assert abs(m1 * v[1, 0] + m2 * v[2, 0] - (m1 * v1 + m2 * v2)) < 1e-5
    for n in range(2, 101):
        sim.step(1)
    s = sim.get_state()
    z = x0[2] - 9.81 * p.dt ** 2 * 100 * 101 / 2
    assert abs(s["obj_pos"][0, 2] - s["obj_pos_comp"][0, 2] - z) < 1e-4


# ----------------------------------------------------------------------------- determinism, checkpoint
def test_determinism_and_checkpoint_resume():
    b = sg.make_batch(2, 128)
    p = sg.params_for(2)
    s1 = _engine(b, p)
    s2 = _engine(b, p, use_graph=True)
    s1.step(100)
    s2.step(50)
    ck = s2.get_state()
    s2.step(50)
    a, c = s1.get_state(), s2.get_state()
    for k in a:
        assert np.array_equal(a[k], c[k]), k
    s3 = _engine(b, p)
    s3.set_state(ck)
    s3.step(50)
    d = s3.get_state()
    for k in a:
        assert np.array_equal(a[k], d[k]), k


# ----------------------------------------------------------------------------- edge cases and failures
def test_edge_cases_empty_and_tiny_envs():
    b = sg.custom_batch([dict(plane=True), dict(plane=False),
                         dict(objects=[dict(shape=1, half=(0.1, 0.1, 0.1), mass=1.0, pos=(0, 0, 0.0995))])])
    p = sg.SimParams()
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    err, flips, _, _ = step_both_and_compare(b, sim, orc, nsteps=5)
    assert not flips.any()
    _assert_errors(err)
    e0 = sg.custom_batch([])
    sim0 = _engine(e0, p)
    sim0.step(3)
    assert sim0.sync()[0] == 0


def test_max_objects_env_and_contact_overflow():
    rng = np.random.default_rng(2)
    objs = [dict(shape=int(i % 2), half=(0.05, 0.05, 0.05) if i % 2 else 0.05, mass=0.5,
                 pos=(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 0.05 + 0.11 * (i // 16))) for i in range(64)]
    b = sg.custom_batch([dict(objects=objs)])
    p = sg.SimParams()
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    err, flips, _, _ = step_both_and_compare(b, sim, orc, nsteps=1)
    if not flips.any():
        _assert_errors(err)
    p2 = sg.SimParams()
    p2.max_contacts = 8
    sim2 = _engine(b, p2)
    sim2.step(2)
    rc, acc, st = sim2.sync()
    assert rc == 5 and acc & 1


def test_failure_detection_numeric_and_timeout():
    from paper_2106_14405_gb300 import SimError
    b = sg.make_batch(2, 8)
    p = sg.params_for(2)
    sim = _engine(b, p)
    sim.step(20)
    s = sim.get_state()
    s["obj_vel"][3, 0] = np.nan
    sim.set_state({"obj_vel": s["obj_vel"]})
    sim.step(1)
    rc, acc, st = sim.sync()
    assert rc == 4 and st[0] & 2 and not (st[1:] & 2).any()
    p2 = sg.params_for(4)
    p2.pgs_tol = 1e-12
    p2.pgs_max_iters = 2
    sim2 = _engine(sg.make_batch(2, 8), p2)
    sim2.step(25)
    rc, acc, st = sim2.sync()
    assert rc == 6 and acc & 4
    bad = sg.make_batch(2, 2)
    bad["joint_parent"] = bad["joint_parent"].copy()
    bad["joint_parent"][3] = 5
    with pytest.raises(SimError, match="joint_parent"):
        _engine(bad, p)


def test_bounded_device_waits_run_out_and_report():
    """The step's bounded device waits made to run out (sim_debug_hold_async withholds
    the asynchronous completions): the PGS kernel reads the articulation row pool
    from global memory instead -- the step stays bit-identical -- and flags
    SIM_ENV_DEVICE_WAIT;
    the learned warm start's tensor-core wait runs out and flags its environments;
    sim_sync reports SIM_ERR_TIMEOUT and the context stays usable."""
    b = sg.make_batch(2, 64)
    p = sg.params_for(2)
    ref, s = _engine(b, p), _engine(b, p)
    ref.step(30)
    s.step(30)
    s.debug_hold_async(True)
    ref.step(1)
    s.step(1)
    rc, acc, st = s.sync()
    assert rc == 6 and acc & 16 and not acc & 2
    pool = ref.stats()["n_contacts"] > 0
    assert (st[pool] & 16).any()
    want, got = ref.get_state(), s.get_state()
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    s.debug_hold_async(False)
    ref.step(3)
    s.step(3)
    rc, acc, _ = s.sync()
    assert rc == 0 and not acc & 16
    want, got = ref.get_state(), s.get_state()
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    # learned warm start: the tensor-core completion wait runs out
    p2 = sg.params_for(2)
    p2.warm_mode = 2
    sim = _engine(b, p2)
    sim.set_mlp(sg.mlp_init(3) * 0.1)
    sim.step(20)
    assert sim.sync()[0] == 0
    sim.debug_hold_async(True)
    sim.step(1)
    rc, acc, st = sim.sync()
    assert rc == 6 and acc & 16 and not acc & 2
    sim.debug_hold_async(False)
    sim.step(2)
    rc, acc, _ = sim.sync()
    assert rc == 0 and not acc & 16


def test_set_targets_and_base_pose_through_device_buffers():
    b = sg.make_batch(2, 16)
    p = sg.params_for(2)
    sim = _engine(b, p)
    orc = O.Oracle(b, p)
    tg = torch.tensor(b["joint_target"] * 0.5, dtype=torch.float32, device="cuda")
    sim.set_joint_targets(tg)
    xy = torch.zeros((16, 3), device="cuda")
    xy[:, 0] = 0.3
    xy[:, 2] = 0.7
    sim.set_base_pose(xy)
    s = sim.get_state()
    assert np.allclose(s["joint_target"], b["joint_target"] * 0.5, atol=1e-7)
    k = b["art_off"][:-1]
    assert np.allclose(s["art_base_pos"][k, 0], 0.3) and np.allclose(s["art_base_quat"][k, 0], np.cos(0.35), atol=1e-7)
    err, flips, _, _ = step_both_and_compare(b, sim, orc, nsteps=1)
    assert flips.mean() <= 0.1
    _assert_errors(err)


def test_contact_log_features_match_oracle():
    b = sg.make_batch(2, 32)
    p = sg.params_for(2)
    sim = _engine(b, p, log_features=True)
    orc = O.Oracle(b, p)
    sim.step(25)
    identical_start(sim, orc)
    sim.step(1)
    f, l, n = sim.log_contacts(1 << 14)
    st, of, ol = orc.step_logged()
    f, l = f.cpu().numpy(), l.cpu().numpy()
    gc = sim.contacts()
    go = np.concatenate([[0], np.cumsum(gc["count"])])
    oo = np.concatenate([[0], np.cumsum([len(orc.contacts(e)["sep"]) for e in range(b.n_envs)])])
    assert n == go[-1] and len(of) == oo[-1]
    compared = 0
    for e in range(b.n_envs):
        ok = orc.contacts(e)["key"]
        if gc["count"][e] != len(ok) or not np.array_equal(gc["key"][e, :len(ok)], ok):
            continue
        ge, oe = slice(go[e], go[e + 1]), slice(oo[e], oo[e + 1])
        assert np.abs(f[ge] - of[oe]).max(initial=0) < 1e-3 * max(1, np.abs(of[oe]).max(initial=0))
        assert np.abs(l[ge] - ol[oe]).max(initial=0) < 1e-2 * max(1, np.abs(ol[oe]).max(initial=0))
        compared += go[e + 1] - go[e]
    assert compared > 0.9 * n
