"""Fast reset of environment subsets from the device-resident reset template.

A reset environment must hold exactly its template state and then step exactly
as a freshly created environment; the other environments must not change.
"""
import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu

ENV_FIELDS = {  # state field -> per-item class used to find an environment's range
    "obj_pos": "obj", "obj_pos_comp": "obj", "obj_quat": "obj", "obj_vel": "obj", "obj_omega": "obj",
    "obj_awake": "obj", "obj_ctr": "obj", "joint_q": "joint", "joint_q_comp": "joint", "joint_qd": "joint",
    "joint_target": "joint", "joint_lim_lambda": "joint", "joint_lim_side": "joint", "joint_motor_lambda": "joint",
    "art_base_pos": "art",
    "art_base_quat": "art",
}


def _sim(batch, params, **kw):
    from paper_2106_14405_gb300 import Sim
    return Sim(batch, params, **kw)


def _ranges(batch):
    a = batch.arrays
    return {"obj": a["obj_off"], "joint": a["joint_off"][a["art_off"]], "art": a["art_off"]}


def _env_equal(s1, s2, rng, e, fields=ENV_FIELDS):
    for k, cls in fields.items():
        lo, hi = rng[cls][e], rng[cls][e + 1]
        if not np.array_equal(s1[k][lo:hi], s2[k][lo:hi]):
            return False
    return True


def test_reset_envs_restore_template_and_step_like_fresh():
    b = sg.make_batch(3, 512)
    p = sg.params_for(3)
    rng = _ranges(b)
    fresh = _sim(b, p)
    init = fresh.get_state()
    sim = _sim(b, p, use_graph=True)
    sim.step(30)
    before = sim.get_state()
    ids = np.arange(0, 512, 7)
    sim.reset_envs(ids)
    after = sim.get_state()
    reset = np.zeros(512, bool)
    reset[ids] = True
    for e in range(512):
        if reset[e]:
            assert _env_equal(after, init, rng, e), e
            assert after["cache_count"][e] == 0
        else:
            assert _env_equal(after, before, rng, e), e
            assert after["cache_count"][e] == before["cache_count"][e]
    step_f, _ = sim.robot_force()
    # reset envs now evolve exactly as fresh ones
    sim.step(10)
    fresh.step(10)
    a, f = sim.get_state(), fresh.get_state()
    for e in ids:
        assert _env_equal(a, f, rng, e), e
    assert np.array_equal(sim.robot_force()[1][ids], fresh.robot_force()[1][ids])


def test_reset_from_device_list_and_new_template():
    b = sg.make_batch(2, 256)
    p = sg.params_for(2)
    rng = _ranges(b)
    sim = _sim(b, p)
    sim.step(20)
    snap = sim.get_state()
    sim.set_reset_state(snap)  # template := the state after 20 steps
    sim.step(15)
    ids = torch.arange(0, 256, 3, dtype=torch.int32, device="cuda")
    sim.reset_envs(ids)
    torch.cuda.synchronize()
    after = sim.get_state()
    for e in ids.cpu().numpy():
        assert _env_equal(after, snap, rng, e), e
        assert after["cache_count"][e] == 0
    # an out-of-range index in a host list is refused before anything changes
    from paper_2106_14405_gb300 import SimError
    with pytest.raises(SimError):
        sim.reset_envs([1, 256])
    assert _env_equal(sim.get_state(), after, rng, 1)
