"""Helpers shared by the GPU-vs-oracle parity tests: state transfer between the
two engines and per-environment comparison with decision flips set apart."""
from __future__ import annotations

import numpy as np

import oracle as O

ORACLE_FIELDS = ("obj_pos", "obj_quat", "obj_vel", "obj_omega", "obj_awake", "obj_ctr", "joint_q", "joint_qd",
                 "joint_target", "art_base_pos", "art_base_quat", "joint_lim_lambda", "joint_lim_side",
                 "cache_count", "cache_key", "cache_p", "cache_lambda", "joint_motor_lambda")


def gpu_to_oracle(gs: dict) -> dict:
    """GPU state (float32) -> oracle state (float64, same values)."""
    out = {}
    for k in ORACLE_FIELDS:
        a = gs[k]
        out[k] = a.astype(np.int32) if a.dtype.kind in "iu" else a.astype(np.float64)
    return out


def identical_start(sim, orc):
    """Make both engines hold the GPU's current state exactly (Kahan compensations cleared)."""
    gs = sim.get_state()
    gs["obj_pos_comp"][:] = 0
    gs["joint_q_comp"][:] = 0
    sim.set_state({"obj_pos_comp": gs["obj_pos_comp"], "joint_q_comp": gs["joint_q_comp"]})
    orc.set_state(gpu_to_oracle(gs))
    return gs


def env_ranges(batch):
    a = batch.arrays
    jo = a["joint_off"][a["art_off"]]
    return a["obj_off"], jo


def decision_flips(batch, sim, orc, gs_after, os_after, gpu_contacts=None, compare_iters=False):
    """Per-env boolean: discrete decisions (contact keys, limit rows, awake flags, PGS
    sweep count when residual-driven) differ between the engines."""
    E = batch.n_envs
    oo, jo = env_ranges(batch)
    gc = gpu_contacts if gpu_contacts is not None else sim.contacts()
    flips = np.zeros(E, bool)
    gst = sim.stats()
    ost = orc.stats()
    for e in range(E):
        oc = orc.contacts(e)
        n = gc["count"][e]
        if n != len(oc["sep"]) or not np.array_equal(gc["key"][e, :n], oc["key"]):
            flips[e] = True
            continue
        if not np.array_equal(gs_after["obj_awake"][oo[e]:oo[e + 1]], os_after["obj_awake"][oo[e]:oo[e + 1]]):
            flips[e] = True
            continue
        if not np.array_equal(gs_after["joint_lim_side"][jo[e]:jo[e + 1]], os_after["joint_lim_side"][jo[e]:jo[e + 1]]):
            flips[e] = True
            continue
        if gst["n_colours"][e] != ost["n_colours"][e]:
            flips[e] = True
            continue
        if compare_iters and gst["iters"][e] != ost["iters"][e]:
            flips[e] = True
    return flips


def state_errors(batch, gs, os_, envs):
    """Max abs error per quantity over the given envs (positions m, angles rad, velocities m/s)."""
    oo, jo = env_ranges(batch)
    oi = np.concatenate([np.arange(oo[e], oo[e + 1]) for e in envs]) if len(envs) else np.zeros(0, int)
    ji = np.concatenate([np.arange(jo[e], jo[e + 1]) for e in envs]) if len(envs) else np.zeros(0, int)
    err = {}

    def m(a, b):
        return float(np.abs(a.astype(np.float64) - b).max()) if a.size else 0.0

    gpos = gs["obj_pos"].astype(np.float64) - gs["obj_pos_comp"].astype(np.float64)
    err["obj_pos"] = m(gpos[oi], os_["obj_pos"][oi])
    err["obj_vel"] = m(gs["obj_vel"][oi], os_["obj_vel"][oi])
    err["obj_omega"] = m(gs["obj_omega"][oi], os_["obj_omega"][oi])
    err["obj_quat"] = m(gs["obj_quat"][oi], os_["obj_quat"][oi])
    gq = gs["joint_q"].astype(np.float64) - gs["joint_q_comp"].astype(np.float64)
    err["joint_q"] = m(gq[ji], os_["joint_q"][ji])
    rev = batch["joint_type"][ji] == 0
    err["joint_qd_revolute"] = m(gs["joint_qd"][ji][rev], os_["joint_qd"][ji][rev])
    err["joint_qd_prismatic"] = m(gs["joint_qd"][ji][~rev], os_["joint_qd"][ji][~rev])
    return err


def step_both_and_compare(batch, sim, orc, nsteps=1, compare_iters=False):
    """From an identical state, advance both engines and compare; returns (errors, flips)."""
    identical_start(sim, orc)
    sim.step(nsteps)
    rc, acc, _ = sim.sync()
    orc.step(nsteps)
    gs = sim.get_state()
    os_ = orc.get_state()
    flips = decision_flips(batch, sim, orc, gs, os_, compare_iters=compare_iters)
    ok = np.nonzero(~flips)[0]
    return state_errors(batch, gs, os_, ok), flips, gs, os_
