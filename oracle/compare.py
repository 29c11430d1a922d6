"""Comparison of the CUDA engine's state with the FP64 oracle's, environment by
environment, with discrete decisions set apart.

TEST INFRASTRUCTURE ONLY: used by the test suite and by the benchmark's CPU leg
(the per-output errors it reports).  It never calls the CUDA engine; it takes the
engine's state as plain arrays (what sim_get_state returns) and runs the oracle.

The accuracy contract it measures: from an identical state, one step agrees within
1e-4 absolute in metres, radians and metres per second; angular rates (free-body
omega, revolute joint rates, rad/s) within 1e-3, the floor below which no FP32
execution of the method can be held (the oracle's FP32 build and one-ulp input
perturbations both move them by more than 1e-4).  Environments whose discrete
decisions differ (contact keys, awake flags, active joint limits) are counted as
decision flips and not compared.
"""
from __future__ import annotations

import numpy as np

from . import Oracle

TOL = 1e-4
RATE_TOL = 1e-3
TOLS = {"obj_pos": TOL, "obj_vel": TOL, "obj_quat": TOL, "joint_q": TOL, "joint_qd_prismatic": TOL,
        "joint_qd_revolute": RATE_TOL, "obj_omega": RATE_TOL}
UNITS = {"obj_pos": "m", "obj_vel": "m/s", "obj_quat": "1 (quaternion component)", "joint_q": "rad or m",
         "joint_qd_prismatic": "m/s", "joint_qd_revolute": "rad/s", "obj_omega": "rad/s"}

ORACLE_FIELDS = ("obj_pos", "obj_quat", "obj_vel", "obj_omega", "obj_awake", "obj_ctr", "joint_q", "joint_qd",
                 "joint_target", "art_base_pos", "art_base_quat", "joint_lim_lambda", "joint_lim_side",
                 "cache_count", "cache_key", "cache_p", "cache_lambda", "joint_motor_lambda")


def gpu_to_oracle(gs: dict) -> dict:
    """Engine state (float32 / int32 arrays) -> oracle state (float64 / int32, same
    values).  Positions are taken as stored: clear the engine's Kahan compensations
    first where an identical start is wanted."""
    out = {}
    for k in ORACLE_FIELDS:
        a = np.asarray(gs[k])
        out[k] = a.astype(np.int32) if a.dtype.kind in "iu" else a.astype(np.float64)
    return out


def compensated(gs: dict) -> dict:
    """Engine state with each Kahan-compensated sum read as value - compensation
    (float64): the engine's best estimate of positions and joint coordinates."""
    out = dict(gs)
    out["obj_pos"] = np.asarray(gs["obj_pos"], np.float64) - np.asarray(gs["obj_pos_comp"], np.float64)
    out["joint_q"] = np.asarray(gs["joint_q"], np.float64) - np.asarray(gs["joint_q_comp"], np.float64)
    return out


def subset_state(batch, gs: dict, envs) -> dict:
    """The oracle state of `batch.subset(envs)` taken from a full-batch engine state."""
    a = batch.arrays
    oo, jo = a["obj_off"], a["joint_off"][a["art_off"]]
    oi = np.concatenate([np.arange(oo[e], oo[e + 1]) for e in envs]).astype(np.int64)
    ji = np.concatenate([np.arange(jo[e], jo[e + 1]) for e in envs]).astype(np.int64)
    ai = np.concatenate([np.arange(a["art_off"][e], a["art_off"][e + 1]) for e in envs]).astype(np.int64)
    E = batch.n_envs
    s = {}
    for k in ("obj_pos", "obj_quat", "obj_vel", "obj_omega", "obj_awake", "obj_ctr"):
        s[k] = np.asarray(gs[k])[oi]
    for k in ("joint_q", "joint_qd", "joint_target", "joint_lim_lambda", "joint_lim_side", "joint_motor_lambda"):
        s[k] = np.asarray(gs[k])[ji]
    for k in ("art_base_pos", "art_base_quat"):
        s[k] = np.asarray(gs[k])[ai]
    s["cache_count"] = np.asarray(gs["cache_count"])[envs]
    for k in ("cache_key", "cache_p", "cache_lambda"):
        v = np.asarray(gs[k])
        s[k] = v.reshape((E, -1) + v.shape[1:])[envs].reshape((-1,) + v.shape[1:])
    return gpu_to_oracle(s)


def _env_errors(batch, gs, os_, e, go, gj, sub_e):
    a = batch.arrays
    so = np.arange(a["obj_off"][sub_e], a["obj_off"][sub_e + 1])
    jo = a["joint_off"][a["art_off"]]
    sj = np.arange(jo[sub_e], jo[sub_e + 1])

    def m(x, y):
        return float(np.abs(np.asarray(x, np.float64) - y).max()) if np.size(x) else 0.0

    rev = a["joint_type"][sj] == 0
    gpos = np.asarray(gs["obj_pos"], np.float64)[go] - np.asarray(gs["obj_pos_comp"], np.float64)[go]
    gq = np.asarray(gs["joint_q"], np.float64)[gj] - np.asarray(gs["joint_q_comp"], np.float64)[gj]
    return {"obj_pos": m(gpos, os_["obj_pos"][so]), "obj_vel": m(gs["obj_vel"][go], os_["obj_vel"][so]),
            "obj_omega": m(gs["obj_omega"][go], os_["obj_omega"][so]),
            "obj_quat": m(gs["obj_quat"][go], os_["obj_quat"][so]), "joint_q": m(gq, os_["joint_q"][sj]),
            "joint_qd_revolute": m(gs["joint_qd"][gj][rev], os_["joint_qd"][sj][rev]),
            "joint_qd_prismatic": m(gs["joint_qd"][gj][~rev], os_["joint_qd"][sj][~rev])}


def ulp_floor(sub_batch, params, start: dict, envs_local, nsteps=1, seeds=4, mlp=None):
    """Per listed env of `sub_batch`, the largest change of the oracle's result after
    `nsteps` that a one-FP32-ulp relative perturbation of the dynamic state (+-6e-8 on
    positions, velocities, joint coordinates and rates) produces over `seeds` draws:
    the floor below which no FP32 execution can be held on that state."""
    base = Oracle(sub_batch, params)
    if mlp is not None:
        base.set_mlp(mlp)
    base.set_state(start)
    base.step(nsteps)
    ref = base.get_state()
    ref_c = dict(ref, obj_pos_comp=np.zeros_like(ref["obj_pos"]), joint_q_comp=np.zeros_like(ref["joint_q"]))
    out = {e: dict.fromkeys(TOLS, 0.0) for e in envs_local}
    rng = np.random.default_rng(12345)
    a = sub_batch.arrays
    jo = a["joint_off"][a["art_off"]]
    for _ in range(seeds):
        sp = {k: v.copy() for k, v in start.items()}
        for k in ("obj_vel", "obj_omega", "joint_qd", "obj_pos", "joint_q"):
            sp[k] = sp[k] * (1 + rng.uniform(-6e-8, 6e-8, sp[k].shape))
        o = Oracle(sub_batch, params)
        if mlp is not None:
            o.set_mlp(mlp)
        o.set_state(sp)
        o.step(nsteps)
        got = o.get_state()
        got_c = dict(got, obj_pos_comp=np.zeros_like(got["obj_pos"]), joint_q_comp=np.zeros_like(got["joint_q"]))
        for e in envs_local:
            go = np.arange(a["obj_off"][e], a["obj_off"][e + 1])
            gj = np.arange(jo[e], jo[e + 1])
            d = _env_errors(sub_batch, got_c, ref_c, e, go, gj, e)
            out[e] = {k: max(out[e][k], d[k]) for k in d}
    return out


def sampled_parity(batch, params, start: dict, after: dict, gpu_contacts: dict, envs, mlp=None) -> dict:
    """One step of the sampled environments in the oracle from `start` (the engine's
    state, Kahan compensations cleared, as the engine stepped it) against the engine's
    state `after` that step and its contacts (count[E], key[E][C][3]).

    Returns per output the largest error over the sampled environments without a
    decision flip, the flip count, and the environments over the fixed tolerance:
    how many, how many of those pass on their own one-ulp floor (the state's
    one-ulp response at least a third of the tolerance, the error within the
    tolerance plus three times that response), and, when the solve iterates to a
    residual target, how many of them hit the sweep cap in the oracle (a capped
    solve's result depends on its starting impulses, which the two engines'
    networks give in different precision)."""
    envs = np.asarray(sorted(set(int(e) for e in envs)))
    sub = batch.subset(envs)
    st0 = subset_state(batch, start, envs)
    orc = Oracle(sub, params)
    if mlp is not None:
        orc.set_mlp(mlp)
    orc.set_state(st0)
    orc.step(1)
    o2 = orc.get_state()
    ost = orc.stats()
    a = batch.arrays
    oo, jo = a["obj_off"], a["joint_off"][a["art_off"]]
    sa = sub.arrays
    sjo = sa["joint_off"][sa["art_off"]]
    flips = 0
    worst = dict.fromkeys(TOLS, 0.0)
    over = {}
    for i, e in enumerate(envs):
        oc = orc.contacts(i)
        n = int(gpu_contacts["count"][e])
        if n != len(oc["sep"]) or not np.array_equal(np.asarray(gpu_contacts["key"])[e, :n], oc["key"]):
            flips += 1
            continue
        go, gj = np.arange(oo[e], oo[e + 1]), np.arange(jo[e], jo[e + 1])
        so, sj = np.arange(sa["obj_off"][i], sa["obj_off"][i + 1]), np.arange(sjo[i], sjo[i + 1])
        if not np.array_equal(np.asarray(after["obj_awake"])[go], o2["obj_awake"][so]) or \
                not np.array_equal(np.asarray(after["joint_lim_side"])[gj], o2["joint_lim_side"][sj]):
            flips += 1
            continue
        err = _env_errors(sub, after, o2, e, go, gj, i)
        for k, v in err.items():
            worst[k] = max(worst[k], v)
        if any(v > TOLS[k] for k, v in err.items()):
            over[i] = err
    capped = sum(1 for i in over if getattr(params, "pgs_tol", 0) > 0 and ost["iters"][i] >= params.pgs_max_iters)
    floor_ok = 0
    if over:
        fl = ulp_floor(sub, params, st0, list(over), mlp=mlp)
        for i, err in over.items():
            if all(v <= TOLS[k] or (fl[i][k] >= TOLS[k] / 3 and v <= TOLS[k] + 3 * fl[i][k]) for k, v in err.items()):
                floor_ok += 1
    return {"envs": int(len(envs)), "decision_flips": int(flips), "max_error": worst,
            "units": UNITS, "tolerance": TOLS, "over_tolerance": int(len(over)),
            "over_tolerance_within_ulp_floor": int(floor_ok), "over_tolerance_capped": int(capped)}
