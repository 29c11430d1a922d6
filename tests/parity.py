"""Helpers shared by the GPU-vs-oracle parity tests: state transfer between the
two engines and per-environment comparison with decision flips set apart."""
from __future__ import annotations

import numpy as np

import oracle as O

from oracle.compare import ORACLE_FIELDS, gpu_to_oracle  # noqa: E402,F401  (shared with the benchmark's CPU leg)


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


def env_errors(batch, gs, os_, e, go=None, gj=None):
    """Max abs error per quantity for one env of `batch` (oracle side); `go`/`gj` are
    the env's object/joint indices on the GPU side when its batch is larger."""
    oo, jo = env_ranges(batch)
    so, sj = np.arange(oo[e], oo[e + 1]), np.arange(jo[e], jo[e + 1])
    go = so if go is None else go
    gj = sj if gj is None else gj

    def m(a, b):
        return float(np.abs(a.astype(np.float64) - b).max()) if a.size else 0.0

    rev = batch["joint_type"][sj] == 0
    gpos = gs["obj_pos"][go].astype(np.float64) - gs["obj_pos_comp"][go]
    return {"obj_pos": m(gpos, os_["obj_pos"][so]), "obj_vel": m(gs["obj_vel"][go], os_["obj_vel"][so]),
            "obj_omega": m(gs["obj_omega"][go], os_["obj_omega"][so]),
            "joint_qd_revolute": m(gs["joint_qd"][gj][rev], os_["joint_qd"][sj][rev]),
            "joint_qd_prismatic": m(gs["joint_qd"][gj][~rev], os_["joint_qd"][sj][~rev])}


def input_ulp_sensitivity(batch, params, state, nsteps=1, seeds=4, mlp=None):
    """Per env of `batch`, the largest change of the FP64 oracle's result after `nsteps`
    that a one-FP32-ulp relative perturbation of the dynamic state (positions,
    velocities, joint coordinates and rates, +-6e-8) produces over `seeds` draws.

    This is the floor below which no FP32 execution of the method can be held on
    that state: where contact and joint-limit rows couple a light body (a gripper
    finger) to a heavy chain, a fixed number of projected Gauss-Seidel sweeps
    amplifies input rounding far beyond the typical state.  Returns a list of
    per-env dicts shaped like `env_errors`.  `mlp` is the network of the learned
    warm start, where the step uses it."""
    base = O.Oracle(batch, params)
    if mlp is not None:
        base.set_mlp(mlp)
    base.set_state(state)
    base.step(nsteps)
    ref = base.get_state()
    out = [dict.fromkeys(("obj_pos", "obj_vel", "obj_omega", "joint_qd_revolute", "joint_qd_prismatic"), 0.0)
           for _ in range(batch.n_envs)]
    rng = np.random.default_rng(12345)
    for _ in range(seeds):
        sp = {k: v.copy() for k, v in state.items()}
        for k in ("obj_vel", "obj_omega", "joint_qd", "obj_pos", "joint_q"):
            sp[k] = sp[k] * (1 + rng.uniform(-6e-8, 6e-8, sp[k].shape))
        o = O.Oracle(batch, params)
        if mlp is not None:
            o.set_mlp(mlp)
        o.set_state(sp)
        o.step(nsteps)
        got = o.get_state()
        got["obj_pos_comp"] = np.zeros_like(got["obj_pos"])
        for e in range(batch.n_envs):
            d = env_errors(batch, got, ref, e)
            out[e] = {k: max(out[e][k], d[k]) for k in d}
    return out
