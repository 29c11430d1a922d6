"""Derivation of the parity tolerances from the arithmetic (oracle only, CPU).

The GPU engine computes in FP32.  Two measurements bound what any FP32
execution of this method can achieve against the FP64 oracle after one step
from an identical (FP32-representable) state:

  1. the same algorithm compiled in single precision (liboracle_f32), and
  2. the FP64 oracle with its inputs perturbed by one FP32 ulp (6e-8 relative).

Positions (m), angles (rad), linear velocities (m/s) and prismatic joint rates
(m/s) stay well inside 1e-4, so the parity tests hold them to 1e-4.  Angular
velocities of small tumbling boxes (inverse inertia up to ~2e4 / (kg m^2))
exceed 1e-4 rad/s in both measurements, so no FP32 engine meets 1e-4 there:
the parity tests hold angular rates (free-body omega, revolute joint rates) to
1e-3 rad/s, at least 3x the floors measured here.
"""
import numpy as np
import pytest

import oracle as O
import scenegen as sg

TOL = 1e-4
RATE_TOL = 1e-3
SCENES = ((2, 64, 40), (3, 48, 30), (5, 24, 40))


def _fp32_state(o):
    return {k: (v.astype(np.float32).astype(np.float64) if v.dtype.kind == "f" else v)
            for k, v in o.get_state().items()}


def _deviation(a, c, rev):
    d = {k: float(np.abs(a[k] - c[k]).max()) for k in ("obj_pos", "obj_vel", "obj_omega", "joint_q")}
    dq = np.abs(a["joint_qd"] - c["joint_qd"])
    d["qd_revolute"] = float(dq[rev].max())
    d["qd_prismatic"] = float(dq[~rev].max())
    return d



@pytest.mark.parametrize("cfg,n,warm", SCENES)
def test_fp32_floor_of_the_algorithm(cfg, n, warm):
    b = sg.make_batch(cfg, n)
    p = sg.params_for(cfg)
    o = O.Oracle(b, p)
    o.step(warm)
    s = _fp32_state(o)
    o.set_state(s)
    o.step(1)
    ref = o.get_state()
    f = O.Oracle(b, p, fp32=True)
    f.set_state(s)
    f.step(1)
    d = _deviation(ref, f.get_state(), b["joint_type"] == 0)
    assert d["obj_pos"] < 1e-6 and d["joint_q"] < 1e-5
    assert d["obj_vel"] < TOL / 3 and d["qd_prismatic"] < TOL / 3
    assert d["obj_omega"] < RATE_TOL / 3 and d["qd_revolute"] < RATE_TOL / 3



def test_angular_rates_exceed_1e4_in_fp32():
    worst = 0.0
    for cfg, n, warm in SCENES:
        b = sg.make_batch(cfg, n)
        p = sg.params_for(cfg)
        o = O.Oracle(b, p)
        o.step(warm)
        s = _fp32_state(o)
        o.set_state(s)
        o.step(1)
        ref = o.get_state()
        f = O.Oracle(b, p, fp32=True)
        f.set_state(s)
        f.step(1)
        worst = max(worst, float(np.abs(ref["obj_omega"] - f.get_state()["obj_omega"]).max()))
        # one FP32 ulp of input moves the FP64 result by a comparable amount
        rng = np.random.default_rng(0)
        sp = {k: v.copy() for k, v in s.items()}
        for k in ("obj_vel", "obj_omega", "joint_qd", "obj_pos", "joint_q"):
            sp[k] = sp[k] * (1 + rng.uniform(-6e-8, 6e-8, sp[k].shape))
        o.set_state(sp)
        o.step(1)
        worst = max(worst, float(np.abs(o.get_state()["obj_omega"] - ref["obj_omega"]).max()))
    assert worst > TOL
    assert worst < RATE_TOL / 3
