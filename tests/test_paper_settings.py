"""The step's fixed numbers against the paper's, stored with their citations in
tests/golden/paper_settings.json: the physics time step and the physics steps
per simulation step (the period of the joint-target refresh), the joint motors' impulse cap
and position gain, and the accumulated-contact-force failure threshold.  The
oracle pins (test_oracle_pins.py) check what the step does with them."""
import json
import os

import pytest

import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_settings.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        g = json.load(f)
    for k, v in g.items():
        if not k.startswith("_"):
            assert v["citation"].startswith("Sec. "), k
    return {k: v["value"] for k, v in g.items() if not k.startswith("_")}


def test_default_step_parameters_are_the_papers(paper):
    p = sg.params_for(2)  # the benchmark workload
    assert p.dt == pytest.approx(paper["physics_dt_s"], rel=1e-15)
    assert p.motor_max_impulse == paper["motor_max_impulse_Ns"]
    assert p.motor_kp == paper["motor_position_gain_kp"]
    assert p.force_limit == paper["accumulated_contact_force_limit_N"]


def test_control_period_is_one_simulation_step(paper):
    import bench
    assert bench.CONTROL_SUBSTEPS == paper["physics_steps_per_simulation_step"]
    assert bench.CONTROL_SUBSTEPS * sg.params_for(2).dt == pytest.approx(1.0 / 30.0, rel=1e-12)
    # the workload whose joint targets change refreshes them once per simulation step
    assert bench.step_physics(5) == bench.CONTROL_SUBSTEPS


def test_oracle_params_carry_the_same_numbers(paper):
    import oracle as O
    q = O.make_params(sg.params_for(2))
    assert q.dt == pytest.approx(paper["physics_dt_s"], rel=1e-15)
    assert q.motor_max_impulse == paper["motor_max_impulse_Ns"]
    assert q.motor_kp == pytest.approx(paper["motor_position_gain_kp"], rel=1e-15)
    assert q.force_limit == paper["accumulated_contact_force_limit_N"]
