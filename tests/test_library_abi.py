"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function that include/sim.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*((?:sim|mlp)_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sim_create", "sim_set_joint_targets", "sim_step", "sim_get_state", "sim_set_state", "sim_sync",
              "sim_destroy", "sim_set_mlp", "sim_log_contacts", "sim_last_error"):
        assert n in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2106_14405_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_2106_14405_gb300 import _native
    assert set(_native.EXPORTS) <= set(declared_functions())


def test_invalid_description_is_rejected_without_a_gpu():
    """sim_create validates the description before touching the device."""
    import numpy as np
    import scenegen as sg
    from paper_2106_14405_gb300 import _native as N
    from paper_2106_14405_gb300.engine import make_params, _ptr
    lib = N.load()
    b = sg.make_batch(2, 2)
    keep = {k: np.ascontiguousarray(v) for k, v in b.arrays.items()}
    keep["obj_mass"] = keep["obj_mass"].copy()
    keep["obj_mass"][0] = -1.0
    d = N.SimBatchDesc()
    d.n_envs = b.n_envs
    for name in N.DESC_FIELDS:
        setattr(d, name, _ptr(keep[name]))
    p = make_params(sg.params_for(2))
    h = ctypes.c_void_p()
    rc = lib.sim_create(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"obj_mass" in lib.sim_last_error(None)
    p.max_contacts = 100000
    keep["obj_mass"][0] = 1.0
    rc = lib.sim_create(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h))
    assert rc == 1 and b"max_contacts" in lib.sim_last_error(None)


def test_package_refuses_to_run_without_cuda(monkeypatch):
    import torch
    import scenegen as sg
    from paper_2106_14405_gb300 import Sim
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    with pytest.raises(RuntimeError, match="CUDA"):
        Sim(sg.make_batch(1, 2), sg.params_for(1))
