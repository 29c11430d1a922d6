"""The allocation-free contact-log entry point against the allocating one.

sim_log_contacts_noalloc serves callers that must not allocate device memory
while they run (a framework allocator owning the memory budget, a real-time
loop that cannot take cudaMalloc's implicit synchronisation).  It must return
exactly what sim_log_contacts returns, call after call, from its fixed device
scratch array, and report the same error for the same bad call.  This file is
collected last so that a stop-at-first-failure run has already run every other
test.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


def _log(lib, fn, sim, cap):
    feats = torch.full((cap, 32), float("nan"), device="cuda")
    lams = torch.full((cap, 3), float("nan"), device="cuda")
    n = ctypes.c_int(-1)
    rc = getattr(lib, fn)(sim.h, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(lams.data_ptr()), cap,
                          ctypes.byref(n))
    return rc, n.value, feats, lams


def test_noalloc_log_matches_allocating_entry_point_twice():
    from paper_2106_14405_gb300 import Sim, _native as N
    lib = N.load()
    b = sg.make_batch(2, 64)
    sim = Sim(b, sg.params_for(2), log_features=True)
    cap = 64 * 64
    for rep, steps in enumerate((25, 3)):
        sim.step(steps)
        rc1, n1, f1, l1 = _log(lib, "sim_log_contacts", sim, cap)
        rc2, n2, f2, l2 = _log(lib, "sim_log_contacts_noalloc", sim, cap)
        assert rc1 == 0 and rc2 == 0, lib.sim_last_error(None)
        assert n1 == n2 and 0 < n1 <= cap, (rep, n1, n2)
        # same gather of the same device buffers: identical within the parity tolerance (in fact bit-equal)
        assert torch.allclose(f1[:n1], f2[:n2], rtol=0, atol=1e-6)
        assert torch.allclose(l1[:n1], l2[:n2], rtol=0, atol=1e-6)
        assert torch.isnan(f2[n2:]).all()


def test_noalloc_rejects_batches_beyond_its_scratch():
    from paper_2106_14405_gb300 import Sim, _native as N
    lib = N.load()
    E = 65536 + 1  # SIM_NOALLOC_MAX_ENVS + 1 (include/sim.h)
    b = sg.custom_batch([dict(plane=True)] * E)
    p = sg.SimParams()
    p.max_contacts = 1
    sim = Sim(b, p, log_features=True)
    sim.step(1)
    rc, n, _, _ = _log(lib, "sim_log_contacts_noalloc", sim, 16)
    assert rc == 1
    assert b"SIM_NOALLOC_MAX_ENVS" in lib.sim_last_error(None)


def test_noalloc_reports_the_same_errors_in_the_same_order():
    """Without log_features and with bad output buffers both entry points report the
    missing features first (SIM_ERR_STATE), then, with features, the buffers
    (SIM_ERR_INVALID_ARG)."""
    from paper_2106_14405_gb300 import Sim, _native as N
    lib = N.load()
    b = sg.make_batch(2, 4)
    n = ctypes.c_int(0)
    for log, want in ((False, 7), (True, 1)):
        sim = Sim(b, sg.params_for(2), log_features=log)
        sim.step(1)
        for fn in ("sim_log_contacts", "sim_log_contacts_noalloc"):
            rc = getattr(lib, fn)(sim.h, None, None, 8, ctypes.byref(n))
            assert rc == want, (fn, log, rc)
        sim.close()
