"""Python face of the C ABI: `Sim` wraps one handle (argument marshalling only).

PyTorch provides the CUDA stream and device buffers; every step of the physics
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def make_params(p, use_graph: bool = False, log_features: bool = False) -> N.SimParams:
    o = N.SimParams()
    o.dt = p.dt
    o.gravity = (C.c_double * 3)(*p.gravity)
    for k in ("pgs_iters", "pgs_max_iters", "sleep_steps", "sleep_enabled", "warm_mode", "max_contacts"):
        setattr(o, k, int(getattr(p, k)))
    for k in ("pgs_tol", "baumgarte", "slop", "margin", "rest_thresh", "sleep_lin", "sleep_ang", "plane_mu",
              "lambda_floor", "match_dist", "fp64_cond"):
        setattr(o, k, float(getattr(p, k)))
    o.use_graph = int(use_graph)
    o.log_features = int(log_features)
    o.force_limit = float(getattr(p, "force_limit", 0.0))
    o.motor_mode = int(getattr(p, "motor_mode", 0))
    o.motor_kp = float(getattr(p, "motor_kp", 0.3))
    o.motor_max_impulse = float(getattr(p, "motor_max_impulse", 10.0))
    return o


class Sim:
    """Batched physics engine on the current CUDA device.

    batch  : scenegen.Batch (flat CSR scene description, float64 / int32 numpy arrays)
    params : scenegen.SimParams
    stream : torch.cuda.Stream (default: the current stream)
    """

    def __init__(self, batch, params, stream=None, use_graph: bool = False, log_features: bool = False):
        if not torch.cuda.is_available():
            raise RuntimeError("the physics engine needs a CUDA device")
        self.lib = N.load()
        self.batch = batch
        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._use_graph = use_graph
        self._log = log_features
        keep = {k: np.ascontiguousarray(v) for k, v in batch.arrays.items()}
        d = N.SimBatchDesc()
        d.n_envs = batch.n_envs
        for name in N.DESC_FIELDS:
            setattr(d, name, _ptr(keep[name]))
        self._p = make_params(params, use_graph, log_features)
        h = C.c_void_p()
        N.check(self.lib.sim_create(C.byref(d), C.byref(self._p), C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.E = batch.n_envs
        self.C = int(params.max_contacts)
        self.sizes = dict(E=self.E, NO=batch.n_objects, NJ=batch.n_joints, NA=batch.n_arts, EC=self.E * self.C)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- control
    def set_params(self, params, use_graph=None, log_features=None):
        if use_graph is not None:
            self._use_graph = use_graph
        if log_features is not None:
            self._log = log_features
        self.params = params
        self._p = make_params(params, self._use_graph, self._log)
        N.check(self.lib.sim_set_params(self.h, C.byref(self._p)))

    def step(self, n: int = 1):
        N.check(self.lib.sim_step(self.h, int(n)))

    def sync(self):
        st = np.zeros(self.E, np.uint32)
        acc = C.c_uint32(0)
        rc = self.lib.sim_sync(self.h, C.byref(acc), _ptr(st))
        return rc, int(acc.value), st

    def set_joint_targets(self, targets):
        if isinstance(targets, torch.Tensor) and targets.is_cuda:
            t = targets.contiguous().float()
            N.check(self.lib.sim_set_joint_targets(self.h, _ptr(t), 1))
        else:
            t = np.ascontiguousarray(targets, np.float32)
            N.check(self.lib.sim_set_joint_targets(self.h, _ptr(t), 0))

    def set_base_pose(self, xy_yaw):
        if isinstance(xy_yaw, torch.Tensor) and xy_yaw.is_cuda:
            t = xy_yaw.contiguous().float()
            N.check(self.lib.sim_set_base_pose(self.h, _ptr(t), 1))
        else:
            t = np.ascontiguousarray(xy_yaw, np.float32)
            N.check(self.lib.sim_set_base_pose(self.h, _ptr(t), 0))

    # ---- state
    def _alloc_state(self, device: bool, pinned: bool = False):
        out = {}
        for name, kind, w, n in N.STATE_FIELDS:
            if pinned:
                shape = (self.sizes[n], w) if w > 1 else (self.sizes[n],)
                out[name] = torch.zeros(shape, dtype=torch.float32 if kind == "f" else torch.int32,
                                        pin_memory=True).numpy()
                continue
            shape = (self.sizes[n], w) if w > 1 else (self.sizes[n],)
            if device:
                out[name] = torch.zeros(shape, dtype=torch.float32 if kind == "f" else torch.int32, device="cuda")
            else:
                out[name] = np.zeros(shape, np.float32 if kind == "f" else np.int32)
        return out

    def get_state(self, to_device: bool = False, fields=None, out=None) -> dict:
        """Copy the state out (numpy, or torch.cuda tensors with to_device); `fields`
        restricts the copy to some entries; `out` reuses previously returned buffers."""
        s = out if out is not None else self._alloc_state(to_device)
        if fields is not None:
            s = {k: s[k] for k in fields}
        v = N.SimStateView(**{k: _ptr(a) for k, a in s.items()})
        N.check(self.lib.sim_get_state(self.h, C.byref(v), int(to_device)))
        return s

    def set_state(self, s: dict):
        """Host (numpy) or device (torch.cuda) arrays; missing fields are left unchanged."""
        v, on_dev, _keep = self._state_view(s)
        N.check(self.lib.sim_set_state(self.h, C.byref(v), int(bool(on_dev))))

    def set_reset_state(self, s: dict):
        """Replace the reset template (same fields as set_state; cache fields ignored)."""
        v, on_dev, _keep = self._state_view(s)
        N.check(self.lib.sim_set_reset_state(self.h, C.byref(v), int(bool(on_dev))))

    def reset_envs(self, env_ids):
        """Restore the listed environments from the reset template (host list, or a
        torch.cuda int32 tensor for the asynchronous device path)."""
        if isinstance(env_ids, torch.Tensor) and env_ids.is_cuda:
            ids = env_ids.contiguous().to(torch.int32)
            N.check(self.lib.sim_reset_envs(self.h, _ptr(ids), int(ids.numel()), 1))
        else:
            ids = np.ascontiguousarray(env_ids, np.int32)
            N.check(self.lib.sim_reset_envs(self.h, _ptr(ids) if len(ids) else None, len(ids), 0))

    def _state_view(self, s: dict):
        conv = {}
        on_dev = None
        for name, kind, w, n in N.STATE_FIELDS:
            if name not in s:
                continue
            a = s[name]
            dev = isinstance(a, torch.Tensor) and a.is_cuda
            on_dev = dev if on_dev is None else on_dev
            if dev != on_dev:
                raise ValueError("set_state: mix of host and device arrays")
            if dev:
                conv[name] = a.contiguous().to(torch.float32 if kind == "f" else torch.int32)
            else:
                conv[name] = np.ascontiguousarray(a, np.float32 if kind == "f" else np.int32)
        v = N.SimStateView(**{k: _ptr(a) for k, a in conv.items()})
        return v, on_dev, conv

    # ---- diagnostics
    def stats(self) -> dict:
        E = self.E
        out = dict(status=np.zeros(E, np.int32), iters=np.zeros(E, np.int32), resid=np.zeros(E, np.float32),
                   n_contacts=np.zeros(E, np.int32), n_rows=np.zeros(E, np.int32),
                   n_limit_rows=np.zeros(E, np.int32), n_colours=np.zeros(E, np.int32),
                   fp64_used=np.zeros(E, np.int32))
        N.check(self.lib.sim_get_env_stats(self.h, *[_ptr(out[k]) for k in (
            "status", "iters", "resid", "n_contacts", "n_rows", "n_limit_rows", "n_colours", "fp64_used")], 0))
        return out

    def contacts(self) -> dict:
        E, Cc = self.E, self.C
        out = dict(count=np.zeros(E, np.int32), key=np.zeros((E, Cc, 3), np.int32), p=np.zeros((E, Cc, 3), np.float32),
                   n=np.zeros((E, Cc, 3), np.float32), sep=np.zeros((E, Cc), np.float32),
                   lam=np.zeros((E, Cc, 3), np.float32))
        N.check(self.lib.sim_get_contacts(self.h, *[_ptr(out[k]) for k in ("count", "key", "p", "n", "sep", "lam")], 0))
        return out

    def contact_keys(self):
        """Contact count per env [E] and keys (a, b, feature) [E][C][3] of the last step."""
        E, Cc = self.E, self.C
        count, key = np.zeros(E, np.int32), np.zeros((E, Cc, 3), np.int32)
        N.check(self.lib.sim_get_contacts(self.h, _ptr(count), _ptr(key), None, None, None, None, 0))
        return {"count": count, "key": key}

    def pairs(self, cap: int = 256):
        count = np.zeros(self.E, np.int32)
        pairs = np.zeros((self.E, cap), np.int32)
        N.check(self.lib.sim_get_pairs(self.h, cap, _ptr(count), _ptr(pairs), 0))
        return count, pairs

    def articulation(self) -> dict:
        NJ, NA = self.sizes["NJ"], self.sizes["NA"]
        out = dict(com=np.zeros((NJ, 3), np.float32), rot=np.zeros((NJ, 3, 3), np.float32),
                   qdd=np.zeros(NJ, np.float32), minv=np.zeros((NA, 9, 9), np.float32))
        N.check(self.lib.sim_get_articulation(self.h, *[_ptr(out[k]) for k in ("com", "rot", "qdd", "minv")], 0))
        return out

    # ---- timing
    def set_profiling(self, on):
        """True / 1: events around every kernel of each step; "pgs" / 2: around the
        PGS kernel only (lighter); False / 0: off."""
        N.check(self.lib.sim_set_profiling(self.h, 2 if on == "pgs" else int(on)))

    def kernel_times(self):
        """Summed device ms per stage of the last step call and launches per stage."""
        names = ("aba", "collide", "rows", "mlp", "lpt", "pgs", "integrate")
        ms = (C.c_float * len(names))()
        ln = (C.c_int * len(names))()
        N.check(self.lib.sim_kernel_times(self.h, ms, ln))
        return dict(zip(names, list(ms))), dict(zip(names, list(ln)))

    # ---- contact force on the robot
    def robot_force(self):
        """(this step's, accumulated) contact force on the robot per env (N), host arrays."""
        step, acc = np.zeros(self.E, np.float32), np.zeros(self.E, np.float32)
        N.check(self.lib.sim_get_robot_force(self.h, _ptr(step), _ptr(acc), 0))
        return step, acc

    def reset_robot_force(self, env_ids=None):
        if env_ids is None:
            N.check(self.lib.sim_reset_robot_force(self.h, None, 0, 0))
        else:
            ids = np.ascontiguousarray(env_ids, np.int32)
            N.check(self.lib.sim_reset_robot_force(self.h, _ptr(ids), len(ids), 0))

    # ---- launch shapes
    def launch_shape(self) -> dict:
        k = N.SimLaunchShape()
        N.check(self.lib.sim_get_launch_shape(self.h, C.byref(k)))
        return {n: int(getattr(k, n)) for n in N.SHAPE_FIELDS}

    def set_launch_shape(self, **fields):
        """Change some fields of the current launch shape (see sim_set_launch_shape)."""
        cur = self.launch_shape()
        unknown = set(fields) - set(cur)
        if unknown:
            raise ValueError(f"unknown launch-shape fields {sorted(unknown)}")
        cur.update(fields)
        k = N.SimLaunchShape(**cur)
        N.check(self.lib.sim_set_launch_shape(self.h, C.byref(k)))

    def autotune(self, steps_per_trial: int = 2, rounds: int = 3) -> dict:
        """Run the library's autotuner (advances the batch by the returned steps_taken
        physics steps) and return the chosen shape with every trial's stage times."""
        k = N.SimLaunchShape()
        rep = N.SimTuneReport()
        N.check(self.lib.sim_autotune(self.h, int(steps_per_trial), int(rounds), C.byref(k), C.byref(rep)))
        trials = []
        for t in range(rep.n_trials):
            sh = {n: int(getattr(rep.trial[t], n)) for n in N.SHAPE_FIELDS}
            trials.append({"shape": sh, "ms": [float(x) for x in rep.ms[t]]})
        return {"chosen": {n: int(getattr(k, n)) for n in N.SHAPE_FIELDS},
                "chosen_ms": {"collide": float(rep.chosen_ms[0]), "rows": float(rep.chosen_ms[1]),
                              "pgs": float(rep.chosen_ms[2]), "step": float(rep.chosen_ms[3]),
                              "aba": float(rep.chosen_ms[4])},
                "steps_taken": int(rep.steps_taken), "trials": trials}

    def launch_count(self) -> int:
        n = C.c_longlong(0)
        N.check(self.lib.sim_launch_count(self.h, C.byref(n)))
        return int(n.value)

    def totals(self) -> dict:
        """Batch totals of the last step (sim_get_stats)."""
        o = N.SimStats()
        N.check(self.lib.sim_get_stats(self.h, C.byref(o)))
        return {k: getattr(o, k) for k, _ in N.SimStats._fields_}

    # ---- learned warm start
    def set_warm_start(self, mode, params=None):
        """Warm start of the solver: "cold" / "prior" / "learned" (or 0 / 1 / 2); `params`
        loads the learned network (host array or torch.cuda tensor)."""
        m = {"cold": 0, "prior": 1, "learned": 2}.get(mode, mode)
        if params is None:
            N.check(self.lib.sim_set_warm_start(self.h, int(m), None, 0))
        elif isinstance(params, torch.Tensor) and params.is_cuda:
            p = params.contiguous().float()
            N.check(self.lib.sim_set_warm_start(self.h, int(m), _ptr(p), 1))
        else:
            p = np.ascontiguousarray(params, np.float32)
            N.check(self.lib.sim_set_warm_start(self.h, int(m), _ptr(p), 0))
        self._p.warm_mode = int(m)

    def set_mlp(self, params):
        if params is None:
            N.check(self.lib.sim_set_mlp(self.h, None, 0))
            return
        if isinstance(params, torch.Tensor) and params.is_cuda:
            p = params.contiguous().float()
            N.check(self.lib.sim_set_mlp(self.h, _ptr(p), 1))
        else:
            p = np.ascontiguousarray(params, np.float32)
            N.check(self.lib.sim_set_mlp(self.h, _ptr(p), 0))

    def debug_hold_async(self, on: bool):
        """Testing: withhold the step's asynchronous completions so that its bounded
        device waits run out (see sim_debug_hold_async)."""
        N.check(self.lib.sim_debug_hold_async(self.h, int(bool(on))))

    def log_predictions(self, cap: int):
        """The learned warm start's network outputs of the last step (warm_mode 2), per
        contact in env then contact order: (device tensor [min(cap, n)][3], n)."""
        preds = torch.empty((cap, 3), dtype=torch.float32, device="cuda")
        n = C.c_int(0)
        N.check(self.lib.sim_log_predictions(self.h, _ptr(preds), int(cap), C.byref(n)))
        return preds[:min(cap, n.value)], n.value

    def log_contacts(self, cap: int):
        feats = torch.empty((cap, 32), dtype=torch.float32, device="cuda")
        lams = torch.empty((cap, 3), dtype=torch.float32, device="cuda")
        n = C.c_int(0)
        N.check(self.lib.sim_log_contacts(self.h, _ptr(feats), _ptr(lams), int(cap), C.byref(n)))
        m = min(cap, n.value)
        return feats[:m], lams[:m], n.value


def fp32_fma_peak(iters: int = 4096, reps: int = 5, stream=None):
    """The library's FP32 FMA throughput probe on the current device: (TFLOP/s, ms)."""
    lib = N.load()
    st = stream if stream is not None else torch.cuda.current_stream()
    t = C.c_double(0.0)
    ms = C.c_double(0.0)
    N.check(lib.sim_fp32_fma_peak(C.c_void_p(st.cuda_stream), int(iters), int(reps), C.byref(t), C.byref(ms)))
    return t.value, ms.value
