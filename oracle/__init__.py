"""ctypes front end of the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  Nothing here touches the
CUDA engine; both consume the same scene batches from `scenegen`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
# a directory of prebuilt oracle libraries to load instead (used by the test that
# plants mistakes in a copy of the source); nothing is rebuilt from it
_LIBDIR_OVERRIDE = os.environ.get("ORACLE_LIBDIR")
_SRC = os.path.join(_HERE, "oracle.cpp")
_libs: dict = {}
_lock = threading.Lock()

MLP_IN = 32
MLP_H = 128
MLP_OUT = 3
STAGES = ("aba", "predict", "collide", "rows", "pgs", "integrate", "mlp")


def build(force: bool = False) -> None:
    """Compile liboracle.so, the op-counting liboracle_count.so and the single-precision
    liboracle_f32.so (g++, no GPU)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    jobs = []
    for name, extra in (("liboracle.so", []), ("liboracle_count.so", ["-DORACLE_COUNT_OPS"]),
                        ("liboracle_f32.so", ["-DORACLE_FP32"])):
        out = os.path.join(_LIBDIR, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", *extra, _SRC, "-o", out + ".tmp", "-lpthread"]
        jobs.append((subprocess.Popen(cmd), out))
    for p, out in jobs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed")
        os.replace(out + ".tmp", out)


def _lib(counting: bool = False, fp32: bool = False):
    name = "liboracle_count.so" if counting else ("liboracle_f32.so" if fp32 else "liboracle.so")
    with _lock:
        if name not in _libs:
            if _LIBDIR_OVERRIDE:
                path = os.path.join(_LIBDIR_OVERRIDE, name)
                if not os.path.exists(path):
                    raise RuntimeError(f"no {name} in ORACLE_LIBDIR={_LIBDIR_OVERRIDE}")
            else:
                path = os.path.join(_LIBDIR, name)
                if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
                    build()
            lib = C.CDLL(path)
            lib.oracle_create.restype = C.c_void_p
            lib.oracle_create.argtypes = [C.c_void_p, C.c_void_p]
            lib.oracle_destroy.argtypes = [C.c_void_p]
            lib.oracle_step.argtypes = [C.c_void_p, C.c_int, C.c_int]
            lib.oracle_step_logged.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
            lib.oracle_set_params.argtypes = [C.c_void_p, C.c_void_p]
            lib.oracle_get_state.argtypes = [C.c_void_p, C.c_void_p]
            lib.oracle_set_state.argtypes = [C.c_void_p, C.c_void_p]
            lib.oracle_get_stats.argtypes = [C.c_void_p] + [C.c_void_p] * 7
            lib.oracle_get_contacts.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 5
            lib.oracle_get_pairs.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
            lib.oracle_get_colouring.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 3
            lib.oracle_articulation.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 5
            lib.oracle_dynamics_check.argtypes = [C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 5
            lib.oracle_narrowphase.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_int]
            lib.oracle_mlp_nparam.restype = C.c_int
            lib.oracle_set_mlp.argtypes = [C.c_void_p, C.c_void_p]
            lib.oracle_mlp_forward.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            lib.oracle_mlp_loss_grad.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_mlp_loss_grad.restype = C.c_double
            lib.oracle_get_op_counts.argtypes = [C.c_void_p]
            lib.oracle_get_robot_force.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_reset_robot_force.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
            _libs[name] = lib
        return _libs[name]


class OrDesc(C.Structure):
    _fields_ = [("n_envs", C.c_int)] + [(n, C.c_void_p) for n in (
        "obj_off", "obj_shape", "obj_half", "obj_mass", "obj_mu", "obj_rest", "obj_pos", "obj_quat", "obj_vel",
        "obj_omega", "stat_off", "stat_pos", "stat_quat", "stat_half", "stat_mu", "art_off", "joint_off",
        "art_base_pos", "art_base_quat", "art_has_base_coll", "art_base_coll_off", "art_base_coll_half",
        "art_kinematic", "joint_parent", "joint_type", "joint_axis", "joint_origin_pos", "joint_origin_quat",
        "joint_com", "joint_half", "joint_mass", "joint_lo", "joint_hi", "joint_has_limit", "joint_kp", "joint_kd",
        "joint_mu", "joint_q0", "joint_qd0", "joint_target", "env_plane")]


class OrParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("pgs_iters", C.c_int), ("pgs_tol", C.c_double),
                ("pgs_max_iters", C.c_int), ("baumgarte", C.c_double), ("slop", C.c_double),
                ("margin", C.c_double), ("rest_thresh", C.c_double), ("sleep_lin", C.c_double),
                ("sleep_ang", C.c_double), ("sleep_steps", C.c_int), ("sleep_enabled", C.c_int),
                ("warm_mode", C.c_int), ("plane_mu", C.c_double), ("lambda_floor", C.c_double),
                ("match_dist", C.c_double), ("max_contacts", C.c_int), ("use_colouring", C.c_int),
                ("force_limit", C.c_double), ("motor_mode", C.c_int), ("motor_kp", C.c_double),
                ("motor_max_impulse", C.c_double)]


class OrState(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "obj_pos", "obj_quat", "obj_vel", "obj_omega", "obj_awake", "obj_ctr", "joint_q", "joint_qd",
        "joint_target", "art_base_pos", "art_base_quat", "joint_lim_lambda", "joint_lim_side", "cache_count",
        "cache_key", "cache_p", "cache_lambda", "joint_motor_lambda")]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_params(p, use_colouring: int = 1) -> OrParams:
    o = OrParams()
    o.dt = p.dt
    o.gravity = (C.c_double * 3)(*p.gravity)
    for k in ("pgs_iters", "pgs_max_iters", "sleep_steps", "sleep_enabled", "warm_mode", "max_contacts"):
        setattr(o, k, int(getattr(p, k)))
    for k in ("pgs_tol", "baumgarte", "slop", "margin", "rest_thresh", "sleep_lin", "sleep_ang", "plane_mu",
              "lambda_floor", "match_dist"):
        setattr(o, k, float(getattr(p, k)))
    o.use_colouring = int(use_colouring)
    o.force_limit = float(getattr(p, "force_limit", 0.0))
    o.motor_mode = int(getattr(p, "motor_mode", 0))
    o.motor_kp = float(getattr(p, "motor_kp", 0.3))
    o.motor_max_impulse = float(getattr(p, "motor_max_impulse", 10.0))
    return o


def empty_state(n_envs, n_obj, n_joint, n_art, max_contacts) -> dict:
    C_ = max_contacts
    return dict(
        obj_pos=np.zeros((n_obj, 3)), obj_quat=np.zeros((n_obj, 4)), obj_vel=np.zeros((n_obj, 3)),
        obj_omega=np.zeros((n_obj, 3)), obj_awake=np.zeros(n_obj, np.int32), obj_ctr=np.zeros(n_obj, np.int32),
        joint_q=np.zeros(n_joint), joint_qd=np.zeros(n_joint), joint_target=np.zeros(n_joint),
        art_base_pos=np.zeros((n_art, 3)), art_base_quat=np.zeros((n_art, 4)),
        joint_lim_lambda=np.zeros(n_joint), joint_lim_side=np.zeros(n_joint, np.int32),
        joint_motor_lambda=np.zeros(n_joint),
        cache_count=np.zeros(n_envs, np.int32), cache_key=np.zeros((n_envs, C_, 3), np.int32),
        cache_p=np.zeros((n_envs, C_, 3)), cache_lambda=np.zeros((n_envs, C_, 4)))


class Oracle:
    """One FP64 oracle world built from a `scenegen.Batch` and `scenegen.SimParams`."""

    def __init__(self, batch, params, use_colouring: int = 1, counting: bool = False, fp32: bool = False):
        self.lib = _lib(counting, fp32)
        self.batch = batch
        self.params = params
        self._keep = {k: np.ascontiguousarray(v) for k, v in batch.arrays.items()}
        d = OrDesc()
        d.n_envs = batch.n_envs
        for name, _ in OrDesc._fields_[1:]:
            setattr(d, name, _ptr(self._keep[name]))
        self._p = make_params(params, use_colouring)
        self.h = self.lib.oracle_create(C.byref(d), C.byref(self._p))
        self.E = batch.n_envs

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_destroy(h)
            self.h = None

    def set_params(self, params, use_colouring: int = 1):
        self.params = params
        self._p = make_params(params, use_colouring)
        self.lib.oracle_set_params(self.h, C.byref(self._p))

    def step(self, n: int = 1, threads: int = 1) -> int:
        return self.lib.oracle_step(self.h, int(n), int(threads))

    def step_logged(self, cap: int = 1 << 16):
        f = np.zeros((cap, MLP_IN))
        l = np.zeros((cap, 3))
        n = C.c_int(0)
        st = self.lib.oracle_step_logged(self.h, _ptr(f), _ptr(l), cap, C.byref(n))
        m = min(cap, n.value)
        return st, f[:m], l[:m]

    def get_state(self) -> dict:
        b = self.batch
        s = empty_state(self.E, b.n_objects, b.n_joints, b.n_arts, self.params.max_contacts)
        st = OrState(**{k: _ptr(v) for k, v in s.items()})
        self.lib.oracle_get_state(self.h, C.byref(st))
        return s

    def set_state(self, s: dict):
        s = {k: np.ascontiguousarray(v, dtype=np.int32 if v.dtype.kind in "iu" else np.float64) for k, v in s.items()}
        st = OrState(**{k: _ptr(s[k]) for k, _ in OrState._fields_ if k in s})
        self.lib.oracle_set_state(self.h, C.byref(st))

    def stats(self) -> dict:
        E = self.E
        out = dict(status=np.zeros(E, np.int32), iters=np.zeros(E, np.int32), resid=np.zeros(E),
                   n_contacts=np.zeros(E, np.int32), n_rows=np.zeros(E, np.int32),
                   n_limit_rows=np.zeros(E, np.int32), n_colours=np.zeros(E, np.int32))
        self.lib.oracle_get_stats(self.h, *[_ptr(out[k]) for k in
                                            ("status", "iters", "resid", "n_contacts", "n_rows", "n_limit_rows",
                                             "n_colours")])
        return out

    def robot_force(self):
        """(this step's, accumulated) contact force on the robot per env, N."""
        step, acc = np.zeros(self.E), np.zeros(self.E)
        self.lib.oracle_get_robot_force(self.h, _ptr(step), _ptr(acc))
        return step, acc

    def reset_robot_force(self, env_ids=None):
        if env_ids is None:
            self.lib.oracle_reset_robot_force(self.h, None, 0)
        else:
            ids = np.ascontiguousarray(env_ids, np.int32)
            self.lib.oracle_reset_robot_force(self.h, _ptr(ids), len(ids))

    def contacts(self, e: int) -> dict:
        cap = self.params.max_contacts
        key = np.zeros((cap, 3), np.int32)
        p, n, lam = np.zeros((cap, 3)), np.zeros((cap, 3)), np.zeros((cap, 3))
        sep = np.zeros(cap)
        m = self.lib.oracle_get_contacts(self.h, int(e), cap, _ptr(key), _ptr(p), _ptr(n), _ptr(sep), _ptr(lam))
        m = min(m, cap)
        return dict(key=key[:m], p=p[:m], n=n[:m], sep=sep[:m], lam=lam[:m])

    def pairs(self, e: int) -> np.ndarray:
        out = np.zeros(8192, np.int32)
        m = self.lib.oracle_get_pairs(self.h, int(e), 8192, _ptr(out))
        return out[:min(m, 8192)]

    def colouring(self, e: int) -> dict:
        """Env e's units at the last step, in unit order: colour (64: the serial overflow
        colour, -1: colouring off) and the two colouring nodes (-1: static)."""
        cap = 4096
        col, na, nb = (np.zeros(cap, np.int32) for _ in range(3))
        n = self.lib.oracle_get_colouring(self.h, int(e), cap, _ptr(col), _ptr(na), _ptr(nb))
        n = min(n, cap)
        return dict(colour=col[:n], node_a=na[:n], node_b=nb[:n])

    def articulation(self, e: int, a: int) -> dict:
        com, rot = np.zeros((9, 3)), np.zeros((9, 3, 3))
        qdd = np.zeros(9)
        M, Minv = np.zeros(81), np.zeros(81)
        n = self.lib.oracle_articulation(self.h, int(e), int(a), _ptr(com), _ptr(rot), _ptr(qdd), _ptr(M), _ptr(Minv))
        return dict(n=n, com=com[:n], rot=rot[:n], qdd=qdd[:n], M=M[:n * n].reshape(n, n),
                    Minv=Minv[:n * n].reshape(n, n))

    def dynamics_check(self, e: int, a: int, tau, qdd_in):
        n = len(tau)
        tau = np.ascontiguousarray(tau, np.float64)
        qdd_in = np.ascontiguousarray(qdd_in, np.float64)
        qdd, tr, M = np.zeros(n), np.zeros(n), np.zeros(n * n)
        self.lib.oracle_dynamics_check(self.h, int(e), int(a), _ptr(tau), _ptr(qdd), _ptr(qdd_in), _ptr(tr), _ptr(M))
        return qdd, tr, M.reshape(n, n)

    def set_mlp(self, params):
        if params is None:
            self.lib.oracle_set_mlp(self.h, None)
        else:
            self._mlp = np.ascontiguousarray(params, np.float64)
            self.lib.oracle_set_mlp(self.h, _ptr(self._mlp))

    def op_counts(self) -> dict:
        out = (C.c_ulonglong * len(STAGES))()
        self.lib.oracle_get_op_counts(out)
        return dict(zip(STAGES, [int(x) for x in out]))

    def reset_op_counts(self):
        self.lib.oracle_reset_op_counts()


def narrowphase(shape_a, xa, qa, ha, shape_b, xb=None, qb=None, hb=None, margin=0.02, cap=16):
    lib = _lib()
    f = lambda a, n: np.ascontiguousarray(a if a is not None else np.zeros(n), np.float64)
    xa, qa, ha = f(xa, 3), f(qa, 4), f(ha, 3)
    xb, qb, hb = f(xb, 3), f(qb if qb is not None else [1, 0, 0, 0], 4), f(hb, 3)
    p, n = np.zeros((cap, 3)), np.zeros((cap, 3))
    sep = np.zeros(cap)
    feat = np.zeros(cap, np.int32)
    m = lib.oracle_narrowphase(int(shape_a), _ptr(xa), _ptr(qa), _ptr(ha), int(shape_b), _ptr(xb), _ptr(qb),
                               _ptr(hb), float(margin), _ptr(p), _ptr(n), _ptr(sep), _ptr(feat), cap)
    m = min(m, cap)
    return dict(p=p[:m], n=n[:m], sep=sep[:m], feat=feat[:m])


def mlp_nparam() -> int:
    return _lib().oracle_mlp_nparam()


def mlp_forward(params, X) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float64)
    P = np.ascontiguousarray(params, np.float64)
    Y = np.zeros((X.shape[0], MLP_OUT))
    _lib().oracle_mlp_forward(_ptr(P), X.shape[0], _ptr(X), _ptr(Y))
    return Y


def mlp_loss_grad(params, X, T):
    X = np.ascontiguousarray(X, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    P = np.ascontiguousarray(params, np.float64)
    G = np.zeros_like(P)
    loss = _lib().oracle_mlp_loss_grad(_ptr(P), X.shape[0], _ptr(X), _ptr(T), _ptr(G))
    return loss, G
