"""ctypes declarations of the C ABI in include/sim.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_lib = None

SIM_OK = 0
ERRORS = {1: "SIM_ERR_INVALID_ARG", 2: "SIM_ERR_CUDA", 3: "SIM_ERR_OOM", 4: "SIM_ERR_NUMERIC",
          5: "SIM_ERR_OVERFLOW", 6: "SIM_ERR_TIMEOUT", 7: "SIM_ERR_STATE"}
ENV_OVERFLOW, ENV_NUMERIC, ENV_ITER_CAP = 1, 2, 4
MAX_CONTACTS = 256
PAIR_CAP = 1024


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


DESC_FIELDS = ("obj_off", "obj_shape", "obj_half", "obj_mass", "obj_mu", "obj_rest", "obj_pos", "obj_quat",
               "obj_vel", "obj_omega", "stat_off", "stat_pos", "stat_quat", "stat_half", "stat_mu", "art_off",
               "joint_off", "art_base_pos", "art_base_quat", "art_has_base_coll", "art_base_coll_off",
               "art_base_coll_half", "art_kinematic", "joint_parent", "joint_type", "joint_axis",
               "joint_origin_pos", "joint_origin_quat", "joint_com", "joint_half", "joint_mass", "joint_lo",
               "joint_hi", "joint_has_limit", "joint_kp", "joint_kd", "joint_mu", "joint_q0", "joint_qd0",
               "joint_target", "env_plane")


class SimBatchDesc(C.Structure):
    _fields_ = [("n_envs", C.c_int)] + [(n, C.c_void_p) for n in DESC_FIELDS]


class SimParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("pgs_iters", C.c_int), ("pgs_tol", C.c_double),
                ("pgs_max_iters", C.c_int), ("baumgarte", C.c_double), ("slop", C.c_double),
                ("margin", C.c_double), ("rest_thresh", C.c_double), ("sleep_lin", C.c_double),
                ("sleep_ang", C.c_double), ("sleep_steps", C.c_int), ("sleep_enabled", C.c_int),
                ("warm_mode", C.c_int), ("plane_mu", C.c_double), ("lambda_floor", C.c_double),
                ("match_dist", C.c_double), ("max_contacts", C.c_int), ("fp64_cond", C.c_double),
                ("use_graph", C.c_int), ("log_features", C.c_int), ("force_limit", C.c_double),
                ("motor_mode", C.c_int), ("motor_kp", C.c_double), ("motor_max_impulse", C.c_double)]


STATE_FIELDS = (("obj_pos", "f", 3, "NO"), ("obj_pos_comp", "f", 3, "NO"), ("obj_quat", "f", 4, "NO"),
                ("obj_vel", "f", 3, "NO"), ("obj_omega", "f", 3, "NO"), ("obj_awake", "i", 1, "NO"),
                ("obj_ctr", "i", 1, "NO"), ("joint_q", "f", 1, "NJ"), ("joint_q_comp", "f", 1, "NJ"),
                ("joint_qd", "f", 1, "NJ"), ("joint_target", "f", 1, "NJ"), ("art_base_pos", "f", 3, "NA"),
                ("art_base_quat", "f", 4, "NA"), ("joint_lim_lambda", "f", 1, "NJ"), ("joint_lim_side", "i", 1, "NJ"),
                ("cache_count", "i", 1, "E"), ("cache_key", "i", 3, "EC"), ("cache_p", "f", 3, "EC"),
                ("cache_lambda", "f", 4, "EC"), ("joint_motor_lambda", "f", 1, "NJ"))


class SimStateView(C.Structure):
    _fields_ = [(f[0], C.c_void_p) for f in STATE_FIELDS]


SHAPE_FIELDS = ("collide_warps", "collide_persistent", "rows_warps", "rows_persistent", "pgs_warps",
                "pgs_persistent", "pgs_lpt", "pgs_lanes", "pgs_min_blocks", "pgs_heavy_sms", "pgs_stage_contacts",
                "pgs_stage_pool", "aba_lanes", "partitions", "aba_overlap", "fused")
TUNE_MAX_TRIALS = 96


class SimLaunchShape(C.Structure):
    _fields_ = [(n, C.c_int32) for n in SHAPE_FIELDS]


class SimTuneReport(C.Structure):
    _fields_ = [("n_trials", C.c_int32), ("steps_taken", C.c_int32),
                ("trial", SimLaunchShape * TUNE_MAX_TRIALS), ("ms", (C.c_float * 5) * TUNE_MAX_TRIALS),
                ("chosen_ms", C.c_float * 5)]


EXPORTS = ("sim_create", "sim_destroy", "sim_set_params", "sim_set_joint_targets", "sim_set_base_pose", "sim_step",
           "sim_sync", "sim_get_state", "sim_set_state", "sim_get_env_stats", "sim_get_contacts", "sim_get_pairs",
           "sim_get_articulation", "sim_set_mlp", "sim_log_contacts", "sim_log_predictions", "sim_debug_hold_async",
           "sim_set_profiling",
           "sim_kernel_times",
           "sim_launch_count", "sim_get_robot_force", "sim_reset_robot_force", "sim_reset_envs",
           "sim_set_reset_state", "sim_get_launch_shape", "sim_set_launch_shape", "sim_autotune",
           "sim_log_contacts_noalloc", "sim_last_error", "sim_set_warm_start", "sim_get_stats", "sim_fp32_fma_peak",
           "mlp_train_create", "mlp_train_destroy", "mlp_train_step", "mlp_loss_grad", "mlp_forward", "mlp_get_params",
           "mlp_select_rows", "mlp_feature_stats")


class SimStats(C.Structure):
    _fields_ = [("n_envs", C.c_int32), ("max_iters", C.c_int32), ("sum_iters", C.c_int64), ("row_sweeps", C.c_int64),
                ("n_contacts", C.c_int64), ("n_rows", C.c_int64), ("n_limit_rows", C.c_int64),
                ("n_pool_slots", C.c_int64), ("n_awake", C.c_int64), ("n_iter_cap", C.c_int32), ("n_fp64", C.c_int32),
                ("max_colours", C.c_int32), ("status_or", C.c_uint32), ("max_resid", C.c_float),
                ("n_net_rows", C.c_int64)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsim.so (building it first if it is missing or stale).  Raises if it cannot be loaded:
    there is no other implementation of the engine."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA engine library missing: {path} (run paper_2106_14405_gb300.build.build())")
    lib = C.CDLL(path)
    vp, i, f = C.c_void_p, C.c_int, C.c_void_p
    lib.sim_create.argtypes = [vp, vp, vp, C.POINTER(vp)]
    lib.sim_destroy.argtypes = [vp]
    lib.sim_destroy.restype = None
    lib.sim_set_params.argtypes = [vp, vp]
    lib.sim_set_joint_targets.argtypes = [vp, f, i]
    lib.sim_set_base_pose.argtypes = [vp, f, i]
    lib.sim_step.argtypes = [vp, i]
    lib.sim_sync.argtypes = [vp, vp, vp]
    lib.sim_get_state.argtypes = [vp, vp, i]
    lib.sim_set_state.argtypes = [vp, vp, i]
    lib.sim_get_env_stats.argtypes = [vp] + [vp] * 8 + [i]
    lib.sim_get_contacts.argtypes = [vp] + [vp] * 6 + [i]
    lib.sim_get_pairs.argtypes = [vp, i, vp, vp, i]
    lib.sim_get_articulation.argtypes = [vp] + [vp] * 4 + [i]
    lib.sim_set_mlp.argtypes = [vp, vp, i]
    lib.sim_log_contacts.argtypes = [vp, vp, vp, i, vp]
    lib.sim_log_predictions.argtypes = [vp, vp, i, vp]
    lib.sim_debug_hold_async.argtypes = [vp, i]
    lib.sim_log_contacts_noalloc.argtypes = [vp, vp, vp, i, vp]
    lib.sim_set_profiling.argtypes = [vp, i]
    lib.sim_kernel_times.argtypes = [vp, vp, vp]
    lib.sim_launch_count.argtypes = [vp, vp]
    lib.sim_get_robot_force.argtypes = [vp, vp, vp, i]
    lib.sim_reset_robot_force.argtypes = [vp, vp, i, i]
    lib.sim_reset_envs.argtypes = [vp, vp, i, i]
    lib.sim_set_reset_state.argtypes = [vp, vp, i]
    lib.sim_get_launch_shape.argtypes = [vp, vp]
    lib.sim_set_launch_shape.argtypes = [vp, vp]
    lib.sim_autotune.argtypes = [vp, i, i, vp, vp]
    lib.mlp_train_create.argtypes = [vp, i, i, vp, vp, vp, C.POINTER(vp)]
    lib.mlp_train_destroy.argtypes = [vp]
    lib.mlp_train_destroy.restype = None
    lib.mlp_train_step.argtypes = [vp, vp, vp, i, C.c_float, vp]
    lib.mlp_loss_grad.argtypes = [vp, vp, vp, i, vp, vp]
    lib.mlp_forward.argtypes = [vp, vp, i, vp]
    lib.mlp_get_params.argtypes = [vp, vp, i]
    lib.sim_set_warm_start.argtypes = [vp, i, vp, i]
    lib.sim_get_stats.argtypes = [vp, vp]
    lib.sim_fp32_fma_peak.argtypes = [vp, i, i, vp, vp]
    lib.mlp_select_rows.argtypes = [vp, vp, i, i, C.c_float, C.c_float, vp, vp, vp, vp]
    lib.mlp_feature_stats.argtypes = [vp, i, vp, vp, i, vp]
    lib.sim_last_error.restype = C.c_char_p
    lib.sim_last_error.argtypes = [vp]
    _lib = lib
    return lib


def check(rc: int):
    if rc != SIM_OK:
        raise SimError(rc, _lib.sim_last_error(None).decode(errors="replace"))
