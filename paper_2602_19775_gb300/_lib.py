"""ctypes binding of libssa.so (the C ABI in include/ssa.h): argument marshalling only.

The library is loaded from this package directory. There is no fallback: if libssa.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssa.so")

SSA_OK = 0
SSA_READOUT_HOLD = 0
SSA_READOUT_LINEAR = 1
SSA_READOUT_BIN = 2
SSA_SELECT_GUMBEL = 0
SSA_SELECT_DIRECT = 1
SSA_SELECT_SOFT = 2
SSA_BIN_MAX_OBS = 4
TRAJ_CODES = ("OK", "ABSORBED", "STEP_CAP", "NEG_COUNT", "OVERFLOW", "BAD_RATE", "BAD_INPUT", "REPLAY_MISMATCH")
SSA_TRAJ_N_CODES = len(TRAJ_CODES)

# every symbol the header declares
EXPORTS = (
    "ssa_create_network", "ssa_destroy_network", "ssa_forward_workspace_bytes", "ssa_forward",
    "ssa_forward_replay", "ssa_backward", "ssa_backward_wide", "ssa_backward_multi", "ssa_run_status", "ssa_run_events", "ssa_run_brackets", "ssa_destroy_run",
    "ssa_ensemble_mean_workspace_bytes", "ssa_ensemble_mean", "ssa_ensemble_mean_static", "ssa_philox_uniforms",
    "ssa_bf16_gemm", "ssa_bf16_gemm_work_words", "ssa_pipe_rates", "ssa_last_error", "ssa_grn_create", "ssa_grn_destroy",
    "ssa_grn_workspace_bytes", "ssa_grn_forward", "ssa_grn_backward", "ssa_grn_activations",
    "ssa_batch_create", "ssa_batch_destroy", "ssa_batch_set_plan", "ssa_batch_set_soft", "ssa_batch_workspace_bytes", "ssa_batch_run",
    "ssa_batch_item_outputs", "ssa_batch_autotune", "ssa_batch_item_variant", "ssa_batch_item_events",
    "ssa_batch_item_brackets", "ssa_batch_item_ckpt_interval", "ssa_run_variant", "ssa_network_specialize", "ssa_exp_variates",
)


class SSAError(RuntimeError):
    pass


class FwdOpts(ctypes.Structure):
    _fields_ = [
        ("readout", ctypes.c_int32),
        ("record", ctypes.c_int32),
        ("ckpt_interval", ctypes.c_int32),
        ("threads_per_traj", ctypes.c_int32),
        ("max_steps", ctypes.c_int64),
        ("block_threads", ctypes.c_int32),
        ("no_specialize", ctypes.c_int32),
        ("selector", ctypes.c_int32),
        ("temperature", ctypes.c_float),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("net", ctypes.c_void_p),
        ("log_rates", ctypes.c_void_p),
        ("x0", ctypes.c_void_p),
        ("n_traj", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
        ("traj_offset", ctypes.c_int64),
        ("t_end", ctypes.c_double),
        ("sample_times", ctypes.c_void_p),
        ("n_samples", ctypes.c_int32),
        ("n_obs", ctypes.c_int32),
        ("obs_species", ctypes.c_void_p),
        ("max_steps", ctypes.c_int64),
        ("ckpt_interval", ctypes.c_int32),
        ("threads_per_traj", ctypes.c_int32),
        ("obs_out", ctypes.c_void_p),
        ("dl_dobs", ctypes.c_void_p),
        ("dl_traj_stride", ctypes.c_int64),
        ("dl_dlog_rates", ctypes.c_void_p),
    ]


_lib = None
_lock = threading.Lock()


def _declare(lib):
    p, i32, i64, u64, f32, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                      ctypes.c_float, ctypes.c_double, ctypes.c_size_t)
    opts = ctypes.POINTER(FwdOpts)
    sig = {
        "ssa_create_network": (i32, [i32, i32, p, p, p, p, i32, p, ctypes.POINTER(p)]),
        "ssa_destroy_network": (None, [p]),
        "ssa_forward_workspace_bytes": (sz, [p, i64, i32, opts]),
        "ssa_forward": (i32, [p, p, i64, i64, p, i32, f64, p, i32, p, i32, u64, opts, p, sz, p, p, p, p,
                              ctypes.POINTER(p)]),
        "ssa_forward_replay": (i32, [p, p, i64, i64, p, i32, f64, p, i32, p, i32, u64, opts, p, p, i64, p, sz,
                                     p, p, p, p, ctypes.POINTER(p)]),
        "ssa_backward": (i32, [p, p, i64, f32, p, p]),
        "ssa_backward_wide": (i32, [p, p, i64, f32, p, p]),
        "ssa_backward_multi": (i32, [p, p, i64, p, i32, p, p]),
        "ssa_run_status": (i32, [p, p, p, p]),
        "ssa_run_events": (i32, [p, p, i64, p]),
        "ssa_run_brackets": (i32, [p, p, p]),
        "ssa_destroy_run": (None, [p]),
        "ssa_ensemble_mean_workspace_bytes": (sz, [i64, i64]),
        "ssa_ensemble_mean": (i32, [p, i32, i64, i64, p, sz, p, p]),
        "ssa_ensemble_mean_static": (i32, [p, i32, i64, i64, p, p]),
        "ssa_philox_uniforms": (i32, [u64, p, p, i64, i32, p, p]),
        "ssa_pipe_rates": (i32, [p, p, p]),
        "ssa_bf16_gemm": (i32, [p, p, i32, i32, i32, i32, i32, p, p, i32, p, i64, p, p]),
        "ssa_bf16_gemm_work_words": (i64, [i32, i32, i32]),
        "ssa_last_error": (ctypes.c_char_p, []),
        "ssa_grn_create": (i32, [i32, i32, i32, f32, ctypes.POINTER(p)]),
        "ssa_grn_destroy": (None, [p]),
        "ssa_grn_workspace_bytes": (sz, [p, i64, i64, i32, opts]),
        "ssa_grn_forward": (i32, [p, p, p, p, p, p, i64, i64, i64, p, f64, p, i32, u64, opts, p, sz, p, p, p, p,
                                  ctypes.POINTER(p)]),
        "ssa_grn_backward": (i32, [p, p, i64, f32, p, p, p, p, p, p]),
        "ssa_grn_activations": (i32, [p, p, p, p]),
        "ssa_batch_create": (i32, [ctypes.POINTER(BatchItem), i32, i32, f32, ctypes.POINTER(p)]),
        "ssa_batch_destroy": (None, [p]),
        "ssa_batch_set_plan": (i32, [p, i32, i32, i32, f64]),
        "ssa_batch_set_soft": (i32, [p, i32]),
        "ssa_batch_workspace_bytes": (sz, [p]),
        "ssa_batch_run": (i32, [p, p, sz, i32, p]),
        "ssa_batch_item_outputs": (i32, [p, i32, p, p, p, p]),
        "ssa_batch_autotune": (i32, [p, i64, p, p]),
        "ssa_batch_item_variant": (i32, [p, i32]),
        "ssa_batch_item_ckpt_interval": (i32, [p, i32]),
        "ssa_batch_item_events": (i32, [p, i32, p, i64, p]),
        "ssa_batch_item_brackets": (i32, [p, i32, p, p]),
        "ssa_run_variant": (i32, [p]),
        "ssa_exp_variates": (i32, [p, i64, p, p]),
        "ssa_network_specialize": (i32, [p, ctypes.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    """The loaded library (raises SSAError if it is not built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise SSAError(f"{LIB_PATH} is not built; run paper_2602_19775_gb300.build.build()")
                l = ctypes.CDLL(LIB_PATH)
                _declare(l)
                _lib = l
    return _lib


def check(status: int):
    if status != SSA_OK:
        msg = lib().ssa_last_error().decode(errors="replace")
        raise SSAError(f"libssa error {status}: {msg}")
