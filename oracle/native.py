"""ctypes front end of the FP64 C oracle (``ssa_oracle.c``).  Test infrastructure only.

``run`` simulates trajectories exactly as Section 2 and the Gumbel-max equation of Section 3.2
state them, reads them out on a sample grid (HOLD, the LINEAR interpolation of Section 4.1, or the
exact bin average BIN of Section 4.4 over the bins (t_{s-1}, t_s], t_{-1} = 0),
and, when an upstream gradient dL/dobs is given, returns the straight-through gradient of
Eqs. 5 and 7 with the waiting-time term of Section 3.1, per trajectory, in float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HOLD = 0
LINEAR = 1
BIN = 2
STATUS = {"OK": 0, "ABSORBED": 1, "STEP_CAP": 2, "NEG_COUNT": 3, "OVERFLOW": 4, "BAD_RATE": 5}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ssa_oracle.c into liboracle.so with gcc (portable flags; no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Net(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("n_reactions", ctypes.c_int32),
        ("reactants", ctypes.c_void_p),
        ("stoich_ptr", ctypes.c_void_p),
        ("stoich_species", ctypes.c_void_p),
        ("stoich_delta", ctypes.c_void_p),
        ("n_params", ctypes.c_int32),
        ("log_rates", ctypes.c_void_p),
        ("rate_index", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run.argtypes = [p, i64, i64, p, i32, f64, p, i32, p, i32, u64, i32, i64, p, f64,
                                p, p, p, p, p, p, p, i64, p, i32]
        lib.orc_run_sel.restype = ctypes.c_int
        lib.orc_run_sel.argtypes = [i32] + lib.orc_run.argtypes
        lib.orc_uniforms.restype = None
        lib.orc_uniforms.argtypes = [u64, u64, u64, i64, p]
        lib.orc_philox_blocks.restype = None
        lib.orc_philox_blocks.argtypes = [u64, p, i64, p]
        lib.orc_grn_run.restype = ctypes.c_int
        lib.orc_grn_run.argtypes = [p, i64, i64, i64, p, f64, p, i32, u64, i64, p, f64, p, p, p, p, p, p, p,
                                    p, p, i64, i32]
        lib.orc_grn_run_sel.restype = ctypes.c_int
        lib.orc_grn_run_sel.argtypes = [i32] + lib.orc_grn_run.argtypes
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox_blocks(seed: int, counters: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of each counter row [n, 4] (uint32) under key (seed_lo, seed_hi)."""
    lib = _load()
    ctr = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib.orc_philox_blocks(ctypes.c_uint64(seed), _ptr(ctr), ctr.shape[0], _ptr(out))
    return out


def uniforms(seed: int, traj: int, step: int, n_words: int) -> np.ndarray:
    """The first n_words uniforms of step `step` of trajectory `traj` (u_0 drives tau)."""
    lib = _load()
    out = np.zeros(n_words, dtype=np.float64)
    lib.orc_uniforms(ctypes.c_uint64(seed), ctypes.c_uint64(traj), ctypes.c_uint64(step), n_words, _ptr(out))
    return out


@dataclass
class OracleResult:
    obs: np.ndarray            # [n_traj, S, n_obs] float64
    draws: np.ndarray          # [n_traj] int64, reaction draws including a crossing draw
    status: np.ndarray         # [n_traj] int32
    dtheta: np.ndarray | None  # [n_traj, P] float64
    events: np.ndarray | None  # [n_traj, ev_cap] int32, -1 padded
    margins: np.ndarray | None # [n_traj, ev_cap] float64
    times: np.ndarray | None   # [n_traj, ev_cap] t_{k+1} of each draw
    final_x: np.ndarray        # [n_traj, N] int32, last visited state


def run(net, log_rates, x0, n_traj: int, t_end: float, sample_times, obs_species, seed: int,
        readout: int = HOLD, max_steps: int = 1 << 30, traj_offset: int = 0, dl_dobs=None,
        temperature: float = 1.0, ev_cap: int = 0, n_threads: int | None = None,
        selector: str = "gumbel") -> OracleResult:
    """Run the oracle. `net` is a ssa_workloads.NetworkSpec; x0 is [N] or [n_traj, N]. selector "gumbel"
    is the Gumbel-max choice (Section 3.2); "direct" the standard direct method (Section 2: u_1 a0 against
    the cumulative propensities), forward only; its margins are distances of u_1 a0 to the nearest
    cumulative boundary, relative to a0. "soft" is the relaxed forward of Eq. 4 at temperature
    `temperature` (real-valued states, obs as float64; final_x truncated to int32); with dl_dobs its
    gradient is the exact gradient of that relaxed model."""
    lib = _load()
    reactants = np.ascontiguousarray(net.reactants, dtype=np.int32)
    sptr = np.ascontiguousarray(net.stoich_ptr, dtype=np.int32)
    ssp = np.ascontiguousarray(net.stoich_species, dtype=np.int32)
    sdl = np.ascontiguousarray(net.stoich_delta, dtype=np.int32)
    ridx = np.ascontiguousarray(net.rate_index, dtype=np.int32)
    th = np.ascontiguousarray(log_rates, dtype=np.float64)
    assert th.shape == (net.n_params,)
    cnet = _Net(net.n_species, net.n_reactions, _ptr(reactants), _ptr(sptr), _ptr(ssp), _ptr(sdl),
                net.n_params, _ptr(th), _ptr(ridx))
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    per_traj = 1 if x0.ndim == 2 else 0
    if per_traj:
        assert x0.shape == (n_traj, net.n_species)
    ts = np.ascontiguousarray(sample_times, dtype=np.float64)
    S = int(ts.shape[0])
    obs_sp = np.ascontiguousarray(obs_species, dtype=np.int32)
    n_obs = int(obs_sp.shape[0])
    obs = np.zeros((n_traj, S, n_obs), dtype=np.float64)
    draws = np.zeros(n_traj, dtype=np.int64)
    status = np.zeros(n_traj, dtype=np.int32)
    final_x = np.zeros((n_traj, net.n_species), dtype=np.int32)
    dth = None
    g = None
    if dl_dobs is not None:
        g = np.ascontiguousarray(dl_dobs, dtype=np.float64)
        assert g.shape == (n_traj, S, n_obs)
        dth = np.zeros((n_traj, net.n_params), dtype=np.float64)
    ev = mg = tm = None
    if ev_cap > 0:
        ev = np.zeros((n_traj, ev_cap), dtype=np.int32)
        mg = np.zeros((n_traj, ev_cap), dtype=np.float64)
        tm = np.zeros((n_traj, ev_cap), dtype=np.float64)
    if n_threads is None:
        n_threads = min(os.cpu_count() or 1, max(1, n_traj // 8))
    sel = {"gumbel": 0, "direct": 1, "soft": 2}[selector]
    rc = lib.orc_run_sel(sel, ctypes.byref(cnet), n_traj, traj_offset, _ptr(x0), per_traj, float(t_end),
                     _ptr(ts), S, _ptr(obs_sp), n_obs, ctypes.c_uint64(seed), readout, max_steps,
                     _ptr(g), float(temperature), _ptr(obs), _ptr(draws), _ptr(status), _ptr(dth),
                     _ptr(ev), _ptr(mg), _ptr(tm), ev_cap, _ptr(final_x), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected its inputs (orc_run returned %d)" % rc)
    return OracleResult(obs, draws, status, dth, ev, mg, tm, final_x)


class _GRN(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hid", ctypes.c_int32), ("n_out", ctypes.c_int32),
                ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("W2", ctypes.c_void_p), ("b2", ctypes.c_void_p),
                ("log_d", ctypes.c_void_p), ("k_max", ctypes.c_double)]


@dataclass
class GRNResult:
    obs: np.ndarray            # [n_traj, S, n_out] float64 (HOLD counts of the outputs)
    draws: np.ndarray
    status: np.ndarray
    dE1: np.ndarray | None     # [n_traj, n_hid] dL/dE1 per trajectory
    dW2: np.ndarray | None     # [n_traj, n_out, n_hid]
    db2: np.ndarray | None     # [n_traj, n_out]
    dlogd: np.ndarray | None   # [n_traj, n_hid + n_out]
    events: np.ndarray | None
    margins: np.ndarray | None

    def grads(self, x_img, traj_per_img):
        """Parameter gradients summed over trajectories: dW1 = sum_traj dE1 x^T, db1 = sum dE1, ..."""
        n_img = x_img.shape[0]
        g_img = self.dE1.reshape(n_img, traj_per_img, -1).sum(1)
        return {"W1": g_img.T @ x_img.astype(np.float64), "b1": g_img.sum(0), "W2": self.dW2.sum(0),
                "b2": self.db2.sum(0), "log_d": self.dlogd.sum(0)}


def grn_run(params, x_img, traj_per_img: int, t_end: float, sample_times, seed: int, max_steps: int = 1 << 30,
            traj_offset: int = 0, dl_dobs=None, temperature: float = 1.0, ev_cap: int = 0,
            n_threads: int | None = None, soft: bool = False) -> GRNResult:
    """GRN oracle (FP64): HOLD readout of the output genes at the sample times. soft: the relaxed forward
    of Eq. 4 at `temperature` (real-valued counts) and, with dl_dobs, the exact gradient of that model."""
    lib = _load()
    W1 = np.ascontiguousarray(params.W1, dtype=np.float64)
    b1 = np.ascontiguousarray(params.b1, dtype=np.float64)
    W2 = np.ascontiguousarray(params.W2, dtype=np.float64)
    b2 = np.ascontiguousarray(params.b2, dtype=np.float64)
    ld = np.ascontiguousarray(params.log_d, dtype=np.float64)
    n_hid, n_in = W1.shape
    n_out = W2.shape[0]
    g = _GRN(n_in, n_hid, n_out, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(ld), float(params.k_max))
    x = np.ascontiguousarray(x_img, dtype=np.int32)
    n_img = x.shape[0]
    n_traj = n_img * traj_per_img
    ts = np.ascontiguousarray(sample_times, dtype=np.float64)
    S = ts.shape[0]
    obs = np.zeros((n_traj, S, n_out))
    draws = np.zeros(n_traj, np.int64)
    status = np.zeros(n_traj, np.int32)
    gl = dE1 = dW2 = db2 = dld = None
    if dl_dobs is not None:
        gl = np.ascontiguousarray(dl_dobs, dtype=np.float64)
        assert gl.shape == (n_traj, S, n_out)
        dE1 = np.zeros((n_traj, n_hid))
        dW2 = np.zeros((n_traj, n_out, n_hid))
        db2 = np.zeros((n_traj, n_out))
        dld = np.zeros((n_traj, n_hid + n_out))
    ev = mg = None
    if ev_cap > 0:
        ev = np.zeros((n_traj, ev_cap), np.int32)
        mg = np.zeros((n_traj, ev_cap))
    if n_threads is None:
        n_threads = min(os.cpu_count() or 1, max(1, n_traj // 4))
    rc = lib.orc_grn_run_sel(1 if soft else 0, ctypes.byref(g), n_img, traj_per_img, traj_offset, _ptr(x), float(t_end), _ptr(ts), S,
                         ctypes.c_uint64(seed), max_steps, _ptr(gl), float(temperature), _ptr(obs), _ptr(draws),
                         _ptr(status), _ptr(dE1), _ptr(dW2), _ptr(db2), _ptr(dld), _ptr(ev), _ptr(mg), ev_cap,
                         int(n_threads))
    if rc != 0:
        raise ValueError("GRN oracle rejected its inputs")
    return GRNResult(obs, draws, status, dE1, dW2, db2, dld, ev, mg)
