"""PyTorch front end of libssa: device buffers, streams and a torch.autograd.Function.

PyTorch provides device memory and the current CUDA stream; every step of the simulation and of
the straight-through adjoint runs in the library's CUDA kernels (include/ssa.h). Nothing here
computes on the CPU, and there is no fallback: without a CUDA device or without libssa.so the
calls raise.

    net = Network(spec)                                   # any object with the array fields
    out = forward(net, theta, n_traj=65536, x0=x0, t_end=50.0, sample_times=ts,
                  obs_species=[0], seed=0, readout="linear", record=True)
    dtheta = backward(out, dl_dobs, temperature=0.5)      # dL/dlog k  [P]

    obs = simulate(net, theta, ..., temperature=0.5)      # autograd: obs.backward(...) -> theta.grad
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import FwdOpts, SSAError, check

READOUTS = {"hold": _lib.SSA_READOUT_HOLD, "linear": _lib.SSA_READOUT_LINEAR, "bin": _lib.SSA_READOUT_BIN}
SELECTORS = {"gumbel": _lib.SSA_SELECT_GUMBEL, "direct": _lib.SSA_SELECT_DIRECT, "soft": _lib.SSA_SELECT_SOFT}


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _require_cuda(t: torch.Tensor, name: str, dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise SSAError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise SSAError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise SSAError(f"{name} must be contiguous")


class Network:
    """A mass-action network held by the library (ssa_create_network)."""

    def __init__(self, spec):
        self.spec = spec
        self.n_species = int(spec.n_species)
        self.n_reactions = int(spec.n_reactions)
        self.n_params = int(spec.n_params)
        L = _lib.lib()
        arrs = [np.ascontiguousarray(getattr(spec, f), dtype=np.int32)
                for f in ("reactants", "stoich_ptr", "stoich_species", "stoich_delta", "rate_index")]
        self._keep = arrs
        h = ctypes.c_void_p()
        check(L.ssa_create_network(self.n_species, self.n_reactions,
                                   *(a.ctypes.data_as(ctypes.c_void_p) for a in arrs[:4]),
                                   self.n_params, arrs[4].ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h

    def specialize(self) -> tuple[bool, str]:
        """ssa_network_specialize: compile the network-specialised kernels now; (available, reason)."""
        ok = ctypes.c_int32(0)
        check(_lib.lib().ssa_network_specialize(self.handle, ctypes.byref(ok)))
        return bool(ok.value), ("" if ok.value else _lib.lib().ssa_last_error().decode(errors="replace"))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.lib().ssa_destroy_network(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Run:
    """A forward's run handle plus the buffers it references (workspace, outputs)."""

    def __init__(self, handle, workspace, net, n_traj, S, n_obs, readout):
        self.handle = handle
        self.workspace = workspace
        self.net = net
        self.n_traj = n_traj
        self.S = S
        self.n_obs = n_obs
        self.readout = readout

    def status_counts(self, stream=None):
        counts = (ctypes.c_int64 * _lib.SSA_TRAJ_N_CODES)()
        mism = ctypes.c_int64()
        check(_lib.lib().ssa_run_status(self.handle, counts, ctypes.byref(mism), _stream(stream)))
        return {name: int(counts[c]) for c, name in enumerate(_lib.TRAJ_CODES)}, int(mism.value)

    def events(self, stride: int, stream=None) -> torch.Tensor:
        out = torch.empty((self.n_traj, stride), dtype=torch.int32, device=self.workspace.device)
        check(_lib.lib().ssa_run_events(self.handle, _ptr(out), stride, _stream(stream)))
        return out

    def brackets(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n_traj, self.S), dtype=torch.int32, device=self.workspace.device)
        check(_lib.lib().ssa_run_brackets(self.handle, _ptr(out), _stream(stream)))
        return out

    @property
    def variant(self) -> int:
        """1 generic thread kernels, 2 network-specialised thread kernels, 32 warp kernels."""
        return int(_lib.lib().ssa_run_variant(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.lib().ssa_destroy_run(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class ForwardResult:
    obs: torch.Tensor       # [n_traj, S, n_obs] int32 (hold) or float32 (linear)
    draws: torch.Tensor     # [n_traj] int32
    status: torch.Tensor    # [n_traj] int32
    run: Run


def make_opts(readout="hold", record=False, ckpt_interval=64, max_steps=1 << 20, threads_per_traj=0,
              block_threads=0, specialize=True, selector="gumbel", temperature=None) -> FwdOpts:
    """ssa_fwd_opts; temperature is the soft forward's T (selector "soft" only)."""
    ro = READOUTS[readout] if isinstance(readout, str) else int(readout)
    sel = SELECTORS[selector]
    T = float(temperature) if sel == _lib.SSA_SELECT_SOFT and temperature is not None else 0.0
    return FwdOpts(ro, 1 if record else 0, int(ckpt_interval), int(threads_per_traj), int(max_steps),
                   int(block_threads), 0 if specialize else 1, sel, T)


def workspace_bytes(net: Network, n_traj: int, n_samples: int, opts: FwdOpts) -> int:
    n = _lib.lib().ssa_forward_workspace_bytes(net.handle, n_traj, n_samples, ctypes.byref(opts))
    if n == 0:
        raise SSAError("invalid arguments for ssa_forward_workspace_bytes")
    return int(n)


def _as_cuda(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.asarray(x), dtype=dtype, device=device).contiguous()


def forward(net: Network, log_rates, n_traj: int, x0, t_end: float, sample_times, obs_species, seed: int,
            readout="hold", record=False, ckpt_interval=64, max_steps=1 << 20, traj_offset=0,
            threads_per_traj=0, block_threads=0, specialize=True, selector="gumbel", temperature=None,
            replay_events=None,
            replay_n_events=None,
            workspace: torch.Tensor | None = None, obs_out: torch.Tensor | None = None,
            stream=None, device=None) -> ForwardResult:
    """ssa_forward (or ssa_forward_replay when replay_events is given) on the current stream.

    readout: "hold", "linear" or "bin" (the exact bin average over (t_{s-1}, t_s], t_{-1} = 0). selector:
    "gumbel" (the method), "direct" (the plain direct method, forward only) or "soft" (the relaxed forward of
    Eq. 4 at `temperature`; float observables for every readout). Observables are int32 for "hold" with an
    exact selector, float32 otherwise."""
    device = torch.device(device) if device is not None else (
        log_rates.device if isinstance(log_rates, torch.Tensor) and log_rates.is_cuda else torch.device("cuda"))
    theta = _as_cuda(log_rates, torch.float32, device)
    x0 = _as_cuda(x0, torch.int32, device)
    ts = _as_cuda(sample_times, torch.float64, device)
    obs_sp = _as_cuda(obs_species, torch.int32, device)
    S, n_obs = int(ts.numel()), int(obs_sp.numel())
    opts = make_opts(readout, record, ckpt_interval, max_steps, threads_per_traj, block_threads, specialize, selector,
                     temperature)
    need = workspace_bytes(net, n_traj, S, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    soft = opts.selector == _lib.SSA_SELECT_SOFT  # real-valued states: float observables
    odt = torch.int32 if opts.readout == _lib.SSA_READOUT_HOLD and not soft else torch.float32
    if obs_out is None:
        obs_out = torch.empty((n_traj, S, n_obs), dtype=odt, device=device)
    draws = torch.empty(n_traj, dtype=torch.int32, device=device)
    status = torch.empty(n_traj, dtype=torch.int32, device=device)
    per_traj = 1 if x0.dim() == 2 else 0
    h = ctypes.c_void_p()
    L = _lib.lib()
    common = (net.handle, _ptr(theta), int(n_traj), int(traj_offset), _ptr(x0), per_traj, float(t_end), _ptr(ts), S,
              _ptr(obs_sp), n_obs, ctypes.c_uint64(int(seed) & (2**64 - 1)), ctypes.byref(opts))
    if replay_events is None:
        check(L.ssa_forward(*common, _ptr(workspace), need, _ptr(obs_out), _ptr(draws), _ptr(status),
                            _stream(stream), ctypes.byref(h)))
    else:
        ev = _as_cuda(replay_events, torch.int32, device).to(torch.uint16) if not (
            isinstance(replay_events, torch.Tensor) and replay_events.dtype == torch.uint16) else replay_events
        nev = _as_cuda(replay_n_events, torch.int32, device)
        check(L.ssa_forward_replay(*common, _ptr(ev), _ptr(nev), int(ev.shape[1]), _ptr(workspace), need,
                                   _ptr(obs_out), _ptr(draws), _ptr(status), _stream(stream), ctypes.byref(h)))
    run = Run(h, workspace, net, n_traj, S, n_obs, opts.readout)
    run._keep = (theta, x0, ts, obs_sp)
    return ForwardResult(obs_out, draws, status, run)


def _upstream(run: Run, dl_dobs: torch.Tensor):
    g = dl_dobs.to(torch.float32).contiguous()
    if tuple(g.shape) == (run.n_traj, run.S, run.n_obs):
        stride = run.S * run.n_obs
    elif tuple(g.shape) == (run.S, run.n_obs):
        stride = 0  # the same upstream gradient for every trajectory
    else:
        raise SSAError(f"dl_dobs shape {tuple(g.shape)} is neither {(run.n_traj, run.S, run.n_obs)} "
                       f"nor {(run.S, run.n_obs)}")
    return g, stride


def backward(fwd: ForwardResult | Run, dl_dobs: torch.Tensor, temperature: float, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """ssa_backward: dL/dlog k [P] (float32) for a recorded forward."""
    run = fwd.run if isinstance(fwd, ForwardResult) else fwd
    g, stride = _upstream(run, dl_dobs)
    if out is None:
        out = torch.empty(run.net.n_params, dtype=torch.float32, device=g.device)
    check(_lib.lib().ssa_backward(run.handle, _ptr(g), stride, ctypes.c_float(float(temperature)), _ptr(out),
                                  _stream(stream)))
    return out


def backward_multi(fwd: ForwardResult | Run, dl_dobs: torch.Tensor, temperatures, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """ssa_backward_multi: dL/dlog k [n_T, P] (float32), row t at temperatures[t], from one walk of the
    recorded forward for up to three temperatures at a time (network-specialised kernels)."""
    run = fwd.run if isinstance(fwd, ForwardResult) else fwd
    g, stride = _upstream(run, dl_dobs)
    temps = (ctypes.c_float * len(temperatures))(*[float(t) for t in temperatures])
    if out is None:
        out = torch.empty((len(temperatures), run.net.n_params), dtype=torch.float32, device=g.device)
    check(_lib.lib().ssa_backward_multi(run.handle, _ptr(g), stride, temps, len(temperatures), _ptr(out),
                                        _stream(stream)))
    return out


def backward_wide(fwd: ForwardResult | Run, dl_dobs: torch.Tensor, temperature: float,
                  out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """ssa_backward_wide: dL/dlog k [P] (float64) with a per-trajectory exponent in the walk, for
    trajectories whose adjoint grows beyond the binary32 range (network-specialised kernels, HOLD or LINEAR)."""
    run = fwd.run if isinstance(fwd, ForwardResult) else fwd
    g, stride = _upstream(run, dl_dobs)
    if out is None:
        out = torch.empty(run.net.n_params, dtype=torch.float64, device=g.device)
    check(_lib.lib().ssa_backward_wide(run.handle, _ptr(g), stride, ctypes.c_float(float(temperature)), _ptr(out),
                                       _stream(stream)))
    return out



class Batch:
    """Many networks simulated and differentiated together (ssa_batch_*): one persistent forward and one
    persistent adjoint launch per run, optionally replayed from a captured CUDA graph.

    items: dicts with keys net, log_rates, n_traj, x0, t_end, sample_times, obs_species, seed and
    optionally traj_offset, max_steps, ckpt_interval, threads_per_traj, shared_dl (True: one upstream
    gradient [S, n_obs] for all trajectories). The batch owns fixed device tensors per item --
    log_rates[i], obs[i], dl_dobs[i], dtheta[i] -- whose addresses are baked into the plan: write new
    parameters or upstream gradients into them in place (copy_) between runs. soft: every item runs the soft
    forward of Eq. 4 at `temperature` and the exact gradient of that relaxed model (float observables).
    """

    def __init__(self, items, readout="hold", temperature=0.5, device=None, soft=False):
        device = torch.device(device) if device is not None else torch.device("cuda")
        ro = READOUTS[readout] if isinstance(readout, str) else int(readout)
        odt = torch.int32 if ro == _lib.SSA_READOUT_HOLD and not soft else torch.float32
        self.readout, self.device = ro, device
        self.log_rates, self.obs, self.dl_dobs, self.dtheta, self._keep = [], [], [], [], []
        self.nets = []
        arr = (_lib.BatchItem * len(items))()
        for q, it in enumerate(items):
            net = it["net"]
            theta = _as_cuda(it["log_rates"], torch.float32, device).clone()
            x0 = _as_cuda(it["x0"], torch.int32, device)
            ts = _as_cuda(it["sample_times"], torch.float64, device)
            sp = _as_cuda(it["obs_species"], torch.int32, device)
            n, S, o = int(it["n_traj"]), int(ts.numel()), int(sp.numel())
            obs = torch.zeros((n, S, o), dtype=odt, device=device)
            shared = bool(it.get("shared_dl", False))
            dl = torch.zeros((S, o) if shared else (n, S, o), dtype=torch.float32, device=device)
            dth = torch.zeros(net.n_params, dtype=torch.float32, device=device)
            self.nets.append(net)
            self.log_rates.append(theta)
            self.obs.append(obs)
            self.dl_dobs.append(dl)
            self.dtheta.append(dth)
            self._keep.append((x0, ts, sp))
            b = arr[q]
            b.net = net.handle
            b.log_rates = theta.data_ptr()
            b.x0 = x0.data_ptr()
            b.n_traj = n
            b.seed = int(it["seed"]) & (2**64 - 1)
            b.traj_offset = int(it.get("traj_offset", 0))
            b.t_end = float(it["t_end"])
            b.sample_times = ts.data_ptr() if S else None
            b.n_samples = S
            b.n_obs = o
            b.obs_species = sp.data_ptr() if o else None
            b.max_steps = int(it.get("max_steps", 1 << 14))
            b.ckpt_interval = int(it.get("ckpt_interval", 0))
            b.threads_per_traj = int(it.get("threads_per_traj", 0))
            b.obs_out = obs.data_ptr() if obs.numel() else None
            b.dl_dobs = dl.data_ptr() if dl.numel() else None
            b.dl_traj_stride = 0 if shared else S * o
            b.dl_dlog_rates = dth.data_ptr()
        self._items = arr
        h = ctypes.c_void_p()
        check(_lib.lib().ssa_batch_create(arr, len(items), ro, ctypes.c_float(float(temperature)), ctypes.byref(h)))
        self.handle = h
        if soft:  # the soft forward of Eq. 4 and the gradient of that relaxed model (ssa_batch_set_soft)
            check(_lib.lib().ssa_batch_set_soft(h, 1))
        self.workspace = None

    def __len__(self):
        return len(self.obs)

    def workspace_bytes(self) -> int:
        return int(_lib.lib().ssa_batch_workspace_bytes(self.handle))

    def autotune(self, pilot_traj: int = 256, stream=None) -> list:
        """ssa_batch_autotune: returns the pilot's mean draws per item."""
        out = (ctypes.c_double * len(self))()
        check(_lib.lib().ssa_batch_autotune(self.handle, int(pilot_traj), _stream(stream), out))
        self.workspace = None
        return list(out)

    def set_plan(self, item: int, threads_per_traj: int, ckpt_interval: int, est_draws: float = 0.0):
        check(_lib.lib().ssa_batch_set_plan(self.handle, int(item), int(threads_per_traj), int(ckpt_interval),
                                            float(est_draws)))
        self.workspace = None

    def variant(self, item: int) -> int:
        return int(_lib.lib().ssa_batch_item_variant(self.handle, int(item)))

    def ckpt_interval(self, item: int) -> int:
        """The item's planned checkpoint interval K (the autotuner's choice unless the item fixed one)."""
        return int(_lib.lib().ssa_batch_item_ckpt_interval(self.handle, int(item)))

    def run(self, use_graph: bool = False, stream=None) -> list:
        """ssa_batch_run: fills obs[i] and dtheta[i] for every item; returns dtheta."""
        need = self.workspace_bytes()
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
        check(_lib.lib().ssa_batch_run(self.handle, _ptr(self.workspace), need, 1 if use_graph else 0,
                                       _stream(stream)))
        return self.dtheta

    def outputs(self, item: int, stream=None):
        """(draws, status, adjoint mismatch count) of one item after run()."""
        n = self.obs[item].shape[0]
        draws = torch.empty(n, dtype=torch.int32, device=self.device)
        status = torch.empty(n, dtype=torch.int32, device=self.device)
        mism = ctypes.c_int64(0)
        check(_lib.lib().ssa_batch_item_outputs(self.handle, int(item), _ptr(draws), _ptr(status),
                                                ctypes.byref(mism), _stream(stream)))
        return draws, status, int(mism.value)

    def events(self, item: int, stride: int, stream=None) -> torch.Tensor:
        """Recorded events of one item as int32 [n_traj, stride], -1 after the last draw."""
        out = torch.empty((self.obs[item].shape[0], int(stride)), dtype=torch.int32, device=self.device)
        check(_lib.lib().ssa_batch_item_events(self.handle, int(item), _ptr(out), int(stride), _stream(stream)))
        return out

    def brackets(self, item: int, stream=None) -> torch.Tensor:
        """Sample brackets of one item as int32 [n_traj, n_samples]."""
        n, S = self.obs[item].shape[0], self.obs[item].shape[1]
        out = torch.empty((n, S), dtype=torch.int32, device=self.device)
        check(_lib.lib().ssa_batch_item_brackets(self.handle, int(item), _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            _lib.lib().ssa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ensemble_mean(obs: torch.Tensor, stream=None) -> torch.Tensor:
    """ssa_ensemble_mean over the first axis (deterministic order) -> float32 [obs.shape[1:]]."""
    obs = obs.contiguous()
    n = int(obs.shape[0])
    row = int(np.prod(obs.shape[1:])) if obs.dim() > 1 else 1
    L = _lib.lib()
    need = int(L.ssa_ensemble_mean_workspace_bytes(n, row))
    ws = torch.empty(max(need, 4), dtype=torch.uint8, device=obs.device)
    out = torch.empty(obs.shape[1:], dtype=torch.float32, device=obs.device)
    is_int = 1 if obs.dtype == torch.int32 else 0
    if not is_int and obs.dtype != torch.float32:
        raise SSAError("ensemble_mean takes int32 or float32 observables")
    check(L.ssa_ensemble_mean(_ptr(obs), is_int, n, row, _ptr(ws), need, _ptr(out), _stream(stream)))
    return out


def philox_uniforms(seed: int, traj, step, n_words: int, device="cuda") -> torch.Tensor:
    traj = _as_cuda(np.asarray(traj, dtype=np.int64), torch.int64, device)
    step = _as_cuda(np.asarray(step, dtype=np.int64), torch.int64, device)
    out = torch.empty((traj.numel(), n_words), dtype=torch.float32, device=device)
    check(_lib.lib().ssa_philox_uniforms(ctypes.c_uint64(int(seed) & (2**64 - 1)), _ptr(traj), _ptr(step),
                                         int(traj.numel()), int(n_words), _ptr(out), _stream()))
    return out


def exp_variates(words) -> torch.Tensor:
    """ssa_exp_variates: E = -ln u of the uniforms u of the given Philox words, as the kernels compute it."""
    w = _as_cuda(np.asarray(words, dtype=np.uint32).view(np.int32), torch.int32, "cuda")
    out = torch.empty(w.numel(), dtype=torch.float32, device="cuda")
    check(_lib.lib().ssa_exp_variates(_ptr(w), int(w.numel()), _ptr(out), _stream()))
    return out


def pipe_rates() -> dict:
    """ssa_pipe_rates: measured operations per SM per clock of the instruction classes of a step."""
    rates = (ctypes.c_double * 5)()
    mhz = ctypes.c_double()
    sms = ctypes.c_int32()
    check(_lib.lib().ssa_pipe_rates(rates, ctypes.byref(mhz), ctypes.byref(sms)))
    names = ("ffma", "dadd", "neglog", "imad", "lg2")
    out = {n: float(rates[i]) for i, n in enumerate(names)}
    out["sm_clock_mhz"] = float(mhz.value)
    out["sm_count"] = int(sms.value)
    return out


def bf16_gemm(A: torch.Tensor, B: torch.Tensor, bias: torch.Tensor | None = None, stream=None,
              split_k: bool = True) -> torch.Tensor:
    """ssa_bf16_gemm: A [M, K] bf16, B [N, K] bf16 (K-major) -> A B^T (+ bias) in float32 on tcgen05.
    split_k gives the call its binary64 work buffer (ssa_bf16_gemm_work_words), so that products with few
    output tiles split K across the SMs."""
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16:
        raise SSAError("bf16_gemm takes bfloat16 operands")
    M, K = A.shape
    N = B.shape[0]
    ld = (K + 7) // 8 * 8
    Ap = torch.zeros((M, ld), dtype=torch.bfloat16, device=A.device)
    Bp = torch.zeros((N, ld), dtype=torch.bfloat16, device=A.device)
    Ap[:, :K] = A
    Bp[:, :K] = B
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    b = None if bias is None else bias.to(torch.float32).contiguous()
    L = _lib.lib()
    words = int(L.ssa_bf16_gemm_work_words(M, N, K)) if split_k else 0
    work = torch.empty(max(words, 1), dtype=torch.float64, device=A.device) if words else None
    check(L.ssa_bf16_gemm(_ptr(Ap), _ptr(Bp), M, N, K, ld, ld, _ptr(b), _ptr(D), N, _ptr(work), words, _ptr(err),
                          _stream(stream)))
    if int(err.item()) != 0:
        raise SSAError("tensor-core GEMM timed out waiting for its copies")
    return D


def _bf16_bits(w) -> torch.Tensor:
    """bf16 bit patterns (as int16 storage) of a float tensor/array, rounded to nearest even."""
    t = torch.as_tensor(np.asarray(w, dtype=np.float32)) if not isinstance(w, torch.Tensor) else w.float()
    return t.to(torch.bfloat16).contiguous()


class GRN:
    """The gene-regulatory-network classifier held by the library (ssa_grn_create)."""

    def __init__(self, n_in: int, n_hid: int, n_out: int, k_max: float = 1.0):
        h = ctypes.c_void_p()
        check(_lib.lib().ssa_grn_create(n_in, n_hid, n_out, ctypes.c_float(k_max), ctypes.byref(h)))
        self.handle, self.n_in, self.n_hid, self.n_out, self.k_max = h, n_in, n_hid, n_out, k_max

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.lib().ssa_grn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class GRNForward:
    obs: torch.Tensor       # [n_traj, S, n_out] int32 (float32 for the soft forward)
    draws: torch.Tensor
    status: torch.Tensor
    run: Run


def grn_forward(grn: GRN, W1, b1, W2, b2, log_d, x_img, traj_per_img: int, t_end: float, sample_times, seed: int,
                record=True, ckpt_interval=64, max_steps=1 << 16, traj_offset=0, stream=None,
                device="cuda", soft_temperature=None) -> GRNForward:
    """ssa_grn_forward. W1 [n_hid, n_in] and W2 [n_out, n_hid] are rounded to bf16; x_img int counts.
    soft_temperature: run the soft forward of Eq. 4 at that T instead (float observables); a recorded soft run
    is differentiated by grn_backward at the same T (the exact gradient of the relaxed model)."""
    dev = torch.device(device)
    W1b = _bf16_bits(W1).to(dev)
    W2b = _bf16_bits(W2).to(dev)
    b1t, b2t, ldt = (_as_cuda(v, torch.float32, dev) for v in (b1, b2, log_d))
    x = _as_cuda(x_img, torch.int32, dev)
    ts = _as_cuda(sample_times, torch.float64, dev)
    n_img = int(x.shape[0])
    n = n_img * int(traj_per_img)
    S = int(ts.numel())
    soft = soft_temperature is not None
    opts = make_opts("hold", record, ckpt_interval, max_steps, selector="soft" if soft else "gumbel",
                     temperature=soft_temperature)
    L = _lib.lib()
    need = int(L.ssa_grn_workspace_bytes(grn.handle, n_img, traj_per_img, S, ctypes.byref(opts)))
    if need == 0:
        raise SSAError("invalid arguments for ssa_grn_workspace_bytes")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    obs = torch.empty((n, S, grn.n_out), dtype=torch.float32 if soft else torch.int32, device=dev)
    draws = torch.empty(n, dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    h = ctypes.c_void_p()
    check(L.ssa_grn_forward(grn.handle, _ptr(W1b), _ptr(b1t), _ptr(W2b), _ptr(b2t), _ptr(ldt), n_img,
                            int(traj_per_img), int(traj_offset), _ptr(x), float(t_end), _ptr(ts), S,
                            ctypes.c_uint64(int(seed) & (2**64 - 1)), ctypes.byref(opts), _ptr(ws), need, _ptr(obs),
                            _ptr(draws), _ptr(status), _stream(stream), ctypes.byref(h)))
    run = Run(h, ws, grn, n, S, grn.n_out, 0)
    run._keep = (W1b, W2b, b1t, b2t, ldt, x, ts)
    return GRNForward(obs, draws, status, run)


def grn_backward(fwd: GRNForward, dl_dobs: torch.Tensor, temperature: float, stream=None) -> dict:
    """ssa_grn_backward: gradients of W1, b1, W2, b2 and log_d (float32)."""
    run = fwd.run
    g = dl_dobs.to(torch.float32).contiguous()
    stride = run.S * run.n_obs if tuple(g.shape) == (run.n_traj, run.S, run.n_obs) else 0
    if stride == 0 and tuple(g.shape) != (run.S, run.n_obs):
        raise SSAError("dl_dobs has the wrong shape")
    net = run.net
    dev = g.device
    out = {"W1": torch.empty((net.n_hid, net.n_in), device=dev), "b1": torch.empty(net.n_hid, device=dev),
           "W2": torch.empty((net.n_out, net.n_hid), device=dev), "b2": torch.empty(net.n_out, device=dev),
           "log_d": torch.empty(net.n_hid + net.n_out, device=dev)}
    check(_lib.lib().ssa_grn_backward(run.handle, _ptr(g), stride, ctypes.c_float(float(temperature)),
                                      _ptr(out["W1"]), _ptr(out["b1"]), _ptr(out["W2"]), _ptr(out["b2"]),
                                      _ptr(out["log_d"]), _stream(stream)))
    return out


def grn_activations(fwd: GRNForward, n_img: int, stream=None):
    """E1 [n_img, n_hid] computed on the tensor cores, and the (inexact-input, timeout) flags."""
    run = fwd.run
    E1 = torch.empty((n_img, run.net.n_hid), dtype=torch.float32, device=run.workspace.device)
    flags = (ctypes.c_int32 * 2)()
    check(_lib.lib().ssa_grn_activations(run.handle, _ptr(E1), flags, _stream(stream)))
    return E1, (int(flags[0]), int(flags[1]))


class SSAFunction(torch.autograd.Function):
    """obs = SSA(theta) with the straight-through gradient of Eqs. 5 and 7 in backward."""

    @staticmethod
    def forward(ctx, log_rates, net, n_traj, x0, t_end, sample_times, obs_species, seed, readout, temperature,
                ckpt_interval, max_steps, traj_offset, selector="gumbel"):
        res = forward(net, log_rates.detach(), n_traj, x0, t_end, sample_times, obs_species, seed, readout=readout,
                      record=True, ckpt_interval=ckpt_interval, max_steps=max_steps, traj_offset=traj_offset,
                      selector=selector, temperature=temperature)
        ctx.run = res.run
        ctx.temperature = float(temperature)
        ctx.status = res.status
        return res.obs.to(torch.float32)

    @staticmethod
    def backward(ctx, grad_obs):
        g = backward(ctx.run, grad_obs, ctx.temperature)
        return (g,) + (None,) * 13


def simulate(net: Network, log_rates: torch.Tensor, n_traj: int, x0, t_end: float, sample_times, obs_species,
             seed: int, readout="linear", temperature=1.0, ckpt_interval=64, max_steps=1 << 20, traj_offset=0,
             soft=False):
    """Differentiable forward: obs [n_traj, S, n_obs] float32; obs.backward() fills log_rates.grad. soft: the
    relaxed forward of Eq. 4 at `temperature` and the exact gradient of that model (instead of the exact
    forward with the straight-through gradient)."""
    return SSAFunction.apply(log_rates, net, n_traj, x0, t_end, sample_times, obs_species, seed, readout,
                             temperature, ckpt_interval, max_steps, traj_offset, "soft" if soft else "gumbel")
