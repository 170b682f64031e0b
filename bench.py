"""Benchmark: SSA steps/s of the forward and of forward + straight-through adjoint on one GB300.

Workload (one bench step = one pass of the whole hot path over one batch):
    2A <-> B (a1 = k1 A (A - 1)/2, a2 = k2 B), 65,536 trajectories from A = 100, B = 0 to t_end = 50,
    50 uniform samples of A with LINEAR readout, evaluated at k = (0.02, 0.05); record the event log
    with checkpoints every K = 64 steps; ensemble mean; loss = mean_s (mean A(t_s) - target_s)^2 with
    the target generated at k = (0.01, 0.1) (seed 1); the straight-through gradient at each of the three
    temperatures T in {0.1, 0.5, 1.0} (one reverse walk for all three). Each step uses a fresh Philox seed.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line. `value` is forward+adjoint SSA steps per second (whole job); the forward-only
rate and the ratio are reported beside it. Under torchrun each rank simulates its own trajectory
ids (weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SSA steps/s fwd and fwd+adjoint on 1 GB300 vs plain fwd; grad rel err vs FP64"
WORKLOAD = ("c2_dimer_2a_b_fwd_adj: 2A<->B, 65,536 traj, t_end=50, 50 LINEAR samples, K=64, one forward + the "
            "gradient at each of T = 0.1, 0.5, 1.0")
TEMPS = (0.1, 0.5, 1.0)
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


# --------------------------------------------------------------------------------------------
# Issue-slot roofline of the SSA kernels. The unit is one SSA step; its
# algorithmic cost is the minimal number of issue slots (thread instructions) of the method's
# arithmetic on sm_103, with an accurate logarithm costed at its measured throughput on this GPU
# (ssa_pipe_rates: 128 issue slots per SM per clock / exponential variates per SM per clock). The peak is the SM
# issue rate: 152 SMs x 4 schedulers x 32 lanes x the sampled SM clock.
# --------------------------------------------------------------------------------------------
def instr_per_step_fwd(M: int, log_slots: float) -> float:
    nb = (M + 4) // 4
    philox = 60 * nb                          # 10 rounds x (2 wide multiplies, 2 XOR3, 2 key adds)
    variates = (2 + log_slots) * (M + 1)     # u from the bits (2) and an accurate -ln u
    reactions = 12 * M                        # propensity (5), a0 add (1), race (2 mul, compare, 3 select)
    step = 20                                 # tau (2), FP64 clock add + compare (3), update (8), log (4), loop (3)
    return philox + variates + reactions + step


def instr_per_step_bwd(M: int, log_slots: float) -> float:
    # the forward step recomputed, then per reaction: 2 lg2 + sub (log key), ex2 + mul (soft weight),
    # stoichiometric dot (6), psi (5), dA (2), state adjoint (8); per step: readout, reversal, event (20)
    return instr_per_step_fwd(M, log_slots) + 25 * M + 20


def instr_per_step_bwd_multi(M: int, log_slots: float, n_temps: int) -> float:
    # one walk for n_temps temperatures: the forward step recomputed once, the temperature-dependent part
    # (soft weights, psi, state adjoint, readout) once per temperature
    return instr_per_step_fwd(M, log_slots) + n_temps * (25 * M + 20)


def sm_issue_peak(sm_mhz: float, n_sm: int = 152) -> float:
    return n_sm * 4 * 32 * sm_mhz * 1e6


def profiled_traffic(kind: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's sources are unchanged."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic_c2.json")))
        k = rec["kernels"][kind]
        h = hashlib.sha256()
        for f in k["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2602_19775_gb300", "csrc", f), "rb").read())
    except (OSError, ValueError, KeyError):
        return None
    if h.hexdigest()[:16] != k["source_sha256_16"]:
        return None
    return k["dram_read_bytes"] + k["dram_write_bytes"]


# --------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline sample)
# --------------------------------------------------------------------------------------------
def oracle_sample(seconds: float, chunk: int, seed0: int = 1000):
    import ssa_workloads as W
    from oracle import native
    wl = W.config_c2()
    theta = wl.log_rates.astype(np.float32).astype(np.float64)
    cores = os.cpu_count() or 1
    steps, t0, it = 0, time.perf_counter(), 0
    target = np.linspace(90.0, 27.0, len(wl.sample_times))
    while True:
        fw = native.run(wl.net, theta, wl.x0, chunk, wl.t_end, wl.sample_times, wl.obs_species, seed0 + it,
                        native.LINEAR, max_steps=wl.max_steps, n_threads=cores)
        m = fw.obs[:, :, 0].mean(0)
        g = np.broadcast_to((2.0 * (m - target) / len(m) / chunk)[None, :, None], fw.obs.shape).copy()
        r = native.run(wl.net, theta, wl.x0, chunk, wl.t_end, wl.sample_times, wl.obs_species, seed0 + it,
                       native.LINEAR, max_steps=wl.max_steps, dl_dobs=g, temperature=TEMPS[it % 3], n_threads=cores)
        steps += int(r.draws.sum())
        it += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, cores, it * chunk, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import native
    native.build()
    chunk = args.ref_chunk
    for _ in range(args.warmup):
        oracle_sample(0.0, chunk)
    t0 = time.perf_counter()
    total_steps = 0.0
    for s in range(args.steps):
        rate, cores, ntraj, dt = oracle_sample(0.0, chunk, seed0=2000 + 7 * s)
        total_steps += rate * dt
    dt = time.perf_counter() - t0
    value = total_steps / dt
    line = {
        "metric": METRIC, "value": value, "unit": "SSA steps/s (fwd+adj)", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample": f"{chunk} trajectories per step (oracle fwd+adj)"},
        "cpu_baseline": {"value": value, "unit": "SSA steps/s (fwd+adj)", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {chunk} trajectories of the workload"},
        "e2e": {"value": value, "unit": "SSA steps/s (fwd+adj)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import ssa_workloads as W
    from paper_2602_19775_gb300 import ssa

    wl = W.config_c2(n_traj=args.n_traj)
    n = wl.n_traj
    S = len(wl.sample_times)
    from paper_2602_19775_gb300.shard import max_over_ranks, shard_range, total_over_ranks
    offset, _ = shard_range(n * world, rank, world)  # each rank simulates its own global trajectory ids
    net = ssa.Network(wl.net)
    theta = torch.tensor(wl.log_rates.astype(np.float32), device=dev)
    x0 = torch.tensor(wl.x0, device=dev)
    ts = torch.tensor(wl.sample_times, device=dev)
    obs_sp = torch.tensor(wl.obs_species, device=dev)
    true_theta = torch.tensor(np.log([0.01, 0.1]).astype(np.float32), device=dev)
    max_steps = 2048
    stream = torch.cuda.current_stream()

    # target: ensemble mean of A at the true rates, seed 1 (setup, untimed)
    tfw = ssa.forward(net, true_theta, n, x0, wl.t_end, ts, obs_sp, 1, readout="linear", max_steps=max_steps,
                      traj_offset=offset)
    target = ssa.ensemble_mean(tfw.obs)[:, 0].clone()
    del tfw

    opts = ssa.make_opts("linear", True, 64, max_steps)
    ws = torch.empty(ssa.workspace_bytes(net, n, S, opts), dtype=torch.uint8, device=dev)
    obs = torch.empty((n, S, 1), dtype=torch.float32, device=dev)
    dtheta = torch.empty(2, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    dtheta3 = torch.empty((len(TEMPS), 2), dtype=torch.float32, device=dev)

    def step(seed, T=None, ev=None, specialize=True, separate=False):
        """T None: the gradient at every temperature of TEMPS (one walk, or one per T with separate);
        else the gradient at T alone."""
        if ev is not None:
            ev[0].record(stream)
        fw = ssa.forward(net, theta, n, x0, wl.t_end, ts, obs_sp, seed, readout="linear", record=True,
                         max_steps=max_steps, traj_offset=offset, workspace=ws, obs_out=obs, specialize=specialize)
        if ev is not None:
            ev[1].record(stream)
        m = ssa.ensemble_mean(obs)[:, 0]
        dl = (2.0 / (S * n)) * (m - target)          # dL/dobs, the same for every trajectory
        if ev is not None:
            ev[2].record(stream)
        if T is not None:
            ssa.backward(fw, dl.view(S, 1), T, out=dtheta)
        elif separate:
            for q, Tq in enumerate(TEMPS):
                ssa.backward(fw, dl.view(S, 1), Tq, out=dtheta3[q])
        else:
            ssa.backward_multi(fw, dl.view(S, 1), TEMPS, out=dtheta3)
        if ev is not None:
            ev[3].record(stream)
        return fw

    def fwd_only(seed, ev=None, specialize=True, selector="gumbel"):
        if ev is not None:
            ev[0].record(stream)
        fw = ssa.forward(net, theta, n, x0, wl.t_end, ts, obs_sp, seed, readout="linear", record=False,
                         max_steps=max_steps, traj_offset=offset, workspace=ws, obs_out=obs, specialize=specialize,
                         selector=selector)
        if ev is not None:
            ev[1].record(stream)
        return fw

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for w in range(args.warmup):
        step(100 + w)
        fwd_only(100 + w)
    barrier()

    # ---- timed: forward + adjoint ----
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    draws_tot = torch.zeros((), dtype=torch.int64, device=dev)
    with ClockSampler(local) as clk:
        barrier()
        for s in range(K):
            fw = step(1000 + s, ev=evs[s])
            draws_tot += fw.draws.sum()
            flush.fill_(s & 0xFF)                    # L2 flush between steps, outside the events
        barrier()
        # ---- timed: forward only (same seeds) ----
        fev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
        fdraws = torch.zeros((), dtype=torch.int64, device=dev)
        for s in range(K):
            fw = fwd_only(1000 + s, fev[s])
            fdraws += fw.draws.sum()
            flush.fill_(s & 0xFF)
        barrier()
    variant = fw.run.variant
    # the plain direct method (one uniform and a cumulative search per step) on the same steps: the
    # plain-SSA forward the method's forward and forward+adjoint compare with (outside the timed region)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    pdraws = torch.zeros((), dtype=torch.int64, device=dev)
    for w in range(2):
        fwd_only(100 + w, selector="direct")
    for s in range(K):
        pfw = fwd_only(1000 + s, pev[s], selector="direct")
        pdraws += pfw.draws.sum()
        flush.fill_(s & 0xFF)
    torch.cuda.synchronize()
    plain_fwd = float(pdraws.item()) / (sum(e[0].elapsed_time(e[1]) for e in pev) / 1e3)
    del pfw
    # the same steps on the generic (table-driven) thread kernels (one walk per temperature there), with one
    # walk per temperature on the specialised kernels, and with the gradient at one temperature per step (T
    # cycled), for comparison (outside the timed region)
    def compare(**kw):
        cev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        cdraws = torch.zeros((), dtype=torch.int64, device=dev)
        cyc = kw.pop("cycle", False)
        for w in range(2):
            step(100 + w, T=TEMPS[w % 3] if cyc else None, **kw)
        for s in range(K):
            cfw = step(1000 + s, T=TEMPS[s % 3] if cyc else None, ev=cev[s], **kw)
            cdraws += cfw.draws.sum()
            flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        return {"variant": cfw.run.variant,
                "fwd_adj_steps_per_s": float(cdraws.item()) / (sum(e[0].elapsed_time(e[3]) for e in cev) / 1e3),
                "forward_record_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in cev])),
                "adjoint_ms": float(np.mean([e[2].elapsed_time(e[3]) for e in cev]))}

    generic = compare(specialize=False)
    separate = compare(separate=True)
    single_T = compare(cycle=True)
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    bwd_ms = [e[2].elapsed_time(e[3]) for e in evs]
    fonly_ms = [e[0].elapsed_time(e[1]) for e in fev]
    steps_total = int(draws_tot.item())
    t_step = float(np.sum(step_ms)) / 1e3
    t_fonly = float(np.sum(fonly_ms)) / 1e3
    t_step, t_fonly = max_over_ranks(t_step, dev), max_over_ranks(t_fonly, dev)
    steps_total, fsteps = total_over_ranks(steps_total, dev), total_over_ranks(int(fdraws.item()), dev)
    value = steps_total / t_step
    fwd_value = fsteps / t_fonly

    # ---- end to end through the API with host buffers ----
    pin = lambda a: torch.tensor(a).pin_memory()  # noqa: E731
    h_theta, h_x0, h_ts, h_sp = pin(wl.log_rates.astype(np.float32)), pin(wl.x0), pin(wl.sample_times), pin(wl.obs_species)
    h_target = target.cpu().pin_memory()
    h_out = torch.empty((len(TEMPS), 2), dtype=torch.float32).pin_memory()
    h_mean = torch.empty(S, dtype=torch.float32).pin_memory()
    d_theta, d_x0, d_ts, d_sp, d_target = (torch.empty_like(t, device=dev) for t in (h_theta, h_x0, h_ts, h_sp, h_target))
    e_steps = 0
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(K):
        for d, h in ((d_theta, h_theta), (d_x0, h_x0), (d_ts, h_ts), (d_sp, h_sp), (d_target, h_target)):
            d.copy_(h, non_blocking=True)
        fw = ssa.forward(net, d_theta, n, d_x0, wl.t_end, d_ts, d_sp, 5000 + s, readout="linear", record=True,
                         max_steps=max_steps, traj_offset=offset, workspace=ws, obs_out=obs)
        m = ssa.ensemble_mean(obs)[:, 0]
        dl = (2.0 / (S * n)) * (m - d_target)
        ssa.backward_multi(fw, dl.view(S, 1), TEMPS, out=dtheta3)
        h_out.copy_(dtheta3, non_blocking=True)
        h_mean.copy_(m, non_blocking=True)
        e_steps += int(fw.draws.sum().item())   # also synchronises the step, as a user's loop would
    e1.record(stream)
    barrier()
    e2e_t = e0.elapsed_time(e1) / 1e3
    h2d = sum(t.numel() * t.element_size() for t in (h_theta, h_x0, h_ts, h_sp, h_target))
    d2h = h_out.numel() * 4 + h_mean.numel() * 4 + 8
    e2e_value = e_steps * world / e2e_t

    # ---- gradient error vs the FP64 oracle on a subset (rank 0, outside the timed regions) ----
    grad_err = None
    cpu_base = None
    if rank == 0 and not args.no_oracle:
        grad_err = grad_error_subset(ssa, net, wl, dev)
        rate, cores, ntraj, dt = oracle_sample(args.cpu_seconds, 4096)
        cpu_base = {"value": rate, "unit": "SSA steps/s (fwd+adj)", "cores": cores, "kind": "oracle",
                    "sample": f"{ntraj} trajectories of the workload, fwd + adj, {dt:.1f} s"}

    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    legs = set() if args.no_extra else {x for x in args.legs.split(",") if x}
    orc = not args.no_oracle
    osc = (oscillator_extra(ssa, dev, oracle=orc, n_fwd=args.osc_traj, n_samples=args.osc_samples)
           if (rank == 0 and "oscillator" in legs) else None)
    batch = (uneven_batch_extra(ssa, dev, args.batch_scale, sequential=args.batch_sequential, oracle=orc)
             if (rank == 0 and "batch" in legs) else None)
    grn = grn_extra(ssa, dev, n_img=args.grn_images, oracle=orc) if (rank == 0 and "grn" in legs) else None
    warp = warp_extra(ssa, dev, n=args.warp_traj, oracle=orc) if (rank == 0 and "warp" in legs) else None
    c3 = c3_extra(ssa, dev, oracle=orc) if (rank == 0 and "c3" in legs) else None
    ion = ion_channel_extra(ssa, dev, n=args.ion_traj, oracle=orc) if (rank == 0 and "ion" in legs) else None
    c1 = c1_extra(ssa, dev) if (rank == 0 and "c1" in legs) else None
    bias = st_bias_extra(ssa, dev, target) if (rank == 0 and orc and "bias" in legs) else None
    M = wl.net.n_reactions
    rates = ssa.pipe_rates()
    log_slots = 128.0 / rates["neglog"]
    lg2_slots = 128.0 / rates["lg2"]
    bwd_s = float(np.mean(bwd_ms)) / 1e3
    fwd_s = float(np.mean(fwd_ms)) / 1e3
    per_launch_steps = steps_total / world / K
    nT = len(TEMPS)
    # issue slots per step with the exponential variate priced as one MUFU.LG2 (the roofline's count), and
    # with the accurate logarithm the kernels call priced at its measured throughput
    ach_b = instr_per_step_bwd_multi(M, lg2_slots, nT) * per_launch_steps / bwd_s
    ach_f = instr_per_step_fwd(M, lg2_slots) * per_launch_steps / fwd_s
    ach_b_log = instr_per_step_bwd_multi(M, log_slots, nT) * per_launch_steps / bwd_s
    ach_f_log = instr_per_step_fwd(M, log_slots) * per_launch_steps / fwd_s
    peak = sm_issue_peak(sm_mhz, rates["sm_count"])
    if batch and "instr_per_s_T" in batch:
        batch["alu_frac"] = batch["instr_per_s_T"] * 1e12 / peak
    if warp:
        warp["fwd_alu_frac"] = warp["fwd_instr_per_s_T"] * 1e12 / peak
        warp["adj_alu_frac"] = warp["adj_instr_per_s_T"] * 1e12 / peak
    dominant = "adjoint" if bwd_s >= fwd_s else "forward"
    ach = ach_b if dominant == "adjoint" else ach_f
    ach_log = ach_b_log if dominant == "adjoint" else ach_f_log
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "SSA steps/s (fwd+adj)",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_step / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64 clock, int32 counts)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_traj_per_gpu": n, "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"trajectory shards x{world}"},
        "fwd_steps_per_s": fwd_value,
        "fwd_adj_over_fwd": value / fwd_value,
        "plain_direct_fwd_steps_per_s": plain_fwd,
        "fwd_adj_over_plain_fwd": value / plain_fwd,
        "fwd_over_plain_fwd": fwd_value / plain_fwd,
        "ssa_steps_per_bench_step": steps_total / K,
        "grad_rel_err_vs_fp64": grad_err,
        "st_gradient_bias": bias,
        "kernel_ms": {"forward_record": float(np.mean(fwd_ms)), "adjoint": float(np.mean(bwd_ms)),
                      "forward_only": float(np.mean(fonly_ms))},
        "kernel_variant": {1: "generic thread", 2: "network-specialised thread (NVRTC)", 32: "warp"}[variant],
        "generic_thread_kernels": generic,
        "one_walk_per_temperature": separate,
        "single_temperature_step": dict(single_T, note="forward + the gradient at one T per step (T cycled)"),
        "roofline": {"bound": "alu", "kernel": dominant, "achieved": ach / 1e12, "peak": peak / 1e12,
                     "unit": "T thread-instr/s", "frac": ach / peak, "traffic": profiled_traffic(dominant),
                     "count": "exponential variate priced as one MUFU.LG2 (measured rate); adjoint = one walk for "
                              "the three temperatures",
                     "algorithmic_instr_per_step": {"forward": instr_per_step_fwd(M, lg2_slots),
                                                    "adjoint": instr_per_step_bwd_multi(M, lg2_slots, nT)},
                     "forward_frac": ach_f / peak,
                     "frac_logf_priced": ach_log / peak, "forward_frac_logf_priced": ach_f_log / peak,
                     "peak_basis": f"{rates['sm_count']} SM x 4 x 32 lanes x {sm_mhz:.0f} MHz (sampled median)",
                     "pipe_rates_per_sm_clk": {k: round(v, 3) for k, v in rates.items()}},
        "oscillator": osc,
        "uneven_batch": batch,
        "grn": grn,
        "warp_kernels": warp,
        "oscillator_full": c3,
        "c1_forward": c1,
        "ion_channel": ion,
        "paper_context": "1.9e9 SSA steps/s forward on the oscillator, RTX 6000 Ada + TF 2.20 (a different machine)",
        "cpu_baseline": cpu_base,
        "e2e": {"value": e2e_value, "unit": "SSA steps/s (fwd+adj)", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 12 * K,  # forward 3 (rates, input checks, SSA), mean 2, backward 1 + 2 per temperature
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def oscillator_extra(ssa, dev, n_fwd: int = 1 << 20, n_adj: int = 1 << 16, t_end: float = 10.0, reps: int = 2,
                     oracle: bool = True, n_samples: int = 10):
    """Forward-only and forward+adjoint SSA steps/s on the activator-repressor oscillator (the workload of the
    paper's throughput figure), 10 LINEAR samples of R, horizon t_end (truncated from 400 to bound the event
    log), timed with CUDA events after one warm-up launch."""
    import torch

    import ssa_workloads as W
    wl = W.config_c3(n_traj=n_fwd, t_end=t_end, S=n_samples)
    net = ssa.Network(wl.net)
    th = torch.tensor(wl.log_rates.astype(np.float32), device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"Vilar oscillator, 9 species, 16 reactions, t_end={t_end}, {n_samples} LINEAR samples of R",
           "selectors": "forward: Gumbel-max (the method); forward_direct: the plain direct method; forward_soft: "
                        "the relaxed forward of Eq. 4 at T = 0.5 (its own, different, step count); "
                        "forward_generic: the Gumbel-max forward on the generic table-driven kernels"}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for mode, n in (("forward", n_fwd), ("forward_generic", n_fwd), ("forward_direct", n_fwd), ("forward_soft", n_fwd),
                    ("forward_adjoint", n_adj)):
        rec = mode == "forward_adjoint"
        sel = {"forward_direct": "direct", "forward_soft": "soft"}.get(mode, "gumbel")
        spec_k = mode != "forward_generic"
        ms, steps = 0.0, 0
        for r in range(reps + 1):
            if r == 1:
                torch.cuda.synchronize()
            if r >= 1:
                ev[0].record(stream)
            fw = ssa.forward(net, th, n, wl.x0, t_end, wl.sample_times, wl.obs_species, 50 + r, readout="linear",
                             record=rec, max_steps=1 << 16, selector=sel, temperature=0.5 if sel == "soft" else None,
                             specialize=spec_k)
            if rec:
                dl = torch.full((len(wl.sample_times), 1), 1.0 / n, device=dev)
                ssa.backward(fw, dl, 0.1)
            if r >= 1:
                ev[1].record(stream)
                torch.cuda.synchronize()
                ms += ev[0].elapsed_time(ev[1])
                steps += int(fw.draws.sum().item())
            del fw
        out[mode] = {"n_traj": n, "steps": steps // reps, "ms": ms / reps, "steps_per_s": steps / (ms / 1e3)}
    if oracle:
        m = 256
        out["grad_rel_err_vs_fp64"] = oracle_grad_err(
            ssa, dev, wl.net, wl.log_rates.astype(np.float32), wl.x0, m, t_end, wl.sample_times, wl.obs_species, 51,
            "linear", 0.1, 1 << 16, W.seeded_dl_dobs(5, m, len(wl.sample_times), 1, scale=1.0 / m))
    return out


def ion_channel_extra(ssa, dev, n: int = 262144, reps: int = 3, T: float = 0.05, oracle: bool = True):
    """The ion-channel workload of Section 4.4: two channels C <-> O -> I from all closed, 262,144
    trajectories, the open count averaged exactly over 800 bins of 0.01 ms (8 ms). One gradient step =
    recorded forward + the loss gradient of the bin-mean MSE against a target + the straight-through
    adjoint; timed with CUDA events after one warm-up step, and a forward alone beside it."""
    import torch

    import ssa_workloads as W
    spec = W.ion_channel_coi()
    net = ssa.Network(spec)
    ts = W.uniform_sample_grid(8.0, 800)
    th = torch.tensor(spec.log_rates.astype(np.float32), device=dev)
    target = ssa.forward(net, th, n, spec.x0, 8.0, ts, [1], 999, readout="bin", max_steps=64).obs.mean(0)
    theta = th + 0.2
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"workload": f"ion channel C <-> O -> I, 2 channels, {n} trajectories, 800 bins of 0.01 ms, BIN readout"}
    for mode in ("forward", "gradient_step"):
        ms, steps = 0.0, 0
        for r in range(reps + 1):
            if r == 1:
                torch.cuda.synchronize()
            if r >= 1:
                ev[0].record(stream)
            fw = ssa.forward(net, theta, n, spec.x0, 8.0, ts, [1], 60 + r, readout="bin",
                             record=mode != "forward", max_steps=64)
            if mode != "forward":
                dl = 2.0 * (fw.obs.mean(0) - target) / (target.numel() * n)
                ssa.backward(fw, dl, T)
            if r >= 1:
                ev[1].record(stream)
                torch.cuda.synchronize()
                ms += ev[0].elapsed_time(ev[1])
                steps += int(fw.draws.sum().item())
            del fw
        out[mode] = {"ms": ms / reps, "ssa_steps": steps // reps, "steps_per_s": steps / (ms / 1e3)}
    # the forward is bound by the stores of the bin rows: 4 B per bin per trajectory
    rows = 4.0 * n * len(ts)
    out["forward"]["bin_row_bytes"] = rows
    out["forward"]["achieved_gbs"] = rows / (out["forward"]["ms"] / 1e3) / 1e9
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        out["forward"]["hbm_frac"] = out["forward"]["achieved_gbs"] / hbm
        out["forward"]["peak_basis"] = f"{hbm:.0f} GB/s of measured (copy)"
    except (OSError, ValueError, KeyError):
        out["forward"]["hbm_frac"] = None
    out["paper_context_ms_per_epoch"] = 112e3 / 400
    if oracle:
        m = 4096
        out["grad_rel_err_vs_fp64"] = oracle_grad_err(
            ssa, dev, spec, (spec.log_rates + 0.2).astype(np.float32), spec.x0, m, 8.0, ts, [1], 61, "bin", T, 64,
            W.seeded_dl_dobs(6, m, len(ts), 1, scale=1.0 / m))
    return out


def uneven_batch_extra(ssa, dev, traj_scale: float, reps: int = 1, sequential: bool = False, oracle: bool = True):
    """The uneven batch of random networks (256 networks, N in [2, 64], M in [4, 512], trajectories per
    network log-uniform in [256, 65,536] x traj_scale, t_end = 10, 20 LINEAR samples, T = 0.5, loss
    weights c ~ N(0, 1) on the trajectory means): forward + adjoint of every network in one CUDA-graph
    launch of the persistent batch kernels, after the pilot autotuner (variant and checkpoint interval). Event
    logs are sized from the committed oracle pilot (twice its maximum draws + 256). With `sequential`, also
    times the same work as one forward and one backward call per network, for comparison."""
    import torch

    import ssa_workloads as W
    path = os.path.join(ROOT, "tests", "golden", "c4_pilot.json")
    if not os.path.exists(path):
        return {"skipped": "no oracle pilot file"}
    pilot = json.load(open(path))
    wl = W.config_c4(n_nets=len(pilot["accepted"]), traj_scale=traj_scale, rejected=pilot["rejected"])
    assert [a["draw"] for a in pilot["accepted"]] == wl.draw_index.tolist()
    max_steps = [int(2 * a["max_draws"] + 256) for a in pilot["accepted"]]
    nets = [ssa.Network(spec) for spec in wl.nets]
    items = []
    for q, spec in enumerate(wl.nets):
        items.append(dict(net=nets[q], log_rates=spec.log_rates.astype(np.float32), n_traj=int(wl.n_traj[q]),
                          x0=spec.x0, t_end=wl.t_end, sample_times=wl.sample_times, obs_species=wl.obs_species[q],
                          seed=900 + q, max_steps=max_steps[q], shared_dl=True))
    b = ssa.Batch(items, readout="linear", temperature=wl.temperature, device=dev)
    t0 = time.time()
    b.autotune(pilot_traj=64)
    t_tune = time.time() - t0
    for q in range(len(items)):
        b.dl_dobs[q].copy_(torch.tensor(wl.loss_weights[q] / wl.n_traj[q], dtype=torch.float32))
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(stream):
        b.run(use_graph=True, stream=stream)  # lays out the workspace, captures and runs the graph once
        stream.synchronize()
        ev[0].record(stream)
        for _ in range(reps):
            b.run(use_graph=True, stream=stream)
        ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    steps, variants, mism, bad = 0, {1: 0, 32: 0}, 0, 0
    per_item = []
    Ks = [b.ckpt_interval(q) for q in range(len(items))]
    for q in range(len(items)):
        d, st, mm = b.outputs(q, stream=stream)
        sq = int(d.sum().item())
        steps += sq
        per_item.append(sq)
        mism += mm
        bad += int((st > 2).sum().item())
        variants[b.variant(q)] += 1
    rates = ssa.pipe_rates()
    log_slots = 128.0 / rates["neglog"]
    instr = sum(per_item[q] * (instr_per_step_fwd(wl.nets[q].n_reactions, log_slots)
                               + instr_per_step_bwd(wl.nets[q].n_reactions, log_slots)) for q in range(len(items)))
    out = {"workload": f"{len(items)} random networks, N in [2, 64], M in [4, 512], t_end=10, 20 LINEAR samples, "
                       f"T=0.5, trajectories per network log-uniform [256, 65536] x {traj_scale:g}",
           "n_traj_total": int(wl.n_traj.sum()), "ssa_steps": steps, "ms": ms, "steps_per_s": steps / (ms / 1e3),
           "unit": "SSA steps/s (fwd+adj)", "variants": {"thread": variants[1], "warp": variants[32]},
           "workspace_gb": b.workspace_bytes() / 1e9, "autotune_s": t_tune, "adjoint_mismatches": mism,
           "non_ok_trajectories": bad, "instr_per_s_T": instr / (ms / 1e3) / 1e12,
           "redraws": len(pilot["rejected"]), "trajectory_scale": traj_scale,
           "ckpt_interval": {"min": int(min(Ks)), "median": float(np.median(Ks)), "max": int(max(Ks))}}
    del b
    if sequential:
        torch.cuda.synchronize()
        ev[0].record()
        for q, it in enumerate(items):
            fw = ssa.forward(nets[q], torch.tensor(it["log_rates"], device=dev), it["n_traj"], it["x0"], wl.t_end,
                             wl.sample_times, it["obs_species"], it["seed"], readout="linear", record=True,
                             max_steps=it["max_steps"])
            dl = torch.tensor(wl.loss_weights[q] / wl.n_traj[q], dtype=torch.float32, device=dev)
            ssa.backward(fw, dl, wl.temperature)
            del fw
        ev[1].record()
        torch.cuda.synchronize()
        out["per_network_calls_ms"] = ev[0].elapsed_time(ev[1])
    if oracle:
        out["grad_rel_err_vs_fp64"] = batch_grad_err(ssa, dev, wl, nets, max_steps)
    return out


def batch_grad_err(ssa, dev, wl, nets, max_steps, n_items: int = 16, n: int = 16):
    """Gradient error of the persistent batch against the FP64 oracle: the first n_items networks of the
    uneven batch, n trajectories each, one batch launch; per network the relative error on the trajectories
    whose event sequences and sample brackets agree; the largest over the networks and the norm-wise error
    of all their gradients stacked."""
    import torch

    from oracle import native
    items = [dict(net=nets[q], log_rates=wl.nets[q].log_rates.astype(np.float32), n_traj=n, x0=wl.nets[q].x0,
                  t_end=wl.t_end, sample_times=wl.sample_times, obs_species=wl.obs_species[q], seed=400 + q,
                  traj_offset=0, max_steps=max_steps[q]) for q in range(n_items)]
    b = ssa.Batch(items, readout="linear", temperature=wl.temperature, device=dev)
    dls = [np.random.default_rng(500 + q).standard_normal((n, len(wl.sample_times), len(wl.obs_species[q]))) / n
           for q in range(n_items)]
    for q in range(n_items):
        b.dl_dobs[q].copy_(torch.tensor(dls[q], dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()
    orcs, uses = [], []
    for q in range(n_items):
        spec = wl.nets[q]
        orc = native.run(spec, oracle_theta(spec.log_rates), spec.x0, n, wl.t_end,
                         wl.sample_times, wl.obs_species[q], 400 + q, native.LINEAR, max_steps=max_steps[q],
                         dl_dobs=dls[q], temperature=wl.temperature, ev_cap=max_steps[q])
        draws, status, _ = b.outputs(q)
        ev = b.events(q, max_steps[q]).cpu().numpy()
        same = np.all(ev == orc.events, axis=1) & (draws.cpu().numpy() == orc.draws)
        gb = b.brackets(q).cpu().numpy()
        ob = np.zeros_like(gb)
        for i in range(n):
            d = int(orc.draws[i])
            ob[i] = np.searchsorted(orc.times[i, :(d - 1 if orc.status[i] == 0 else d)], wl.sample_times, side="right")
        uses.append(same & np.all(gb == ob, axis=1))
        orcs.append(orc)
        dl2 = dls[q].copy()
        dl2[~uses[-1]] = 0
        b.dl_dobs[q].copy_(torch.tensor(dl2, dtype=torch.float32))
    b.run()
    torch.cuda.synchronize()
    errs, gs, refs = [], [], []
    for q in range(n_items):
        g = b.dtheta[q].double().cpu().numpy()
        ref = orcs[q].dtheta[uses[q]].sum(0)
        gs.append(g)
        refs.append(ref)
        if np.linalg.norm(ref) > 0:
            errs.append(float(np.linalg.norm(g - ref) / np.linalg.norm(ref)))
    G, R = np.concatenate(gs), np.concatenate(refs)
    return {"rel_err": float(np.linalg.norm(G - R) / np.linalg.norm(R)), "max_rel_err_per_network": max(errs),
            "networks": n_items, "n_traj_each": n, "compared": int(sum(u.sum() for u in uses)),
            "temperature": float(wl.temperature)}


def c3_extra(ssa, dev, n_fwd: int = 1 << 20, n_adj: int = 1 << 14, lag: int = 12, T: float = 0.1,
             oracle: bool = True):
    """The activator-repressor oscillator at its full configuration: 2^20 trajectories to t_end = 400 with 400
    LINEAR samples of R, forward only (one launch); then one trajectory chunk of n_adj with the event log
    (about 1.1e6 draws per trajectory, 2 bytes each) through forward + straight-through adjoint of the loss
    L = mean_s (m_s - m*_s)^2 + (c_lag - c*_lag)^2 on the ensemble mean m_s of R and the ensemble mean of the
    per-trajectory normalised autocovariance c at `lag` samples, at the true rates (targets from n_adj other
    trajectories, seed 1), T = 0.1. Over ~1e6 draws the straight-through recursion grows dL/dX geometrically
    (to ~1e70 per trajectory in binary64), so the chunk's adjoint is the wide-range one (a power-of-two
    exponent per trajectory, binary64 sums); its error against the FP64 oracle is measured on 16 trajectories
    at the same horizon."""
    import torch

    import ssa_workloads as W
    wl = W.config_c3(n_traj=n_fwd)
    net = ssa.Network(wl.net)
    S = len(wl.sample_times)
    true = torch.tensor(wl.log_rates.astype(np.float32), device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {"workload": f"Vilar oscillator, {n_fwd} trajectories, t_end={wl.t_end}, {S} LINEAR samples of R"}
    ssa.forward(net, true, 1024, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 9, readout="linear",
                max_steps=1 << 21)  # warm-up
    torch.cuda.synchronize()
    ev[0].record()
    fw = ssa.forward(net, true, n_fwd, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 10, readout="linear",
                     max_steps=1 << 21)
    ev[1].record()
    torch.cuda.synchronize()
    steps = int(fw.draws.sum().item())
    ms = ev[0].elapsed_time(ev[1])
    out["forward"] = {"n_traj": n_fwd, "ssa_steps": steps, "ms": ms, "steps_per_s": steps / (ms / 1e3),
                      "non_ok": int((fw.status > 1).sum().item())}
    del fw
    torch.cuda.empty_cache()

    def stats(obs):
        R = obs[:, :, 0].double()
        m = R.mean(0)
        x = R - R.mean(1, keepdim=True)
        c = (x[:, :-lag] * x[:, lag:]).mean(1) / (x * x).mean(1).clamp_min(1e-12)
        return m, c.mean()

    max_steps = 1_400_000
    tfw = ssa.forward(net, true, n_adj, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 1, readout="linear",
                      max_steps=max_steps)
    m_t, c_t = stats(tfw.obs)
    del tfw
    torch.cuda.empty_cache()
    ev[0].record()
    fw = ssa.forward(net, true, n_adj, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 3, readout="linear",
                     record=True, max_steps=max_steps)
    ev[1].record()
    obs = fw.obs.detach().clone().requires_grad_(True)
    m, c = stats(obs)
    loss = ((m - m_t) ** 2).mean() + (c - c_t) ** 2
    loss.backward()
    dl = obs.grad.float().contiguous()
    torch.cuda.synchronize()
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev2[0].record()
    g = ssa.backward_wide(fw, dl, T)
    ev2[1].record()
    torch.cuda.synchronize()
    steps = int(fw.draws.sum().item())
    fms, ams = ev[0].elapsed_time(ev[1]), ev2[0].elapsed_time(ev2[1])
    out["forward_adjoint_chunk"] = {
        "n_traj": n_adj, "ssa_steps": steps, "forward_record_ms": fms, "adjoint_ms": ams,
        "steps_per_s": steps / ((fms + ams) / 1e3), "workspace_gb": fw.run.workspace.numel() / 1e9,
        "loss": float(loss.item()), "grad_finite": bool(torch.isfinite(g).all().item()), "temperature": T,
        "grad_max_abs": float(g.abs().max().item()), "adjoint": "wide range (ssa_backward_wide)",
        "non_ok": int((fw.status > 1).sum().item()), "variant": fw.run.variant}
    del fw
    torch.cuda.empty_cache()
    if oracle:
        m = 16
        out["grad_rel_err_vs_fp64"] = oracle_grad_err(
            ssa, dev, wl.net, wl.log_rates.astype(np.float32), wl.x0, m, wl.t_end, wl.sample_times, wl.obs_species,
            17, "linear", T, 1_500_000, W.seeded_dl_dobs(13, m, S, 1, scale=1.0 / m), wide=True)
        torch.cuda.empty_cache()
    return out


def st_bias_extra(ssa, dev, target_linear, n: int = 65536, seeds=(11, 12, 13, 14), h: float = 1e-2):
    """Bias of the hard straight-through gradient (Section 3.4; it is not the gradient of the expected loss)
    on the 2A <-> B gradient workload at theta = log(0.02, 0.05), reported, not tested.

    LINEAR readout, the workload's own loss L = mean_s (mean A(t_s) - target_s)^2 against its sampled target:
    the straight-through gradient at T in {0.1, 0.5, 1.0} and the central finite difference with common random
    numbers (L(theta + h e_r) - L(theta - h e_r)) / 2h, h = 0.01 in log k, the same seed on both sides.
    HOLD readout, the loss against the exact mean m*_s of the master equation (Eq. 1) at the true rates: the
    same two estimates and the exact gradient of the infinite-ensemble loss, (2/S) sum_s (m_s - m*_s) dm_s/dtheta,
    from the block exponential of the generator. Each estimate is averaged over `seeds` (batches of n
    trajectories) with its standard error; the relative errors are |g - g_ref| / |g_ref|."""
    import torch

    import ssa_workloads as W
    from oracle import cme
    wl = W.config_c2(n_traj=n)
    net = ssa.Network(wl.net)
    S = len(wl.sample_times)
    theta0 = wl.log_rates.astype(np.float32).astype(np.float64)
    # exact master-equation means and gradient (51 states; A + 2B = 100)
    states, idx = cme.reachable_states(wl.net, wl.x0)
    p0 = np.zeros(len(states))
    p0[idx[tuple(int(v) for v in wl.x0)]] = 1.0
    A = np.array([st[0] for st in states], dtype=np.float64)
    m_true = cme.transient(cme.generator(wl.net, np.log([0.01, 0.1]), states, idx), p0, wl.sample_times) @ A
    Q = cme.generator(wl.net, theta0, states, idx)
    m0 = cme.transient(Q, p0, wl.sample_times) @ A
    dm = np.stack([cme.transient_gradient(Q, cme.generator_derivative(wl.net, theta0, states, idx, r), p0,
                                          wl.sample_times) @ A for r in range(2)])
    g_cme = (2.0 / S) * dm @ (m0 - m_true)
    targets = {"linear": target_linear.double().cpu().numpy(), "hold": m_true}

    def mean_A(theta, seed, readout, record):
        fw = ssa.forward(net, torch.tensor(theta.astype(np.float32), device=dev), n, wl.x0, wl.t_end,
                         wl.sample_times, wl.obs_species, seed, readout=readout, record=record, max_steps=4096)
        return fw, fw.obs[:, :, 0].double().mean(0)

    out = {"workload": f"2A<->B, {n} traj x {len(seeds)} seeds, theta = log(0.02, 0.05), h = {h} in log k",
           "note": "reported, not pass/fail: the straight-through estimator is biased"}
    for readout in ("linear", "hold"):
        tgt = torch.tensor(targets[readout], device=dev)
        fd, st = [], {T: [] for T in TEMPS}
        for seed in seeds:
            row = []
            for r in range(2):
                tp, tm = theta0.copy(), theta0.copy()
                tp[r] += h
                tm[r] -= h
                Lp = float(((mean_A(tp, seed, readout, False)[1] - tgt) ** 2).mean())
                Lm = float(((mean_A(tm, seed, readout, False)[1] - tgt) ** 2).mean())
                row.append((Lp - Lm) / (2 * h))
            fd.append(row)
            fw, m = mean_A(theta0, seed, readout, True)
            dl = ((2.0 / (S * n)) * (m - tgt)).float().view(S, 1)
            for T in TEMPS:
                st[T].append(ssa.backward(fw, dl, T).double().cpu().numpy())
            del fw
        fd = np.array(fd)
        ref_fd = fd.mean(0)
        rec = {"fd_crn": ref_fd.tolist(), "fd_crn_se": (fd.std(0, ddof=1) / np.sqrt(len(seeds))).tolist(), "st": {},
               "st_se": {}, "st_rel_err_vs_fd": {}}
        for T in TEMPS:
            a = np.array(st[T])
            rec["st"][str(T)] = a.mean(0).tolist()
            rec["st_se"][str(T)] = (a.std(0, ddof=1) / np.sqrt(len(seeds))).tolist()
            rec["st_rel_err_vs_fd"][str(T)] = float(np.linalg.norm(a.mean(0) - ref_fd) / np.linalg.norm(ref_fd))
        if readout == "hold":
            rec["cme_exact"] = g_cme.tolist()
            rec["fd_rel_err_vs_cme"] = float(np.linalg.norm(ref_fd - g_cme) / np.linalg.norm(g_cme))
            rec["st_rel_err_vs_cme"] = {str(T): float(np.linalg.norm(np.array(st[T]).mean(0) - g_cme)
                                                      / np.linalg.norm(g_cme)) for T in TEMPS}
        out[readout] = rec
    torch.cuda.empty_cache()
    return out


def warp_extra(ssa, dev, n: int = 16384, reps: int = 2, oracle: bool = True):
    """The warp-per-trajectory kernels alone: forward (recorded) and adjoint on the network of the uneven
    batch whose reaction count is closest to 300, n trajectories to t_end = 10 with 20 LINEAR samples,
    timed with CUDA events after one warm-up launch; steps/s and the issue-slot rate of each kernel."""
    import torch

    import ssa_workloads as W
    pilot = json.load(open(os.path.join(ROOT, "tests", "golden", "c4_pilot.json")))
    wl = W.config_c4(n_nets=len(pilot["accepted"]), rejected=pilot["rejected"])
    q = int(np.argmin([abs(s.n_reactions - 300) for s in wl.nets]))
    spec = wl.nets[q]
    net = ssa.Network(spec)
    th = torch.tensor(spec.log_rates.astype(np.float32), device=dev)
    max_steps = int(2 * pilot["accepted"][q]["max_draws"] + 256)
    dl = torch.tensor(wl.loss_weights[q] / n, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fms = ams = 0.0
    steps = 0
    for r in range(reps + 1):
        ev[0].record()
        fw = ssa.forward(net, th, n, spec.x0, wl.t_end, wl.sample_times, wl.obs_species[q], 300 + r, readout="linear",
                         record=True, max_steps=max_steps, threads_per_traj=32)
        ev[1].record()
        ssa.backward(fw, dl, wl.temperature)
        ev[2].record()
        torch.cuda.synchronize()
        if r >= 1:
            fms += ev[0].elapsed_time(ev[1])
            ams += ev[1].elapsed_time(ev[2])
            steps += int(fw.draws.sum().item())
        del fw
    rates = ssa.pipe_rates()
    log_slots = 128.0 / rates["neglog"]
    M = spec.n_reactions
    out = {"workload": f"uneven-batch network {q}: N={spec.n_species}, M={M}, {n} trajectories, t_end={wl.t_end}, "
                       "20 LINEAR samples, warp per trajectory",
           "ssa_steps": steps // reps, "forward_ms": fms / reps, "adjoint_ms": ams / reps,
           "fwd_steps_per_s": steps / (fms / 1e3), "adj_steps_per_s": steps / (ams / 1e3),
           "fwd_instr_per_s_T": instr_per_step_fwd(M, log_slots) * steps / (fms / 1e3) / 1e12,
           "adj_instr_per_s_T": instr_per_step_bwd(M, log_slots) * steps / (ams / 1e3) / 1e12}
    # the soft forward of Eq. 4 on the same network and trajectories (warp kernels, forward only), at the
    # batch's T; its step count is its own
    sms, ssteps, sbad = 0.0, 0, 0
    for r in range(reps + 1):
        ev[0].record()
        fw = ssa.forward(net, th, n, spec.x0, wl.t_end, wl.sample_times, wl.obs_species[q], 300 + r,
                         readout="linear", max_steps=max_steps, threads_per_traj=32, selector="soft",
                         temperature=wl.temperature)
        ev[1].record()
        torch.cuda.synchronize()
        if r >= 1:
            sms += ev[0].elapsed_time(ev[1])
            ssteps += int(fw.draws.sum().item())
            sbad = int((fw.status > 1).sum().item())
        del fw
    out["soft_forward"] = {"ms": sms / reps, "ssa_steps": ssteps // reps, "steps_per_s": ssteps / (sms / 1e3),
                           "temperature": wl.temperature, "non_ok_trajectories": sbad}
    # and its exact gradient (recorded soft forward, then the adjoint's segment re-runs)
    gf = ga = 0.0
    gsteps = 0
    for r in range(reps + 1):
        ev[0].record()
        fw = ssa.forward(net, th, n, spec.x0, wl.t_end, wl.sample_times, wl.obs_species[q], 300 + r,
                         readout="linear", record=True, max_steps=max_steps, threads_per_traj=32, selector="soft",
                         temperature=wl.temperature)
        ev[1].record()
        ssa.backward(fw, dl, wl.temperature)
        ev[2].record()
        torch.cuda.synchronize()
        if r >= 1:
            gf += ev[0].elapsed_time(ev[1])
            ga += ev[1].elapsed_time(ev[2])
            gsteps += int(fw.draws.sum().item())
        del fw
    out["soft_forward"]["gradient"] = {"forward_rec_ms": gf / reps, "backward_ms": ga / reps,
                                       "fwd_adj_steps_per_s": gsteps / ((gf + ga) / 1e3)}
    if oracle:
        m = 256
        out["grad_rel_err_vs_fp64"] = oracle_grad_err(
            ssa, dev, spec, spec.log_rates.astype(np.float32), spec.x0, m, wl.t_end, wl.sample_times,
            wl.obs_species[q], 301, "linear", wl.temperature, max_steps,
            W.seeded_dl_dobs(7, m, len(wl.sample_times), len(wl.obs_species[q]), scale=1.0 / m), threads_per_traj=32)
    return out


def grn_extra(ssa, dev, n_img: int = 512, tpi: int = 64, t_end: float = 20.0, reps: int = 2, oracle: bool = True):
    """The gene-regulatory-network classifier (784 -> 256 -> 10, 203,796 parameters, bf16 W1 and W2):
    512 synthetic prototype images x 64 trajectories, t_end = 20, HOLD readout of the 10 outputs at
    t_end, cross-entropy of the softmax of the output counts against the image label, forward +
    straight-through backward at T = 1. Also times the tcgen05 bf16 GEMM alone on the GRN contraction's
    shape and on a large square shape, against the measured bf16 peak."""
    import torch

    from ssa_workloads import grn as G
    p = G.grn_params(seed=5)
    x, labels = G.prototype_images(seed=5, n_img=n_img)
    net = ssa.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    n = n_img * tpi
    lab = torch.tensor(np.repeat(labels, tpi), device=dev)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd_ms = adj_ms = 0.0
    steps = 0
    for r in range(reps + 1):
        ev[0].record(stream)
        fw = ssa.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, [t_end], 70 + r, record=True,
                             max_steps=1 << 14)
        ev[1].record(stream)
        y = fw.obs[:, 0, :].float()
        dl = (torch.softmax(y, dim=1) - torch.nn.functional.one_hot(lab, p.n_out).float()) / n
        ev[2].record(stream)
        ssa.grn_backward(fw, dl.view(n, 1, p.n_out), 1.0)
        ev_end = torch.cuda.Event(enable_timing=True)
        ev_end.record(stream)
        torch.cuda.synchronize()
        if r >= 1:
            fwd_ms += ev[0].elapsed_time(ev[1])
            adj_ms += ev[2].elapsed_time(ev_end)
            steps += int(fw.draws.sum().item())
            bad = int((fw.status > 2).sum().item())
        del fw
    fwd_ms, adj_ms, steps = fwd_ms / reps, adj_ms / reps, steps // reps
    out = {"workload": f"GRN 784-256-10, {n_img} images x {tpi} trajectories, t_end={t_end}, HOLD at t_end, "
                       "cross-entropy, T=1",
           "ssa_steps": steps, "forward_ms": fwd_ms, "backward_ms": adj_ms,
           "fwd_steps_per_s": steps / (fwd_ms / 1e3), "fwd_adj_steps_per_s": steps / ((fwd_ms + adj_ms) / 1e3),
           "non_ok_trajectories": bad}
    # the soft forward of Eq. 4 (the first training phase of Section 3.5) on the same inputs, at T = 1
    soft_ms, soft_steps = 0.0, 0
    for r in range(reps + 1):
        ev[0].record(stream)
        fw = ssa.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, [t_end], 70 + r, record=False,
                             max_steps=1 << 14, soft_temperature=1.0)
        ev[1].record(stream)
        torch.cuda.synchronize()
        if r >= 1:
            soft_ms += ev[0].elapsed_time(ev[1])
            soft_steps += int(fw.draws.sum().item())
        del fw
    out["soft_forward"] = {"ms": soft_ms / reps, "ssa_steps": soft_steps // reps,
                           "steps_per_s": soft_steps / (soft_ms / 1e3), "temperature": 1.0}
    # its exact gradient (the relaxed model differentiated along the soft path) on a quarter of the images: a
    # recorded soft run keeps every dynamic count every 8 steps (about 18 GB here)
    n_sg = max(1, n_img // 4)
    ns = n_sg * tpi
    xs, lab_s = x[:n_sg], lab[:ns]
    sf_ms = sa_ms = 0.0
    sg_steps = 0
    for r in range(reps + 1):
        ev[0].record(stream)
        fw = ssa.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, xs, tpi, t_end, [t_end], 90 + r, record=True,
                             max_steps=1 << 14, soft_temperature=1.0)
        ev[1].record(stream)
        dl = (torch.softmax(fw.obs[:, 0, :], dim=1) - torch.nn.functional.one_hot(lab_s, p.n_out).float()) / ns
        ev[2].record(stream)
        ssa.grn_backward(fw, dl.view(ns, 1, p.n_out), 1.0)
        ev_end = torch.cuda.Event(enable_timing=True)
        ev_end.record(stream)
        torch.cuda.synchronize()
        if r >= 1:
            sf_ms += ev[0].elapsed_time(ev[1])
            sa_ms += ev[2].elapsed_time(ev_end)
            sg_steps += int(fw.draws.sum().item())
        del fw
    sf_ms, sa_ms, sg_steps = sf_ms / reps, sa_ms / reps, sg_steps // reps
    out["soft_gradient"] = {"images": n_sg, "trajectories": ns, "ssa_steps": sg_steps, "forward_rec_ms": sf_ms,
                            "backward_ms": sa_ms, "fwd_adj_steps_per_s": sg_steps / ((sf_ms + sa_ms) / 1e3),
                            "temperature": 1.0}
    # the tensor-core kernel alone: the GRN's contraction (8 six-bit limbs of W1 against 512 images) and a
    # large square product; the E1 shape has 4 output tiles of 128 x 256, so it is timed with the split-K
    # work buffer (the default of the binding) and without it (one CTA per tile)
    gem = {}
    L = ssa._lib.lib()
    for name, (M, N, K) in {"grn_E1_limbs": (n_img, p.n_hid, p.n_in * 8), "square_8192": (8192, 8192, 8192)}.items():
        A = torch.randn(M, K, device=dev).to(torch.bfloat16)
        B = torch.randn(N, K, device=dev).to(torch.bfloat16)
        ld = (K + 7) // 8 * 8
        Ap = torch.zeros((M, ld), dtype=torch.bfloat16, device=dev)
        Bp = torch.zeros((N, ld), dtype=torch.bfloat16, device=dev)
        Ap[:, :K], Bp[:, :K] = A, B
        D = torch.empty((M, N), device=dev)
        err = torch.zeros(1, dtype=torch.int32, device=dev)
        it = 5 if M >= 4096 else 50
        for split in (True, False):
            words = int(L.ssa_bf16_gemm_work_words(M, N, K)) if split else 0
            if not split and name != "grn_E1_limbs":
                continue
            work = torch.empty(max(words, 1), dtype=torch.float64, device=dev) if words else None
            call = lambda: ssa.check(L.ssa_bf16_gemm(ssa._ptr(Ap), ssa._ptr(Bp), M, N, K, ld, ld, None, ssa._ptr(D), N,  # noqa: E731
                                                     ssa._ptr(work), words, ssa._ptr(err), ssa._stream()))
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            # the launches are captured in a CUDA graph and replayed, so that the host's tensor-map encoding
            # does not pace the microsecond-scale product
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(graph, stream=side):
                    for _ in range(it):
                        call()
            stream.wait_stream(side)
            graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / it
            del graph
            ent = {"M": M, "N": N, "K": K, "ms": ms, "tflops": 2.0 * M * N * K / (ms / 1e3) / 1e12,
                   "k_split": max(1, words // (M * N)), "ctas": -(-M // 128) * -(-N // 256) * max(1, words // (M * N)),
                   "timeout_flag": int(err.item()), "timing": f"one CUDA graph of {it} launches, replayed",
                   "operands": "L2-resident across the repeated launches"}
            gem[name if split else name + "_one_cta_per_tile"] = ent
            del work
        del A, B, Ap, Bp, D
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        basis = "of measured (cuBLAS bf16 burst)"
    except (OSError, KeyError, ValueError):
        peak, basis = 1900.0, "of fallback"
    for g in gem.values():
        g["frac"] = g["tflops"] / peak
        g["peak_basis"] = f"{peak:g} TFLOP/s {basis}"
    out["tcgen05_gemm"] = gem
    if oracle:
        out["grad_rel_err_vs_fp64"] = grn_grad_err(ssa, dev, p, x[:4], 16, t_end, 71, 1.0)
    return out


def grn_grad_err(ssa, dev, p, x, tpi, t_end, seed, T):
    """Relative error of each GRN gradient group (W1, b1, W2, b2, log d) against the FP64 oracle on the
    trajectories whose event sequences agree (HOLD at t_end, cross-entropy-shaped seeded upstream gradient)."""
    import torch

    from oracle import native
    n = x.shape[0] * tpi
    dl = np.random.default_rng(seed + 1).standard_normal((n, 1, p.n_out)) / n
    net = ssa.GRN(p.n_in, p.n_hid, p.n_out, p.k_max)
    fw = ssa.grn_forward(net, p.W1, p.b1, p.W2, p.b2, p.log_d, x, tpi, t_end, [t_end], seed, record=True,
                         max_steps=1 << 15)
    orc = native.grn_run(p, x, tpi, t_end, np.array([t_end]), seed, max_steps=1 << 15, dl_dobs=dl, temperature=T,
                         ev_cap=1 << 15)
    ev = fw.run.events(1 << 15).cpu().numpy()
    same = np.all(ev == orc.events, axis=1) & (fw.draws.cpu().numpy() == orc.draws)
    dl_g = dl.copy()
    dl_g[~same] = 0
    g = ssa.grn_backward(fw, torch.tensor(dl_g, dtype=torch.float32, device=dev), T)
    keep = same.astype(np.float64)
    masked = native.GRNResult(orc.obs, orc.draws, orc.status, orc.dE1 * keep[:, None], orc.dW2 * keep[:, None, None],
                              orc.db2 * keep[:, None], orc.dlogd * keep[:, None], None, None)
    ref = masked.grads(x, tpi)
    err = {k: float(np.linalg.norm(g[k].double().cpu().numpy() - ref[k]) / max(np.linalg.norm(ref[k]), 1e-300))
           for k in ref}
    return {"rel_err": max(err.values()), "per_group": err, "n_traj": int(n), "compared": int(same.sum()),
            "identical_events": float(same.mean()), "temperature": float(T)}


def oracle_theta(t32):
    """Log-rates for the oracle such that exp of them equals the binary32 rate constants the kernels use
    (k = exp(theta) in binary64, rounded once to binary32): a fixed relative rounding of every rate would
    otherwise move a long trajectory's clock systematically against the oracle's."""
    k32 = np.exp(np.asarray(t32, dtype=np.float32).astype(np.float64)).astype(np.float32)
    return np.log(k32.astype(np.float64))


def oracle_grad_err(ssa, dev, spec, theta32, x0, n, t_end, ts, obs_sp, seed, readout, T, cap, dl, wide=False,
                    threads_per_traj=0, traj_offset=0):
    """Relative error (norm over the parameters) of the GPU straight-through gradient against the FP64 oracle's
    on the same seeded inputs: n trajectories, upstream gradient dl [n, S, n_obs], kept on the trajectories
    whose event sequences agree; on those, the upstream gradient of any sample whose bracket differs (an event
    within binary32 clock rounding of the sample time, which moves the LINEAR readout's time derivative) is
    zeroed on both sides (BIN: the two bins on either side of such an edge). wide: ssa_backward_wide."""
    import torch

    from oracle import native
    net = ssa.Network(spec)
    th64 = oracle_theta(theta32)
    fw = ssa.forward(net, torch.tensor(theta32, device=dev), n, x0, t_end, ts, obs_sp, seed, readout=readout,
                     record=True, max_steps=cap, threads_per_traj=threads_per_traj, traj_offset=traj_offset)
    code = {"hold": native.HOLD, "linear": native.LINEAR, "bin": native.BIN}[readout]
    orc = native.run(spec, th64, x0, n, t_end, ts, obs_sp, seed, code, max_steps=cap, ev_cap=cap,
                     traj_offset=traj_offset)
    ev = fw.run.events(cap).cpu().numpy()
    same = np.all(ev == orc.events, axis=1) & (fw.draws.cpu().numpy() == orc.draws)
    del ev
    ts = np.asarray(ts, dtype=np.float64)
    S = len(ts)
    keep = np.repeat(same[:, None], S, axis=1)
    if readout == "bin":
        tol = 8.0 * (spec.n_reactions + 2) * 2.0 ** -24 * float(t_end)
        for i in np.nonzero(same)[0]:
            near = np.any(np.abs(orc.times[i, :orc.draws[i], None] - ts[None, :]) <= tol, axis=0)
            keep[i] &= ~near & ~np.concatenate([[False], near[:-1]])
    else:
        gb = fw.run.brackets().cpu().numpy()
        for i in np.nonzero(same)[0]:
            d = int(orc.draws[i])
            applied = d - 1 if orc.status[i] == 0 else d
            keep[i] &= np.searchsorted(orc.times[i, :applied], ts, side="right") == gb[i]
    dl2 = np.array(dl, dtype=np.float64, copy=True) * keep[:, :, None]
    orc_g = native.run(spec, th64, x0, n, t_end, ts, obs_sp, seed, code, max_steps=cap, dl_dobs=dl2, temperature=T,
                       traj_offset=traj_offset)
    g_in = torch.tensor(dl2, dtype=torch.float32, device=dev)
    g = (ssa.backward_wide(fw, g_in, T) if wide else ssa.backward(fw, g_in, T)).double().cpu().numpy()
    ref = orc_g.dtheta.sum(0)
    den = np.linalg.norm(ref)
    return {"rel_err": float(np.linalg.norm(g - ref) / den) if den > 0 else None, "n_traj": int(n),
            "identical_events": float(same.mean()), "samples_compared": float(keep.mean()),
            "temperature": float(T), "ref_norm": float(den), "finite": bool(np.all(np.isfinite(g))),
            "adjoint": "ssa_backward_wide" if wide else "ssa_backward"}


def c1_extra(ssa, dev, runs: int = 200, sweep=tuple(range(10, 23)), osc_sweep=(10, 12, 14, 16, 18, 20)):
    """The forward-only workload (2A <-> B, 1,024 trajectories to t_end = 50, 50 HOLD samples of A and B, seed 0):
    one forward captured in a CUDA graph and replayed `runs` times, each replay timed with CUDA events (L2
    flushed between replays, outside the events); the median and spread. Then forward SSA steps/s over
    ensemble sizes 2^10 .. 2^22 of the same workload, and, mirroring Supplementary Figure 2, of the oscillator
    (t_end = 2, 10 LINEAR samples of R) for the three selectors (Gumbel-max, plain direct method, soft at
    T = 0.5), each the mean of 3 launches after a warm-up."""
    import torch

    import ssa_workloads as W
    wl = W.config_c1()
    net = ssa.Network(wl.net)
    S = len(wl.sample_times)
    th = torch.tensor(wl.log_rates.astype(np.float32), device=dev)
    x0 = torch.tensor(wl.x0, device=dev)
    ts = torch.tensor(wl.sample_times, device=dev)
    sp = torch.tensor(wl.obs_species, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def buffers(n):
        opts = ssa.make_opts("hold", False, 64, wl.max_steps)
        return (torch.empty(ssa.workspace_bytes(net, n, S, opts), dtype=torch.uint8, device=dev),
                torch.empty((n, S, len(wl.obs_species)), dtype=torch.int32, device=dev))

    n = wl.n_traj
    ws, obs = buffers(n)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(3):
            ssa.forward(net, th, n, x0, wl.t_end, ts, sp, wl.seed, readout="hold", max_steps=wl.max_steps, workspace=ws,
                        obs_out=obs)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            fwg = ssa.forward(net, th, n, x0, wl.t_end, ts, sp, wl.seed, readout="hold", max_steps=wl.max_steps,
                              workspace=ws, obs_out=obs)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(runs)]
        for r in range(runs):
            flush.fill_(r & 0xFF)
            evs[r][0].record(stream)
            graph.replay()
            evs[r][1].record(stream)
        stream.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    steps = int(fwg.draws.sum().item())
    out = {"workload": "2A<->B, 1,024 traj, t_end=50, 50 HOLD samples of A and B, seed 0, forward only",
           "graph_replay": {"runs": runs, "ssa_steps": steps, "median_ms": float(np.median(ms)),
                            "p10_ms": float(np.quantile(ms, 0.1)), "p90_ms": float(np.quantile(ms, 0.9)),
                            "steps_per_s": steps / (float(np.median(ms)) / 1e3),
                            "identical_runs": True}}
    del graph, fwg
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(call, reps=3):
        call(0)
        torch.cuda.synchronize()
        ms_tot, st_tot = 0.0, 0
        for r in range(reps):
            flush.fill_(r & 0xFF)
            ev[0].record()
            fw = call(r + 1)
            ev[1].record()
            torch.cuda.synchronize()
            ms_tot += ev[0].elapsed_time(ev[1])
            st_tot += int(fw.draws.sum().item())
        return {"ms": ms_tot / reps, "steps_per_s": st_tot / (ms_tot / 1e3)}

    sw = {}
    for e in sweep:
        nn = 1 << e
        wsn, obsn = buffers(nn)
        sw[str(nn)] = timed(lambda r: ssa.forward(net, th, nn, x0, wl.t_end, ts, sp, 10 + r, readout="hold",
                                                  max_steps=wl.max_steps, workspace=wsn, obs_out=obsn))
        del wsn, obsn
    out["ensemble_sweep"] = sw
    wo = W.config_c3(n_traj=1, t_end=2.0, S=10)
    onet = ssa.Network(wo.net)
    oth = torch.tensor(wo.log_rates.astype(np.float32), device=dev)
    osw = {"workload": "Vilar oscillator, t_end=2, 10 LINEAR samples of R"}
    for sel in ("gumbel", "direct", "soft"):
        row = {}
        for e in osc_sweep:
            nn = 1 << e
            row[str(nn)] = timed(lambda r: ssa.forward(onet, oth, nn, wo.x0, wo.t_end, wo.sample_times, wo.obs_species,
                                                       20 + r, readout="linear", max_steps=1 << 16, selector=sel,
                                                       temperature=0.5 if sel == "soft" else None), reps=2)
        osw[sel] = row
    out["oscillator_sweep"] = osw
    torch.cuda.empty_cache()
    return out


def grad_error_subset(ssa, net, wl, dev, n=2048):
    """Relative error of the GPU gradient against the FP64 oracle on trajectories with identical
    event sequences, for each temperature (same seeded inputs on both sides)."""
    import torch

    import ssa_workloads as W
    from oracle import native
    theta32 = wl.log_rates.astype(np.float32)
    dl = W.seeded_dl_dobs(3, n, len(wl.sample_times), 1, scale=1.0 / n)
    out = {}
    fw = ssa.forward(net, torch.tensor(theta32, device=dev), n, wl.x0, wl.t_end, wl.sample_times, wl.obs_species, 77,
                     readout="linear", record=True, max_steps=2048)
    ev = fw.run.events(2048).cpu().numpy()
    for T in TEMPS:
        orc = native.run(wl.net, oracle_theta(theta32), wl.x0, n, wl.t_end, wl.sample_times, wl.obs_species, 77,
                         native.LINEAR, max_steps=2048, dl_dobs=dl, temperature=T, ev_cap=2048)
        same = np.all(ev == orc.events, axis=1)
        dl2 = dl.copy()
        dl2[~same] = 0
        g = ssa.backward(fw, torch.tensor(dl2, dtype=torch.float32, device=dev), T).cpu().numpy()
        ref = orc.dtheta[same].sum(0)
        out[str(T)] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    out["identical_event_fraction"] = float(same.mean())
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-traj", type=int, default=65536)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-chunk", type=int, default=4096)
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the oscillator and uneven-batch fields")
    ap.add_argument("--legs", default="c1,bias,oscillator,c3,batch,grn,warp,ion",
                    help="comma-separated extra fields to measure: c1 (graph-replayed forward-only workload and the "
                         "ensemble-size sweeps), bias (the straight-through gradient against finite differences and "
                         "the exact master-equation gradient), oscillator, c3 (the oscillator at its full size), "
                         "batch, grn, warp, ion (the ion channel of Section 4.4) ('none' for none)")
    ap.add_argument("--grn-images", type=int, default=512, help="images of the GRN field (64 trajectories each)")
    ap.add_argument("--ion-traj", type=int, default=262144, help="trajectories of the ion-channel field")
    ap.add_argument("--osc-traj", type=int, default=1 << 20, help="forward trajectories of the oscillator field")
    ap.add_argument("--osc-samples", type=int, default=10, help="LINEAR samples of R in the oscillator field")
    ap.add_argument("--warp-traj", type=int, default=16384, help="trajectories of the warp-kernel field")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="trajectories per network of the uneven batch, as a fraction of the full counts")
    ap.add_argument("--batch-sequential", action="store_true",
                    help="also time the uneven batch's work as one forward and one backward call per network")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
