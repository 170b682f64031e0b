"""Oracle pilot of the uneven-batch workload (random networks, t_end = 10): writes c4_pilot.json.

For each network drawn from the seeded generator stream, 64 trajectories are simulated by the FP64
oracle (forward only, no samples). A draw is rejected -- and the next draw of the same stream takes
its place -- when the mean number of reaction draws per trajectory exceeds 1e6 or a trajectory ends
in any status other than OK or ABSORBED (step cap, overflow, bad rate). The accepted networks' mean
and maximum draw counts size the event logs (max_steps) of the GPU runs.

    python tests/golden/make_c4_pilot.py [--n-nets 256]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ssa_workloads as W  # noqa: E402
from ssa_workloads.configs import HOLD  # noqa: E402
from oracle import native  # noqa: E402

PILOT_TRAJ = 64
MEAN_CAP = 1_000_000
CHUNK = 16


def pilot(net):
    th = net.log_rates.astype(np.float32).astype(np.float64)
    draws = []
    for c in range(0, PILOT_TRAJ, CHUNK):
        o = native.run(net, th, net.x0, CHUNK, 10.0, np.zeros(0), np.array([0], np.int32), 0, HOLD,
                       max_steps=2 * MEAN_CAP, traj_offset=c)
        if np.any(o.status > 1):
            return None
        draws.extend(o.draws.tolist())
        if sum(draws) > MEAN_CAP * PILOT_TRAJ:
            return None
    return np.array(draws)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-nets", type=int, default=256)
    args = ap.parse_args()
    rng = np.random.default_rng(3)  # the generator stream of ssa_workloads.config_c4
    accepted, rejected, d = [], [], 0
    while len(accepted) < args.n_nets:
        net = W.random_network(rng, n_species_range=(2, 64), n_reactions_range=(4, 512))
        r = pilot(net)
        if r is None:
            rejected.append(d)
        else:
            accepted.append({"draw": d, "N": net.n_species, "M": net.n_reactions, "mean_draws": float(r.mean()),
                             "max_draws": int(r.max())})
        d += 1
        print(d, len(accepted), len(rejected), flush=True)
    out = {"pilot_traj": PILOT_TRAJ, "mean_cap": MEAN_CAP, "t_end": 10.0, "seed": 3, "rejected": rejected,
           "accepted": accepted}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_pilot.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
