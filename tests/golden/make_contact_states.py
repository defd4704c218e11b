"""Writes the contact-rich starting states of the full-size contact parity
tests, computed by the CPU oracle alone (no GPU code is involved):

* coil500_state.npz: the 500-node coil of the coil workload (radius 2 cm,
  pitch 2.2 h, h = 1 mm, clamped lower end, dt = 0.25 ms, line search)
  after it has collapsed under gravity until its turns touch;
* gripper5x60_state.npz: the five 60-node gripper fingers (Sec. IV's
  active entanglement gripper, reading C30) after 0.4 s of their natural
  curvature ramp, touching one another.

Each file holds q, qdot (per-rod layout of Eq. 1), the reference directors
d1 and reference twists beta, the step index, and the number of edge pairs
in contact at the stored state.  Run from the repository root:
    python tests/golden/make_contact_states.py [coil|gripper ...]
(about 15 minutes for the coil, 1 for the gripper, on one CPU core)."""
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import OracleSystems  # noqa: E402
from oracle.contact import segment_distance  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def pairs_in_contact(ora):
    """Edge pairs of each system closer than C + delta at its state."""
    n = 0
    for s in ora.systems:
        cand = s.pair_cand
        if len(cand) == 0:
            continue
        nd = torch.as_tensor(s.node_dof)
        nl = torch.as_tensor(s.edge_nl)
        i, j = torch.as_tensor(cand[:, 0]), torch.as_tensor(cand[:, 1])
        idx = torch.stack([nd[nl[i, 0]], nd[nl[i, 1]], nd[nl[j, 0]], nd[nl[j, 1]]], 1)
        x = s.q[(idx[:, :, None] + torch.arange(3)).reshape(-1, 12)]
        D, _, _ = segment_distance(x[:, 0:3], x[:, 3:6], x[:, 6:9], x[:, 9:12])
        C = torch.as_tensor(s.h_edge[cand[:, 0]] + s.h_edge[cand[:, 1]])
        n += int((D < C + ora.p["delta"]).sum())
    return n


def run(name, ora, steps, controls, min_pairs):
    t0 = time.time()
    for k in range(steps):
        if controls is not None:
            controls(ora, k)
        st = ora.step(1)
        assert all(x[0] == 0 for x in st), (k, st)
        if k % 25 == 24:
            n = pairs_in_contact(ora)
            print("%s step %d: %d pairs in contact (%.0f s)" % (name, k + 1, n, time.time() - t0),
                  flush=True)
    n = pairs_in_contact(ora)
    assert n >= min_pairs, n
    q, v = ora.get_state()
    d1, beta = ora.get_frames()
    np.savez_compressed(os.path.join(HERE, name + "_state.npz"), q=q, qdot=v, d1=d1,
                        beta=beta, step=steps, pairs=n)
    print("%s: wrote the state after %d steps, %d pairs in contact" % (name, steps, n))


def coil():
    desc, params, _ = workloads.coil(N=500)
    run("coil500", OracleSystems(desc, params), 400, None, 100)


def gripper():
    desc, params, kfn = workloads.gripper()
    dt = params["dt"]
    ora = OracleSystems(desc, params)
    R = len(desc["nodes_per_rod"])
    run("gripper5x60", ora, 400, lambda o, k: o.set_natural_curvature(0, R, kfn(k * dt)), 5)


if __name__ == "__main__":
    which = sys.argv[1:] or ["gripper", "coil"]
    for w in which:
        {"coil": coil, "gripper": gripper}[w]()
