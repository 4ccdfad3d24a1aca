"""Writes tests/golden/longrun_<case>.json: long runs of the FP64 oracle on the
full-size two-swimmer boxes (Sec. 3 set-ups at the sizes of the benchmark
workloads), for the GPU tests to compare against after the same number of
steps.

Per case it stores
* x_cm of every swimmer (mean of its three bead centres, Sec. 3, Eq.
  vel_swim) every `every` steps, period boundaries included;
* at the end of drive period 1, and at the last period boundary reached, the
  velocity u (Sec. 2.1, with the Guo half-force term) at 2048 cells drawn
  with numpy's default_rng(seed) plus the 512 cells of largest |u| (the near
  field of the beads), and the L2 norm of u over the whole box.

The file is rewritten at every period boundary, so a run that is stopped
keeps the periods it finished ("steps" says how many steps the file holds).
With --state DIR the oracle's state (populations, node positions, step) is
saved there at every period boundary and a later call continues the run from
it (the oracle is deterministic, so a continued run equals an uninterrupted
one).  Every value comes from oracle/ (and the input generators in
workloads/).

Usage: python tests/golden/make_longrun_golden.py [--periods P] [--state DIR] <case> [<case> ...]
Cases: {inline,side}{3,5,8}_256x128x128 (the six pairs of the 256 x 128 x 128
box), side3_256cube (the 256^3 pair).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import assemble, pair_side_256cube, swimmer_pair  # noqa: E402

N_RANDOM, N_LARGEST, SEED = 2048, 512, 7
EVERY = 100


def case_box(name):
    """The BoxSpec of a case name."""
    if name == "side3_256cube":
        return pair_side_256cube()
    head, dims = name.split("_")
    if dims != "256x128x128":
        raise ValueError(name)
    arr, gap = head[:-1], int(head[-1])
    return swimmer_pair({"side": "side", "inline": "inline"}[arr], gap)


def u_sample(u):
    """The stored sample of a velocity field: fixed random cells plus the
    cells of largest |u|, and the L2 norm over all cells."""
    rng = np.random.default_rng(SEED)
    rand = rng.choice(u.shape[0], size=N_RANDOM, replace=False)
    mag = np.linalg.norm(u, axis=1)
    largest = np.argsort(mag, kind="stable")[-N_LARGEST:]
    cells = np.unique(np.concatenate([rand, largest]))
    return {"cells": cells.tolist(), "u": u[cells].tolist(), "u_l2_norm": float(np.linalg.norm(u))}


def run(name, periods, state_dir):
    box = case_box(name)
    asm = assemble(box)
    T = int(box.swimmers[0].period)
    oracle.set_threads(0)
    sim = oracle.OracleSim(box, asm)
    path = os.path.join(HERE, f"longrun_{name}.json")
    traj = [[0, sim.swimmer_centres().tolist()]]
    samples = {}
    st_file = os.path.join(state_dir, f"longrun_{name}.npz") if state_dir else None
    if st_file and os.path.exists(st_file):
        with np.load(st_file) as z:
            sim.f = z["f"].copy()
            sim.r = z["r"].copy()
            sim.t = int(z["t"])
        with open(path) as fh:
            old = json.load(fh)
        if old["steps"] != sim.t:
            raise RuntimeError(f"{path} holds {old['steps']} steps, the saved state {sim.t}")
        traj, samples = old["x_cm"], old["u_samples"]
        print(f"{name}: continuing from step {sim.t}", flush=True)
    t0 = time.time()
    while sim.t < periods * T:
        sim.step(EVERY)
        traj.append([sim.t, sim.swimmer_centres().tolist()])
        print(f"{name}: step {sim.t} / {periods * T}, {time.time() - t0:.0f} s", flush=True)
        if sim.t % T:
            continue
        _, u = oracle.macros(sim.f)
        # keep period 1 (the stated step count of the field error) and the latest period
        samples = {k: v for k, v in samples.items() if int(k) == T}
        samples[str(sim.t)] = u_sample(u)
        out = {
            "case": name, "dims": list(box.dims), "tau": box.tau, "period": T, "steps": sim.t, "every": EVERY,
            "x_cm": traj, "u_samples": samples, "nodes_final_first8": sim.r[:8].tolist(),
            "made_by": "tests/golden/make_longrun_golden.py (FP64 oracle)",
        }
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(out, fh)
        os.replace(tmp, path)
        if st_file:
            os.makedirs(state_dir, exist_ok=True)
            np.savez(st_file + ".tmp.npz", f=sim.f, r=sim.r, t=sim.t)
            os.replace(st_file + ".tmp.npz", st_file)
        print(f"{name}: period {sim.t // T} written, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--periods", type=int, default=1)
    ap.add_argument("--state", default="")
    ap.add_argument("cases", nargs="+")
    a = ap.parse_args()
    for n in a.cases:
        run(n, a.periods, a.state)
