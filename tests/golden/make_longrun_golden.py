"""Writes tests/golden/longrun_<case>.json: long runs of the FP64 oracle on the
full-size two-swimmer boxes (Sec. 3 set-ups at the sizes of the benchmark
workloads), for the GPU tests to compare against after the same number of
steps.

Per case it stores
* x_cm of every swimmer (mean of its three bead centres, Sec. 3, Eq.
  vel_swim) every `every` steps, period boundaries included;
* the velocity u (Sec. 2.1, with the Guo half-force term) after the last
  step at 2048 cells drawn with numpy's default_rng(seed) plus the 512 cells
  of largest |u| (the near field of the beads), and the L2 norm of u over
  the whole box.

Every value comes from oracle/ (and the input generators in workloads/).
Usage: python tests/golden/make_longrun_golden.py <case> [<case> ...]
Cases: side3_256x128x128 (3 drive periods), side3_256cube (1 period),
inline3/inline5/inline8/side5/side8_256x128x128 (1 period).
"""
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


def _case(name):
    """(box, periods) of a case."""
    if name == "side3_256cube":
        return pair_side_256cube(), 1
    arr, gap = name.split("_")[0][:-1], int(name.split("_")[0][-1])
    periods = 3 if name == "side3_256x128x128" else 1
    return swimmer_pair({"side": "side", "inline": "inline"}[arr], gap), periods


def run(name):
    box, periods = _case(name)
    asm = assemble(box)
    T = int(box.swimmers[0].period)
    steps = periods * T
    every = 100
    oracle.set_threads(0)
    sim = oracle.OracleSim(box, asm)
    traj = [[0, sim.swimmer_centres().tolist()]]
    t0 = time.time()
    for k in range(steps // every):
        sim.step(every)
        traj.append([(k + 1) * every, sim.swimmer_centres().tolist()])
        print(f"{name}: step {(k + 1) * every} / {steps}, {time.time() - t0:.0f} s", flush=True)
    _, u = oracle.macros(sim.f)
    rng = np.random.default_rng(SEED)
    rand = rng.choice(box.n_cells, size=N_RANDOM, replace=False)
    mag = np.linalg.norm(u, axis=1)
    largest = np.argsort(mag, kind="stable")[-N_LARGEST:]
    cells = np.unique(np.concatenate([rand, largest]))
    out = {
        "case": name, "dims": list(box.dims), "tau": box.tau, "period": T, "steps": steps, "every": every,
        "x_cm": traj, "cells": cells.tolist(), "u": u[cells].tolist(),
        "u_l2_norm": float(np.linalg.norm(u)), "nodes_final_first8": sim.r[:8].tolist(),
        "made_by": "tests/golden/make_longrun_golden.py (FP64 oracle)",
    }
    with open(os.path.join(HERE, f"longrun_{name}.json"), "w") as fh:
        json.dump(out, fh)
    print(f"{name}: done in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    for n in sys.argv[1:]:
        run(n)
