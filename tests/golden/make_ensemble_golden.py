"""Writes tests/golden/ensemble_samples.json: FP64 oracle runs of four boxes
sampled from the 64-box ensemble (numpy default_rng(0) draws, drive period
2000 steps), one of each size class, over one drive period, for the GPU test
that steps the whole ensemble as one batch and compares these four boxes.

Per sampled box it stores x_cm of every swimmer (mean of its three bead
centres, Sec. 3, Eq. vel_swim) every 100 steps, and after the last step the
velocity u (Sec. 2.1, with the Guo half-force term) at 2048 cells drawn with
default_rng(7) plus the 512 cells of largest |u|, the L2 norm of u over the
box and the first eight node positions.  Every value comes from oracle/ (and
the input generators in workloads/).

Usage: python tests/golden/make_ensemble_golden.py [--steps N]
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
from workloads import assemble, ensemble_boxes  # noqa: E402

N_RANDOM, N_LARGEST, SEED = 2048, 512, 7
EVERY = 100
# the first box of each size class in the seed-0 ensemble: 192x128x128 and
# 96^3, 64^3 with two swimmers each, 48^3 with one
SAMPLED = (0, 1, 2, 15)


def u_sample(u):
    rng = np.random.default_rng(SEED)
    rand = rng.choice(u.shape[0], size=N_RANDOM, replace=False)
    mag = np.linalg.norm(u, axis=1)
    largest = np.argsort(mag, kind="stable")[-N_LARGEST:]
    cells = np.unique(np.concatenate([rand, largest]))
    return {"cells": cells.tolist(), "u": u[cells].tolist(), "u_l2_norm": float(np.linalg.norm(u))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    a = ap.parse_args()
    boxes = ensemble_boxes()
    oracle.set_threads(0)
    out = {"ensemble": "ensemble_boxes(n=64, seed=0, period=2000.0)", "steps": a.steps, "every": EVERY,
           "boxes": {}, "made_by": "tests/golden/make_ensemble_golden.py (FP64 oracle)"}
    for k in SAMPLED:
        box = boxes[k]
        sim = oracle.OracleSim(box, assemble(box))
        traj = [[0, sim.swimmer_centres().tolist()]]
        t0 = time.time()
        while sim.t < a.steps:
            sim.step(min(EVERY, a.steps - sim.t))
            traj.append([sim.t, sim.swimmer_centres().tolist()])
            print(f"box {k} {tuple(box.dims)}: step {sim.t} / {a.steps}, {time.time() - t0:.0f} s", flush=True)
        _, u = oracle.macros(sim.f)
        out["boxes"][str(k)] = {"dims": list(box.dims), "n_swimmers": len(box.swimmers), "x_cm": traj,
                                "u_sample": u_sample(u), "nodes_final_first8": sim.r[:8].tolist()}
    path = os.path.join(HERE, "ensemble_samples.json")
    with open(path + ".tmp", "w") as fh:
        json.dump(out, fh)
    os.replace(path + ".tmp", path)
    print("wrote", path)


if __name__ == "__main__":
    main()
