"""The paper's swimmer study at its own scale on one GPU (Sec. 3): the
1024 x 256 x 256 box with a lone swimmer, two in-line swimmers and two
side-by-side swimmers (workloads.paper_study_box), advanced for whole drive
periods; every swimmer's centre of mass x_cm is recorded at each period
boundary and the swimming velocity of every period is (x_cm(kT) - x_cm((k-1)T)) / T
(Sec. 3, Eq. vel_swim).

    python -m paper_2202_12147_gb300.paper_runs --case inline_2 --periods 12 --out result.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(case, periods, storage="f32", deterministic=False, tau=1.0):
    import numpy as np
    import torch
    from paper_2202_12147_gb300 import Simulation
    from workloads import assemble, paper_study_box
    box = paper_study_box(case, tau=tau)
    T = int(box.swimmers[0].period)
    sim = Simulation(box.dims, assemble(box), tau=box.tau, rho0=box.rho0, storage=storage, forcing=box.forcing,
                     kernel=box.kernel, deterministic=deterministic)
    S = sim.n_swimmers
    xs = [[sim.swimmer_state(s)["x_cm"].tolist() for s in range(S)]]
    t0 = time.perf_counter()
    for _ in range(periods):
        sim.lb_step(T)
        xs.append([sim.swimmer_state(s)["x_cm"].tolist() for s in range(S)])  # synchronises; latched errors raise
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = [sim.swimmer_state(s) for s in range(S)]
    sim.close()
    x = np.array(xs)
    v = (x[1:, :, 0] - x[:-1, :, 0]) / T
    return {"case": case, "dims": list(box.dims), "tau": box.tau, "storage": storage, "forcing": box.forcing,
            "delta_kernel": box.kernel, "period": T, "periods": periods,
            "swimmer_centres": [list(s.center) for s in box.swimmers], "x_cm": xs,
            "v_period_x": v.tolist(), "re_swim": [s["re_swim"] for s in st], "re_bead": [s["re_bead"] for s in st],
            "wall_s": wall, "mlups": box.n_cells * periods * T / wall / 1e6}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", action="append", required=True,
                    help="lone | inline_<n> | side_<n> (n swimmer lengths between the centres); repeatable")
    ap.add_argument("--periods", type=int, default=12)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--tau", type=float, default=1.0, help="relaxation time (viscosity (tau - 1/2) / 3)")
    ap.add_argument("--out", required=True, help="JSON file (one object per case, appended as lines)")
    a = ap.parse_args(argv)
    for c in a.case:
        r = run(c, a.periods, a.storage, tau=a.tau)
        with open(a.out, "a") as fh:
            fh.write(json.dumps(r) + "\n")
        print(f"{c}: last-period velocity {r['v_period_x'][-1]}, {r['wall_s']:.0f} s, {r['mlups']:.0f} MLUPS",
              flush=True)


if __name__ == "__main__":
    main()
