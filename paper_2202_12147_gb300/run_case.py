"""Run one synthetic swimmer box for a number of coupled steps and print the
swimmers' displacement (a command-line runner, also used to drive profilers
on a single box).

    python -m paper_2202_12147_gb300.run_case --case pair_side_3 --steps 4 --storage f32
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _box(name):
    from workloads import adjoint_single_96, pair_side_256cube, single_swimmer_48, swimmer_pair
    if name == "single_48":
        return single_swimmer_48()
    if name.startswith("ensemble_"):  # one box of the 64-box ensemble, by index
        from workloads import ensemble_boxes
        return ensemble_boxes(64, seed=0)[int(name.split("_")[1])]
    if name == "pair_side_256cube":
        return pair_side_256cube()
    if name == "single_96":
        return adjoint_single_96()
    arr, gap = name.split("_")[1], int(name.split("_")[2])
    return swimmer_pair(arr, gap)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="pair_side_3",
                    help="single_48 | single_96 | pair_side_256cube | pair_{inline,side}_{3,5,8} (256x128x128) | ensemble")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--deterministic", action="store_true")
    ap.add_argument("--kernel-by-kernel", action="store_true",
                    help="launch kernels one by one instead of replaying CUDA graphs")
    ap.add_argument("--adjoint", action="store_true",
                    help="run the adjoint engine: forward and backward sweeps over --steps steps, "
                         "gradient of swimmer 0's x displacement w.r.t. its drive")
    ap.add_argument("--K", type=int, default=100, help="adjoint checkpoint interval")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"], help="adjoint fluid precision")
    ap.add_argument("--batch", type=int, default=0, help="advance this many copies of the box as one batch")
    a = ap.parse_args(argv)
    from paper_2202_12147_gb300 import Batch, Simulation
    from workloads import assemble, ensemble_boxes
    if a.case == "ensemble":
        boxes = ensemble_boxes(64, seed=0)
        sims = [Simulation(b.dims, assemble(b), tau=b.tau, rho0=b.rho0, storage=a.storage,
                           deterministic=a.deterministic) for b in boxes]
        batch = Batch(sims)
        if a.kernel_by_kernel:
            batch.profile(True)
        batch.lb_step(a.steps)
        st = sims[0].swimmer_state(0)
        print(f"ensemble of {len(sims)} boxes: step {st['step']}, box 0 swimmer 0 displacement {st['disp'].tolist()}")
        batch.close()
        for s in sims:
            s.close()
        return
    box = _box(a.case)
    if a.adjoint:
        import numpy as np
        from paper_2202_12147_gb300 import Adjoint
        eng = Adjoint(box.dims, assemble(box), n_steps=a.steps, K=a.K, precision=a.precision, tau=box.tau,
                      rho0=box.rho0, g=box.g)
        d = eng.forward()
        seed = np.zeros((eng.n_swimmers, 3))
        seed[0, 0] = 1.0
        g = eng.backward(seed)
        print(f"{box.name}: displacement {d[0].tolist()}, gradient (A1 A2 A3 phi1 phi2 phi3) {g[0].tolist()}, "
              f"timing {eng.timing()}")
        eng.close()
        return
    if a.batch > 0:
        asm = assemble(box)
        sims = [Simulation(box.dims, asm, tau=box.tau, rho0=box.rho0, storage=a.storage,
                           deterministic=a.deterministic, forcing=box.forcing, kernel=box.kernel) for _ in range(a.batch)]
        batch = Batch(sims)
        if a.kernel_by_kernel:
            batch.profile(True)
        batch.lb_step(a.steps)
        st = sims[0].swimmer_state(0) if sims[0].n_swimmers else None
        print(f"batch of {a.batch} x {box.name}: step {a.steps}" + (f", box 0 swimmer 0 displacement {st['disp'].tolist()}" if st else ""))
        batch.close()
        for s in sims:
            s.close()
        return
    sim = Simulation(box.dims, assemble(box), tau=box.tau, rho0=box.rho0, storage=a.storage,
                     deterministic=a.deterministic, forcing=box.forcing, kernel=box.kernel)
    if a.kernel_by_kernel:
        sim.profile(True)
    sim.lb_step(a.steps)
    for k in range(sim.n_swimmers):
        st = sim.swimmer_state(k)
        print(f"{box.name} swimmer {k}: step {st['step']} displacement {st['disp'].tolist()}")
    sim.close()


if __name__ == "__main__":
    main()
