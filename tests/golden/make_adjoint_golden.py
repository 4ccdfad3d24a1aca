"""Write the stored expected values of the drive-parameter gradient of a
swimmer's net displacement over one period, computed by the FP64 oracle only.

    python tests/golden/make_adjoint_golden.py [--out tests/golden/adjoint_single_96.json]

Workload: one swimmer (beads of radius 6 at icosphere subdivision 3, spacing
18, k = 0.005, Gs = 0.01) in a periodic 96^3 box, tau = 1, rho0 = 1, drive
period 1000 steps, run for one period from rest.  The drive is written with
independent per-bead amplitudes and phases theta = (A1, A2, A3, phi1, phi2,
phi3) at the base point that reproduces the paper's balanced protocol
(Sec. 2.2, driving-force equation) with A = B = 1e-3, alpha = pi/2.

Objective: D = x_cm(T) - x_cm(0), x_cm the mean of the three bead centres
(Sec. 3, Eq. vel_swim).  Stored: D, and dD/dtheta for theta in (A1, A2, A3,
phi2, phi3) by
  * the oracle's exact discrete derivative (complex step, h = 1e-30), and
  * central finite differences with h = 1e-6 |theta_p|.
Takes about an hour on eight cores.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from workloads import adjoint_single_96, assemble  # noqa: E402

PARAMS = [(0, 0), (0, 1), (0, 2), (0, 4), (0, 5)]
NAMES = ["A1", "A2", "A3", "phi2", "phi3"]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "adjoint_single_96.json"))
    ap.add_argument("--steps", type=int, default=1000)
    a = ap.parse_args(argv)
    box = adjoint_single_96()
    asm = assemble(box)
    theta = oracle.drive_parameters(asm)
    t0 = time.time()
    D = oracle.displacement(box, a.steps, asm=asm)
    print(f"D = {D[0].tolist()}  ({time.time() - t0:.0f} s)", flush=True)
    cs, fd = [], []
    for p, name in zip(PARAMS, NAMES):
        t0 = time.time()
        cs.append(oracle.displacement_jacobian_cs(box, a.steps, [p], asm=asm)[0, 0])
        t1 = time.time()
        fd.append(oracle.displacement_jacobian_fd(box, a.steps, [p], asm=asm, rel_h=1e-6)[0, 0])
        print(f"{name}: complex step {cs[-1][0]:.12e} ({t1 - t0:.0f} s), "
              f"finite difference {fd[-1][0]:.12e} ({time.time() - t1:.0f} s)", flush=True)
    out = dict(
        workload="one swimmer, beads radius 6 (icosphere subdivision 3, 642 nodes), spacing 18, k 0.005, "
                 "Gs 0.01, periodic 96^3, tau 1, rho0 1, drive period 1000, one period from rest",
        steps=a.steps,
        theta=theta[0].tolist(),
        theta_names=["A1", "A2", "A3", "phi1", "phi2", "phi3"],
        params=NAMES,
        displacement=D[0].tolist(),
        grad_complex_step=[v.tolist() for v in cs],
        grad_finite_difference=[v.tolist() for v in fd],
        finite_difference_rel_h=1e-6,
        complex_step_h=1e-30,
        generator="tests/golden/make_adjoint_golden.py (FP64 oracle only)",
    )
    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()
