"""Analytic comparator of the swimmer velocities: three-bead swimmers with
hydrodynamic interactions between point-like beads (Sec. 2.4, Eq. EOM, with
the Oseen or the Rotne-Prager tensor, and the delayed form of Sec. 4), solved
as an ODE on the CPU.  It brackets the lattice Boltzmann velocities; it is
neither the oracle (which runs the same discrete LB/IB step) nor part of the
GPU path."""
from .eom import (BeadSwimmer, drive_forces, integrate, mobility_velocity, oseen, rotne_prager,  # noqa: F401
                  spring_forces, swim_velocity)
