"""Bead-spring swimmers in an unbounded Stokes fluid (Sec. 2.4).

Each bead i moves with its own Stokes mobility plus the flow that the other
beads' forces make at its centre (Eq. EOM):

    dR_i/dt = (f^d_i + f^s_i) / (6 pi mu a) + sum_{j != i} T(R_i - R_j) . (f^d_j + f^s_j)

with T the Oseen tensor (point forces) or the Rotne-Prager tensor (finite
spheres, Faxen-corrected).  The drive and the springs are those of Sec. 2.2:
f^d_1 = A sin(w t) x, f^d_3 = B sin(w t + alpha) x, f^d_2 = -f^d_1 - f^d_3;
f^s_1 = -k (|R_1 - R_2| - L) (R_1 - R_2)/|R_1 - R_2|, likewise f^s_3 with
R_3 - R_2, and f^s_2 = -f^s_1 - f^s_3.  Every bead of every swimmer interacts
with every other bead.  In the delayed form (Sec. 4, Eq. fit-eq) bead j
acts on bead i with its position and force of time t - tau_delay; before
t = 0 the swimmers rest at their initial positions with no drive.

The ODE is advanced by the classical fourth-order Runge-Kutta method with a
fixed step; delayed values between stored steps come from cubic Hermite
interpolation of the stored positions and velocities.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def oseen(r, mu):
    """Oseen tensor (Sec. 2.4): (I + r r^T / r^2) / (8 pi mu |r|), shape (..., 3, 3)."""
    r = np.asarray(r, dtype=np.float64)
    d = np.linalg.norm(r, axis=-1)[..., None, None]
    rr = r[..., :, None] * r[..., None, :]
    return (np.eye(3) + rr / d ** 2) / (8.0 * math.pi * mu * d)


def rotne_prager(r, mu, a):
    """Rotne-Prager tensor (Sec. 2.4, Eq. Rotne-Prager): the Oseen tensor plus
    a^2 / (12 pi mu |r|^3) (I - 3 r r^T / r^2)."""
    r = np.asarray(r, dtype=np.float64)
    d = np.linalg.norm(r, axis=-1)[..., None, None]
    rr = r[..., :, None] * r[..., None, :]
    return oseen(r, mu) + a * a / (12.0 * math.pi * mu * d ** 3) * (np.eye(3) - 3.0 * rr / d ** 2)


def _tensor(kind, r, mu, a):
    if kind == "oseen":
        return oseen(r, mu)
    if kind == "rotne_prager":
        return rotne_prager(r, mu, a)
    if kind == "none":
        return np.zeros(np.shape(r)[:-1] + (3, 3))
    raise ValueError(kind)


def mobility_velocity(R, F, mu, a, tensor="rotne_prager", R_src=None, F_src=None):
    """Velocities of beads at R (n, 3) under forces F (n, 3) by Eq. EOM: the
    Stokes self term F_i / (6 pi mu a) plus sum_{j != i} T(R_i - R_j) F_j.
    R_src, F_src (default R, F) are the positions and forces the other beads
    act with (the delayed form uses earlier ones)."""
    R = np.asarray(R, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    Rs = R if R_src is None else np.asarray(R_src, dtype=np.float64)
    Fs = F if F_src is None else np.asarray(F_src, dtype=np.float64)
    V = F / (6.0 * math.pi * mu * a)
    n = R.shape[0]
    if n < 2 or tensor == "none":
        return V
    i, j = np.nonzero(~np.eye(n, dtype=bool))  # every ordered pair i != j
    T = _tensor(tensor, R[i] - Rs[j], mu, a)  # (pairs, 3, 3)
    np.add.at(V, i, np.einsum("pab,pb->pa", T, Fs[j]))
    return V


def drive_forces(t, A, B, alpha, period):
    """x components of the three driving forces at time t (Sec. 2.2); zero
    before t = 0."""
    if t < 0.0:
        return np.zeros(3)
    w = 2.0 * math.pi / period
    f1 = A * math.sin(w * t)
    f3 = B * math.sin(w * t + alpha)
    return np.array([f1, -f1 - f3, f3])


def spring_forces(R, k, L):
    """Spring forces on the three beads of one swimmer, R (3, 3) (Sec. 2.2)."""
    d1 = R[0] - R[1]
    d3 = R[2] - R[1]
    n1 = np.linalg.norm(d1)
    n3 = np.linalg.norm(d3)
    f1 = -k * (n1 - L) * d1 / n1
    f3 = -k * (n3 - L) * d3 / n3
    return np.array([f1, -f1 - f3, f3])


@dataclass
class BeadSwimmer:
    """One three-bead swimmer: centre-bead position, bead radius, spring
    stiffness and rest length, drive amplitudes, phase shift and period;
    the beads start at rest spacing along x."""
    center: tuple
    a: float
    k: float
    L: float
    A: float
    B: float
    alpha: float
    period: float

    def rest_positions(self):
        c = np.asarray(self.center, dtype=np.float64)
        return np.array([c - [self.L, 0, 0], c, c + [self.L, 0, 0]])


def _forces(swimmers, R, t):
    """Drive plus spring force of every bead, (3 n_swimmers, 3)."""
    F = np.zeros_like(R)
    for s, sw in enumerate(swimmers):
        Rs = R[3 * s:3 * s + 3]
        F[3 * s:3 * s + 3] = spring_forces(Rs, sw.k, sw.L)
        F[3 * s:3 * s + 3, 0] += drive_forces(t, sw.A, sw.B, sw.alpha, sw.period)
    return F


def integrate(swimmers, t_end, dt, mu, tensor="rotne_prager", delay=0.0, sample_every=None):
    """Advance the swimmers from rest to t_end with step dt.  Returns
    (times, x_cm) with x_cm (samples, n_swimmers, 3) the swimmers' centres
    (the mean of their three beads, Sec. 3) at every sample_every-th step
    (default: every step).  With delay > 0, bead j acts on bead i with its
    position and force of time t - delay; delay must be a multiple of dt."""
    a_all = {sw.a for sw in swimmers}
    if len(a_all) != 1:
        raise ValueError("all beads must have one radius")
    a = a_all.pop()
    n_steps = int(round(t_end / dt))
    m = int(round(delay / dt))
    if abs(m * dt - delay) > 1e-9 * max(1.0, delay):
        raise ValueError("delay must be a multiple of dt")
    R0 = np.concatenate([sw.rest_positions() for sw in swimmers])
    every = sample_every or 1
    hist_R = [R0]      # positions at every step (for the delayed form)
    hist_V = []        # velocities at every step
    R = R0.copy()

    def delayed(t):
        """Positions and forces at time t - delay (rest state before 0)."""
        tq = t - delay
        if tq <= 0.0:
            return R0, _forces(swimmers, R0, tq)
        x = tq / dt
        n = int(math.floor(x + 1e-12))
        th = x - n
        if th < 1e-12:
            Rq = hist_R[n]
        else:
            y0, y1, v0, v1 = hist_R[n], hist_R[n + 1], hist_V[n], hist_V[n + 1]
            h00 = 2 * th ** 3 - 3 * th ** 2 + 1
            h10 = th ** 3 - 2 * th ** 2 + th
            h01 = -2 * th ** 3 + 3 * th ** 2
            h11 = th ** 3 - th ** 2
            Rq = h00 * y0 + h10 * dt * v0 + h01 * y1 + h11 * dt * v1
        return Rq, _forces(swimmers, Rq, tq)

    def rhs(t, Rt):
        F = _forces(swimmers, Rt, t)
        if m == 0:
            return mobility_velocity(Rt, F, mu, a, tensor)
        Rd, Fd = delayed(t)
        return mobility_velocity(Rt, F, mu, a, tensor, R_src=Rd, F_src=Fd)

    times = [0.0]
    xs = [np.array([R[3 * s:3 * s + 3].mean(axis=0) for s in range(len(swimmers))])]
    for n in range(n_steps):
        t = n * dt
        k1 = rhs(t, R)
        hist_V.append(k1)
        k2 = rhs(t + 0.5 * dt, R + 0.5 * dt * k1)
        k3 = rhs(t + 0.5 * dt, R + 0.5 * dt * k2)
        k4 = rhs(t + dt, R + dt * k3)
        R = R + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        hist_R.append(R)
        if (n + 1) % every == 0:
            times.append((n + 1) * dt)
            xs.append(np.array([R[3 * s:3 * s + 3].mean(axis=0) for s in range(len(swimmers))]))
    return np.array(times), np.array(xs)


def swim_velocity(times, xcm, period, last_periods=1):
    """Mean x velocity of every swimmer over the last `last_periods` whole
    drive periods of a trajectory (Sec. 3, Eq. vel_swim)."""
    t_end = times[-1]
    t0 = t_end - last_periods * period
    i0 = int(np.argmin(np.abs(times - t0)))
    if abs(times[i0] - t0) > 1e-9 * max(1.0, period):
        raise ValueError("the trajectory has no sample at the start of the window")
    return (xcm[-1, :, 0] - xcm[i0, :, 0]) / (t_end - times[i0])
