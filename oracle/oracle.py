"""Python driver of the FP64 oracle (lbib_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark; never by the product package.

`OracleSim` runs the coupled step in the order this build reads from the
paper (the paper does not state a sub-step order):
  1. bead centres R_b = mean of their nodes           (Fig. 1 caption)
  2. drive f^d(t) and springs f^s(R) per swimmer       (Sec. 2.2)
  3. nodal force f^tot = f^part + (f^d + f^s)/N_v     (Sec. 2.2, total nodal force)
  4. spread F(x) = sum_j f^tot_j Delta(x - r_j)        (Sec. 2.3, Eq. spreading)
  5. LB collide (+force) and stream                    (Sec. 2.1, Eqs. lbe, lbm:equilibrium)
  6. interpolate u(x, t) at r_j                        (Sec. 2.3, Eq. interpolation)
  7. r_j <- r_j + rdot_j  (forward Euler, dt = 1)      (Sec. 2.3, front tracking)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_LIB = os.path.join(_HERE, "liblbib_oracle.so")
_lock = threading.Lock()
_lib = None

GUO, SHAN_CHEN = 0, 1
PESKIN4, LINEAR2 = 0, 1
NEOHOOKE, SKALAK = 0, 1


def build(force=False):
    """Compile the oracle with gcc (FMA contraction off so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.orc_lattice.argtypes = [P, P]
            L.orc_equilibrium.argtypes = [d, P, P]
            L.orc_lb_step.argtypes = [i, i, i, d, i, P, P, P, P, P, P]
            L.orc_macros.argtypes = [ctypes.c_long, P, P, P]
            L.orc_phi.argtypes = [i, d]
            L.orc_phi.restype = d
            L.orc_spread.argtypes = [i, i, i, i, i, P, P, P]
            L.orc_interpolate.argtypes = [i, i, i, i, i, P, P, P]
            L.orc_bead_centres.argtypes = [i, P, P, P]
            L.orc_drive.argtypes = [P, P, i, d, d, P]
            L.orc_springs.argtypes = [d, d, P, P]
            L.orc_membrane_energy.argtypes = [i, d, d, i, P, P, P]
            L.orc_membrane_energy.restype = d
            L.orc_membrane_forces.argtypes = [i, d, d, i, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib().orc_lattice(_p(c), _p(w))
    return c, w


def equilibrium(rho, u):
    u = _f64(u)
    out = np.zeros(19)
    lib().orc_equilibrium(float(rho), _p(u), _p(out))
    return out


def phi(r, kernel=PESKIN4):
    return lib().orc_phi(kernel, float(r))


def lb_step(f, dims, tau, F=None, g=(0.0, 0.0, 0.0), forcing=GUO):
    """One collide+stream of raw populations f (N,19). Returns (fnew, rho, u)."""
    nx, ny, nz = dims
    f = _f64(f)
    fnew = np.empty_like(f)
    rho = np.empty(f.shape[0])
    u = np.empty((f.shape[0], 3))
    g = _f64(g)
    Fp = _p(_f64(F)) if F is not None else None
    if F is not None:
        F = _f64(F)
        Fp = _p(F)
    lib().orc_lb_step(nx, ny, nz, float(tau), forcing, Fp, _p(g), _p(f), _p(fnew), _p(rho), _p(u))
    return fnew, rho, u


def macros(f):
    f = _f64(f)
    rho = np.empty(f.shape[0])
    u = np.empty((f.shape[0], 3))
    lib().orc_macros(f.shape[0], _p(f), _p(rho), _p(u))
    return rho, u


def spread(r, fn, dims, kernel=PESKIN4, F=None):
    nx, ny, nz = dims
    r, fn = _f64(r), _f64(fn)
    if F is None:
        F = np.zeros((nx * ny * nz, 3))
    lib().orc_spread(kernel, nx, ny, nz, r.shape[0], _p(r), _p(fn), _p(F))
    return F


def interpolate(r, u, dims, kernel=PESKIN4):
    nx, ny, nz = dims
    r, u = _f64(r), _f64(u)
    v = np.zeros((r.shape[0], 3))
    lib().orc_interpolate(kernel, nx, ny, nz, r.shape[0], _p(r), _p(u), _p(v))
    return v


def bead_centres(r, beads):
    beads = np.ascontiguousarray(beads, dtype=np.int32)
    R = np.zeros((beads.shape[0], 3))
    lib().orc_bead_centres(beads.shape[0], _p(beads), _p(_f64(r)), _p(R))
    return R


def drive(amp, phase, balance, period, t):
    out = np.zeros((3, 3))
    lib().orc_drive(_p(_f64(amp)), _p(_f64(phase)), int(balance), float(period), float(t), _p(out))
    return out


def springs(k, L, R):
    out = np.zeros((3, 3))
    lib().orc_springs(float(k), float(L), _p(_f64(R)), _p(out))
    return out


def membrane_energy(X, x, tris, p1, p2=0.0, law=NEOHOOKE):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    return lib().orc_membrane_energy(law, float(p1), float(p2), tris.shape[0], _p(tris), _p(_f64(X)), _p(_f64(x)))


def membrane_forces(X, x, tris, p1, p2=0.0, law=NEOHOOKE, out=None):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    x = _f64(x)
    if out is None:
        out = np.zeros_like(x)
    lib().orc_membrane_forces(law, float(p1), float(p2), tris.shape[0], _p(tris), _p(_f64(X)), _p(x), _p(out))
    return out


class OracleSim:
    """The coupled LB/IB time step in FP64 (order as in the module docstring).

    State: raw populations f (N,19) in the oracle's lattice order, node
    positions (M,3) unwrapped, step counter t.  The rest shape of every
    membrane is the node set given at construction.
    """

    def __init__(self, box, asm=None, f=None):
        from workloads import assemble
        self.box = box
        self.dims = tuple(box.dims)
        self.N = box.n_cells
        self.asm = asm if asm is not None else assemble(box)
        self.c, self.w = lattice()
        self.f = np.tile(self.w * box.rho0, (self.N, 1)) if f is None else _f64(f).copy()
        self.rest = self.asm["nodes"].copy()
        self.r = self.asm["nodes"].copy()
        self.t = 0
        self.forcing = SHAN_CHEN if box.forcing == "shan_chen" else GUO
        self.kernel = LINEAR2 if box.kernel == "linear2" else PESKIN4
        self.u = np.zeros((self.N, 3))
        self.rho = np.full(self.N, box.rho0)
        self.v = np.zeros_like(self.r)
        self.node_force = np.zeros_like(self.r)
        self.F = None

    def node_forces(self):
        """Steps 1-3: f^tot for every node at the current positions and time."""
        a = self.asm
        beads = a["beads"]
        R = bead_centres(self.r, beads)
        fn = np.zeros_like(self.r)
        for b in range(beads.shape[0]):
            n0, nn, t0, nt = beads[b]
            membrane_forces(self.rest, self.r, a["tris"][t0:t0 + nt], a["bead_Gs"][b], out=fn)
        for s in a["swimmers"]:
            ids = s["beads"]
            fd = drive(s["amp"], s["phase"], s["balance"], s["period"], self.t)
            fs = springs(s["k"], s["L"], R[ids])
            for q, b in enumerate(ids):
                n0, nn = beads[b][0], beads[b][1]
                fn[n0:n0 + nn] += (fd[q] + fs[q]) / nn
        return fn

    def step(self, n=1):
        for _ in range(n):
            if self.r.shape[0]:
                self.node_force = self.node_forces()
                self.F = spread(self.r, self.node_force, self.dims, self.kernel)
            else:
                self.F = None
            self.f, self.rho, self.u = lb_step(self.f, self.dims, self.box.tau, self.F, self.box.g, self.forcing)
            if self.r.shape[0]:
                self.v = interpolate(self.r, self.u, self.dims, self.kernel)
                self.r = self.r + self.v
            self.t += 1
        return self

    def swimmer_centres(self):
        """x_cm of every swimmer: the mean of its three bead centres (Sec. 3, Eq. vel_swim)."""
        R = bead_centres(self.r, self.asm["beads"])
        return np.array([R[s["beads"]].mean(axis=0) for s in self.asm["swimmers"]])
