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
_INC = os.path.join(_HERE, "lbib_oracle_step.inc")
_LIB = os.path.join(_HERE, "liblbib_oracle.so")
_lock = threading.Lock()
_lib = None

GUO, SHAN_CHEN = 0, 1
PESKIN4, LINEAR2 = 0, 1
NEOHOOKE, SKALAK = 0, 1


def build(force=False):
    """Compile the oracle with gcc (FMA contraction off so x86 and Arm agree)."""
    stale = not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_INC))
    if force or stale:
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
            L.orc_bending_rest.argtypes = [i, P, P, P]
            L.orc_bending_energy_v.argtypes = [d, i, P, P, P, P]
            L.orc_bending_forces.argtypes = [d, i, P, P, P, P]
            L.orc_volume.argtypes = [i, P, P, P]
            L.orc_volume_forces.argtypes = [d, d, i, P, P, P]
            L.orc_set_threads.argtypes = [i]
            L.orc_set_threads.restype = i
            # complex-step twins (double complex arguments as complex128 arrays)
            L.orc_lb_step_cs.argtypes = [i, i, i, d, i, P, P, P, P, P, P]
            L.orc_phi_cs.argtypes = [i, P, P]
            L.orc_spread_cs.argtypes = [i, i, i, i, i, P, P, P]
            L.orc_interpolate_cs.argtypes = [i, i, i, i, i, P, P, P]
            L.orc_bead_centres_cs.argtypes = [i, P, P, P]
            L.orc_drive_cs.argtypes = [P, P, i, d, d, P]
            L.orc_springs_cs.argtypes = [d, d, P, P]
            L.orc_membrane_energy_v_cs.argtypes = [i, d, d, i, P, P, P, P]
            L.orc_membrane_forces_cs.argtypes = [i, d, d, i, P, P, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _is_c(*arrays):
    """True if any argument is complex: the call then runs the complex-step
    twin of the C function on complex128 copies of every array."""
    return any(np.iscomplexobj(a) for a in arrays if a is not None)


def _fn(name, cplx):
    return getattr(lib(), name + "_cs" if cplx else name)


def set_threads(n):
    """OpenMP threads of the oracle's loops (n <= 0: query); returns the count in effect."""
    return lib().orc_set_threads(int(n))


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
    if _is_c(np.asarray(r)):
        x = np.array([r], dtype=np.complex128)
        out = np.zeros(1, dtype=np.complex128)
        lib().orc_phi_cs(kernel, _p(x), _p(out))
        return complex(out[0])
    return lib().orc_phi(kernel, float(r))


def lb_step(f, dims, tau, F=None, g=(0.0, 0.0, 0.0), forcing=GUO):
    """One collide+stream of raw populations f (N,19). Returns (fnew, rho, u).
    Complex inputs run the complex-step twin."""
    nx, ny, nz = dims
    cplx = _is_c(f, F, np.asarray(g))
    cv = _c128 if cplx else _f64
    f = cv(f)
    fnew = np.empty_like(f)
    rho = np.empty(f.shape[0], dtype=f.dtype)
    u = np.empty((f.shape[0], 3), dtype=f.dtype)
    g = cv(g)
    Fp = None
    if F is not None:
        F = cv(F)
        Fp = _p(F)
    _fn("orc_lb_step", cplx)(nx, ny, nz, float(tau), forcing, Fp, _p(g), _p(f), _p(fnew), _p(rho), _p(u))
    return fnew, rho, u


def macros(f):
    f = _f64(f)
    rho = np.empty(f.shape[0])
    u = np.empty((f.shape[0], 3))
    lib().orc_macros(f.shape[0], _p(f), _p(rho), _p(u))
    return rho, u


def spread(r, fn, dims, kernel=PESKIN4, F=None):
    nx, ny, nz = dims
    cplx = _is_c(r, fn, F)
    cv = _c128 if cplx else _f64
    r, fn = cv(r), cv(fn)
    if F is None:
        F = np.zeros((nx * ny * nz, 3), dtype=r.dtype)
    elif F.dtype != r.dtype or not F.flags.c_contiguous:
        raise TypeError("F must be a C-contiguous array of the arguments' dtype")
    _fn("orc_spread", cplx)(kernel, nx, ny, nz, r.shape[0], _p(r), _p(fn), _p(F))
    return F


def interpolate(r, u, dims, kernel=PESKIN4):
    nx, ny, nz = dims
    cplx = _is_c(r, u)
    cv = _c128 if cplx else _f64
    r, u = cv(r), cv(u)
    v = np.zeros((r.shape[0], 3), dtype=r.dtype)
    _fn("orc_interpolate", cplx)(kernel, nx, ny, nz, r.shape[0], _p(r), _p(u), _p(v))
    return v


def bead_centres(r, beads):
    beads = np.ascontiguousarray(beads, dtype=np.int32)
    cplx = _is_c(r)
    r = (_c128 if cplx else _f64)(r)
    R = np.zeros((beads.shape[0], 3), dtype=r.dtype)
    _fn("orc_bead_centres", cplx)(beads.shape[0], _p(beads), _p(r), _p(R))
    return R


def drive(amp, phase, balance, period, t):
    cplx = _is_c(np.asarray(amp), np.asarray(phase))
    cv = _c128 if cplx else _f64
    out = np.zeros((3, 3), dtype=np.complex128 if cplx else np.float64)
    _fn("orc_drive", cplx)(_p(cv(amp)), _p(cv(phase)), int(balance), float(period), float(t), _p(out))
    return out


def springs(k, L, R):
    cplx = _is_c(R)
    R = (_c128 if cplx else _f64)(R)
    out = np.zeros((3, 3), dtype=R.dtype)
    _fn("orc_springs", cplx)(float(k), float(L), _p(R), _p(out))
    return out


def membrane_energy(X, x, tris, p1, p2=0.0, law=NEOHOOKE):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    if _is_c(X, x):
        W = np.zeros(1, dtype=np.complex128)
        lib().orc_membrane_energy_v_cs(law, float(p1), float(p2), tris.shape[0], _p(tris), _p(_c128(X)),
                                       _p(_c128(x)), _p(W))
        return complex(W[0])
    return lib().orc_membrane_energy(law, float(p1), float(p2), tris.shape[0], _p(tris), _p(_f64(X)), _p(_f64(x)))


def membrane_forces(X, x, tris, p1, p2=0.0, law=NEOHOOKE, out=None):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    cplx = _is_c(X, x, out)
    cv = _c128 if cplx else _f64
    x = cv(x)
    if out is None:
        out = np.zeros_like(x)
    elif out.dtype != x.dtype or not out.flags.c_contiguous:
        raise TypeError("out must be a C-contiguous array of the positions' dtype")
    _fn("orc_membrane_forces", cplx)(law, float(p1), float(p2), tris.shape[0], _p(tris), _p(cv(X)), _p(x), _p(out))
    return out


# Kantor-Nelson bending (Sec. 2.2): the discrete energy kb_disc (1 - cos(theta
# - theta0)) per edge stands for the Helfrich energy kb/2 (2H)^2 dA; on a
# regular triangulation of a sphere of radius R the normals of neighbouring
# triangles (edge l, centroids l / sqrt(3) apart) differ by theta = l / (sqrt(3) R),
# so sum_e (1 - cos theta) -> 4 pi / sqrt(3) against the Helfrich 8 pi:
# kb_disc = 2 sqrt(3) kb.
KB_DISC_PER_KB = 2.0 * 3.0 ** 0.5


def bending_edges(tris):
    """Every edge shared by two triangles as (a, b, c, d): the edge a-b, c the
    third node of the triangle that runs a -> b, d that of the one running
    b -> a (both outward).  Raises unless every edge has exactly those two."""
    tris = np.asarray(tris)
    third = {}
    for t in tris:
        for k in range(3):
            a, b, c = int(t[k]), int(t[(k + 1) % 3]), int(t[(k + 2) % 3])
            if (a, b) in third:
                raise ValueError(f"directed edge {a}->{b} in two triangles")
            third[(a, b)] = c
    out = []
    for (a, b), c in third.items():
        if a < b:
            if (b, a) not in third:
                raise ValueError(f"edge {a}-{b} on one triangle only (open surface)")
            out.append((a, b, c, third[(b, a)]))
    return np.array(out, dtype=np.int32).reshape(-1, 4)


def bending_rest(edges, X):
    """(ne, 2): cos and sin of every edge's angle at the rest positions X."""
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    out = np.zeros((edges.shape[0], 2))
    lib().orc_bending_rest(edges.shape[0], _p(edges), _p(_f64(X)), _p(out))
    return out


def bending_energy(kb, edges, cs0, x):
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    W = np.zeros(1)
    lib().orc_bending_energy_v(KB_DISC_PER_KB * float(kb), edges.shape[0], _p(edges), _p(_f64(cs0)), _p(_f64(x)),
                               _p(W))
    return float(W[0])


def bending_forces(kb, edges, cs0, x, out=None):
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    x = _f64(x)
    if out is None:
        out = np.zeros_like(x)
    elif out.dtype != np.float64 or not out.flags.c_contiguous:
        raise TypeError("out must be a C-contiguous float64 array")
    lib().orc_bending_forces(KB_DISC_PER_KB * float(kb), edges.shape[0], _p(edges), _p(_f64(cs0)), _p(x), _p(out))
    return out


def volume(tris, x):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    V = np.zeros(1)
    lib().orc_volume(tris.shape[0], _p(tris), _p(_f64(x)), _p(V))
    return float(V[0])


def volume_forces(kv, V0, tris, x, out=None):
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    x = _f64(x)
    if out is None:
        out = np.zeros_like(x)
    elif out.dtype != np.float64 or not out.flags.c_contiguous:
        raise TypeError("out must be a C-contiguous float64 array")
    lib().orc_volume_forces(float(kv), float(V0), tris.shape[0], _p(tris), _p(x), _p(out))
    return out


class OracleSim:
    """The coupled LB/IB time step in FP64 (order as in the module docstring).

    State: raw populations f (N,19) in the oracle's lattice order, node
    positions (M,3) unwrapped, step counter t.  The rest shape of every
    membrane is the node set given at construction.

    dtype=np.complex128 runs the complex-step twin of every function; `drive`
    optionally replaces each swimmer's drive parameters by an (n_swimmers, 6)
    array (A1, A2, A3, phi1, phi2, phi3), complex for complex-step
    derivatives.  For a swimmer with `balance`, A2 and phi2 are unused.
    """

    def __init__(self, box, asm=None, f=None, dtype=np.float64, drive=None):
        from workloads import assemble
        self.box = box
        self.dims = tuple(box.dims)
        self.N = box.n_cells
        self.dtype = np.dtype(dtype)
        self.asm = asm if asm is not None else assemble(box)
        self.c, self.w = lattice()
        self.f = (np.tile(self.w * box.rho0, (self.N, 1)) if f is None else np.array(f)).astype(self.dtype)
        self.rest = self.asm["nodes"].astype(self.dtype)
        self.r = self.asm["nodes"].astype(self.dtype)
        self.t = 0
        self.forcing = SHAN_CHEN if box.forcing == "shan_chen" else GUO
        self.kernel = LINEAR2 if box.kernel == "linear2" else PESKIN4
        self.drive = drive_parameters(self.asm) if drive is None else np.array(drive)
        self.drive = self.drive.astype(np.result_type(self.drive.dtype, np.float64))
        self.u = np.zeros((self.N, 3), dtype=self.dtype)
        self.rho = np.full(self.N, box.rho0, dtype=self.dtype)
        self.v = np.zeros_like(self.r)
        self.node_force = np.zeros_like(self.r)
        self.F = None
        # per bead: membrane law, bending edges with their rest angles, rest volume
        nb = self.asm["beads"].shape[0]
        self.law = np.asarray(self.asm.get("bead_law", np.zeros(nb, np.int32)))
        self.skC = np.asarray(self.asm.get("bead_C", np.zeros(nb)))
        self.kb = np.asarray(self.asm.get("bead_kb", np.zeros(nb)))
        self.kv = np.asarray(self.asm.get("bead_kv", np.zeros(nb)))
        self.bend = {}
        self.V0 = {}
        for b in range(nb):
            n0, nn, t0, nt = self.asm["beads"][b]
            tris = self.asm["tris"][t0:t0 + nt]
            if self.kb[b] != 0.0:
                ed = bending_edges(tris)
                self.bend[b] = (ed, bending_rest(ed, self.asm["nodes"]))
            if self.kv[b] != 0.0:
                self.V0[b] = volume(tris, self.asm["nodes"])

    def node_forces(self):
        """Steps 1-3: f^tot for every node at the current positions and time."""
        a = self.asm
        beads = a["beads"]
        R = bead_centres(self.r, beads)
        fn = np.zeros(self.r.shape, dtype=np.result_type(self.r.dtype, self.drive.dtype))
        for b in range(beads.shape[0]):
            n0, nn, t0, nt = beads[b]
            law = SKALAK if self.law[b] == 1 else NEOHOOKE
            membrane_forces(self.rest.astype(fn.dtype), self.r.astype(fn.dtype), a["tris"][t0:t0 + nt],
                            a["bead_Gs"][b], self.skC[b], law=law, out=fn)
            if b in self.bend or b in self.V0:
                if fn.dtype != np.float64:
                    raise NotImplementedError("bending and volume forces are real-valued only")
                if b in self.bend:
                    bending_forces(self.kb[b], *self.bend[b], self.r, out=fn)
                if b in self.V0:
                    volume_forces(self.kv[b], self.V0[b], a["tris"][t0:t0 + nt], self.r, out=fn)
        for k, s in enumerate(a["swimmers"]):
            ids = s["beads"]
            fd = drive(self.drive[k, 0:3], self.drive[k, 3:6], s["balance"], s["period"], self.t)
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


# ----------------------------------------------------------------------------
# Net displacement and its derivatives with respect to the drive parameters
# ----------------------------------------------------------------------------

def drive_parameters(asm):
    """(n_swimmers, 6) array of each swimmer's drive (A1, A2, A3, phi1, phi2, phi3)."""
    return np.array([list(s["amp"]) + list(s["phase"]) for s in asm["swimmers"]], dtype=np.float64).reshape(-1, 6)


def displacement(box, steps, drive=None, asm=None, dtype=np.float64):
    """Net displacement x_cm(steps) - x_cm(0) of every swimmer, (n_swimmers, 3),
    starting from rest (Sec. 3: the swimmer's displacement over its stroke)."""
    sim = OracleSim(box, asm, dtype=dtype, drive=drive)
    x0 = sim.swimmer_centres()
    sim.step(steps)
    return sim.swimmer_centres() - x0


def displacement_jacobian_cs(box, steps, params, drive=None, asm=None, h=1e-30):
    """Exact derivative of the discrete map: d disp / d theta_p for each
    parameter p = (swimmer, index into the 6 drive entries), by the complex
    step theta_p + i h (Squire & Trapp 1998).  Returns (len(params), n_sw, 3)."""
    from workloads import assemble
    asm = asm if asm is not None else assemble(box)
    base = drive_parameters(asm) if drive is None else np.asarray(drive, dtype=np.float64)
    out = []
    for (s, k) in params:
        th = base.astype(np.complex128)
        th[s, k] += 1j * h
        d = displacement(box, steps, th, asm, dtype=np.complex128)
        out.append(d.imag / h)
    return np.array(out)


def displacement_jacobian_fd(box, steps, params, drive=None, asm=None, rel_h=1e-6):
    """Central finite differences of the FP64 displacement with step
    h = rel_h * |theta_p|.  Returns (len(params), n_sw, 3)."""
    from workloads import assemble
    asm = asm if asm is not None else assemble(box)
    base = drive_parameters(asm) if drive is None else np.asarray(drive, dtype=np.float64)
    out = []
    for (s, k) in params:
        h = rel_h * abs(base[s, k])
        tp, tm = base.copy(), base.copy()
        tp[s, k] += h
        tm[s, k] -= h
        dp = displacement(box, steps, tp, asm)
        dm = displacement(box, steps, tm, asm)
        out.append((dp - dm) / (2.0 * h))
    return np.array(out)
