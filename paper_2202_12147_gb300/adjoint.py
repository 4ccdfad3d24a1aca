"""Gradients of swimmer displacements with respect to the drive, through the
hand-written reverse sweep of liblbib (the lb_adjoint_* calls of lbib.h).

    eng = Adjoint(box.dims, assemble(box), n_steps=1000, K=100, precision="f64")
    theta = torch.tensor(eng.theta0, requires_grad=True)     # (n_swimmers, 6)
    disp = displacement(theta, eng)                          # (n_swimmers, 3)
    disp[0, 0].backward()                                    # theta.grad

theta[s] = (A_1, A_2, A_3, phi_1, phi_2, phi_3): the amplitude and phase of
the drive A_b sin(2 pi t / period + phi_b) on each bead of swimmer s (Sec. 2.2,
driving-force equation, with one amplitude and phase per bead).  The
displacement is x_cm(n_steps) - x_cm(0) from the engine's initial state
(Sec. 3, Eq. vel_swim).  Device memory is one torch uint8 tensor; every step of
both sweeps runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check
from .sim import _HostStructure

PRECISION = {"f32": _lib.F32, "f64": _lib.F64}


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Adjoint:
    """One adjoint engine: a periodic box with swimmers, n_steps steps per
    sweep, a checkpoint every K steps, FP32 or FP64 fluid state."""

    def __init__(self, dims, structure, *, n_steps, K=100, precision="f64", tau=1.0, rho0=1.0,
                 g=(0.0, 0.0, 0.0), device="cuda", stream=None):
        self.L = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        p = _lib.LbParams()
        p.nx, p.ny, p.nz = self.dims
        p.tau, p.rho0 = float(tau), float(rho0)
        p.storage = PRECISION[precision]
        p.forcing = _lib.GUO
        p.kernel = _lib.PESKIN4
        p.deterministic = 0
        for a in range(3):
            p.g[a] = float(g[a])
        p.store_scale = 0.0
        self.p = p
        self.hs = _HostStructure(structure)
        self.n_nodes = self.hs.nodes.shape[0]
        self.n_swimmers = self.hs.c.n_swimmers
        self.n_steps, self.K = int(n_steps), int(K)
        nbytes = ctypes.c_size_t()
        check(self.L.lb_adjoint_required_bytes(ctypes.byref(p), ctypes.byref(self.hs.c), self.n_steps, self.K,
                                               ctypes.byref(nbytes)))
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.h = ctypes.c_void_p()
        check(self.L.lb_adjoint_create(ctypes.byref(p), ctypes.byref(self.hs.c), self.n_steps, self.K,
                                       ctypes.c_void_p(self.workspace.data_ptr()), int(nbytes.value),
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.h)))
        sw = structure["swimmers"] if structure else []
        self.theta0 = np.array([list(s["amp"]) + list(s["phase"]) for s in sw], dtype=np.float64).reshape(-1, 6)

    @property
    def workspace_bytes(self):
        return self.workspace.numel()

    def set_drive(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(self.n_swimmers, 6)
        check(self.L.lb_adjoint_set_drive(self.h, _p(th)))

    def set_initial(self, f=None, r=None):
        """f: raw populations (19, n_cells) in the library's lattice order; r: (n_nodes, 3)."""
        fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        ra = None if r is None else np.ascontiguousarray(r, dtype=np.float64).reshape(self.n_nodes, 3)
        check(self.L.lb_adjoint_set_initial(self.h, _p(fa), _p(ra)))

    def forward(self):
        """Run the forward sweep; returns each swimmer's displacement (n_swimmers, 3)."""
        d = np.zeros((max(self.n_swimmers, 1), 3))
        check(self.L.lb_adjoint_forward(self.h, _p(d)))
        return d[: self.n_swimmers]

    def backward(self, seed_disp, seed_f=None, seed_r=None, state_grads=False):
        """Reverse sweep of the last forward sweep for
        L = sum_s seed_disp[s] . disp_s + <seed_f, f(T)> + <seed_r, r(T)>.
        Returns dL/dtheta (n_swimmers, 6), and with state_grads also
        dL/df(0) (19, n_cells) and dL/dr(0) (n_nodes, 3)."""
        sd = np.ascontiguousarray(seed_disp, dtype=np.float64).reshape(max(self.n_swimmers, 1), 3)
        sf = None if seed_f is None else np.ascontiguousarray(seed_f, dtype=np.float64).reshape(19, self.N)
        sr = None if seed_r is None else np.ascontiguousarray(seed_r, dtype=np.float64).reshape(self.n_nodes, 3)
        g = np.zeros((max(self.n_swimmers, 1), 6))
        gf = np.zeros((19, self.N)) if state_grads else None
        gr = np.zeros((max(self.n_nodes, 1), 3)) if state_grads else None
        check(self.L.lb_adjoint_backward(self.h, _p(sd), _p(sf), _p(sr), _p(g), _p(gf), _p(gr)))
        if state_grads:
            return g[: self.n_swimmers], gf, gr[: self.n_nodes]
        return g[: self.n_swimmers]

    def final_state(self):
        f = np.zeros((19, self.N))
        r = np.zeros((max(self.n_nodes, 1), 3))
        check(self.L.lb_adjoint_get_final(self.h, _p(f), _p(r)))
        return f, r[: self.n_nodes]

    def timing(self):
        fm, bm = ctypes.c_double(), ctypes.c_double()
        fl, bl = ctypes.c_longlong(), ctypes.c_longlong()
        check(self.L.lb_adjoint_timing(self.h, ctypes.byref(fm), ctypes.byref(bm), ctypes.byref(fl), ctypes.byref(bl)))
        return dict(forward_ms=fm.value, backward_ms=bm.value, forward_launches=fl.value, backward_launches=bl.value)

    def close(self):
        if self.h:
            check(self.L.lb_adjoint_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DisplacementFn(torch.autograd.Function):
    """theta (n_swimmers, 6) float64 -> displacements (n_swimmers, 3); the
    backward pass is the engine's reverse sweep."""

    @staticmethod
    def forward(ctx, theta, engine):
        engine.set_drive(theta.detach().cpu().numpy())
        disp = engine.forward()
        ctx.engine = engine
        return torch.from_numpy(disp).to(theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.engine.backward(grad_out.detach().cpu().numpy())
        return torch.from_numpy(g).to(grad_out.device), None


def displacement(theta, engine):
    """Differentiable swimmer displacements for drive parameters theta."""
    return DisplacementFn.apply(theta, engine)
