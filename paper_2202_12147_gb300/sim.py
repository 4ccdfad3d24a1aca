"""Python face of liblbib: one periodic box with its swimmers on one GPU.

The caller-owned device buffers are torch tensors (PyTorch provides device
memory and the stream); every computation happens in the CUDA library.

Structure format (host arrays):
  nodes    (M,3) float64  rest shape = initial node positions
  tris     (T,3) int32    global node ids, outward orientation
  beads    (B,4) int32    node_start, node_count, tri_start, tri_count
  bead_Gs  (B,)  float64  neo-Hookean shear modulus of each bead (Skalak: kappa_s)
  bead_law, bead_C, bead_kb, bead_kv (B,), optional: membrane law (0
           neo-Hookean, 1 Skalak), Skalak C, bending and volume moduli
  swimmers list of dicts with keys beads (3 ids), k, L, amp (3), phase (3),
           balance (bool), period
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check

STORAGE = {"f32": _lib.F32, "f16": _lib.F16, "bf16": _lib.BF16}
FORCING = {"guo": _lib.GUO, "shan_chen": _lib.SHAN_CHEN}
KERNEL = {"peskin4": _lib.PESKIN4, "linear2": _lib.LINEAR2}


def lattice():
    """The library's D3Q19 set: c (19,3) int32 and w (19,) in storage order."""
    L = _lib.load()
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    check(L.lbib_lattice(c.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)))
    return c, w


def _params(dims, tau, rho0, storage, forcing, kernel, deterministic, g, store_scale):
    p = _lib.LbParams()
    p.nx, p.ny, p.nz = (int(d) for d in dims)
    p.tau, p.rho0 = float(tau), float(rho0)
    p.storage = STORAGE[storage]
    p.forcing = FORCING[forcing]
    p.kernel = KERNEL[kernel]
    p.deterministic = 1 if deterministic else 0
    for a in range(3):
        p.g[a] = float(g[a])
    p.store_scale = float(store_scale)
    return p


class _HostStructure:
    """Keeps the ctypes views and their backing arrays alive together."""

    def __init__(self, st):
        st = st or dict(nodes=np.zeros((0, 3)), tris=np.zeros((0, 3), np.int32), beads=np.zeros((0, 4), np.int32),
                        bead_Gs=np.zeros(0), swimmers=[])
        self.nodes = np.ascontiguousarray(st["nodes"], dtype=np.float64)
        self.tris = np.ascontiguousarray(st["tris"], dtype=np.int32)
        beads = np.asarray(st["beads"], dtype=np.int32).reshape(-1, 4)
        gs = np.asarray(st["bead_Gs"], dtype=np.float64)
        nb = len(beads)
        law = np.asarray(st.get("bead_law", np.zeros(nb, np.int32)))
        cc = np.asarray(st.get("bead_C", np.zeros(nb)), dtype=np.float64)
        kb = np.asarray(st.get("bead_kb", np.zeros(nb)), dtype=np.float64)
        kv = np.asarray(st.get("bead_kv", np.zeros(nb)), dtype=np.float64)
        self.B = (_lib.Bead * max(1, nb))()
        for b, row in enumerate(beads):
            self.B[b].node_start, self.B[b].node_count, self.B[b].tri_start, self.B[b].tri_count = (int(v) for v in row)
            self.B[b].Gs = float(gs[b])
            self.B[b].law = int(law[b])
            self.B[b].C = float(cc[b])
            self.B[b].kb = float(kb[b])
            self.B[b].kv = float(kv[b])
        sws = st["swimmers"]
        self.S = (_lib.Swimmer * max(1, len(sws)))()
        for k, s in enumerate(sws):
            for q in range(3):
                self.S[k].bead[q] = int(s["beads"][q])
                self.S[k].amp[q] = float(s["amp"][q])
                self.S[k].phase[q] = float(s["phase"][q])
            self.S[k].k_spring = float(s["k"])
            self.S[k].L_spring = float(s["L"])
            self.S[k].balance = 1 if s["balance"] else 0
            self.S[k].period = float(s["period"])
        self.c = _lib.Structure()
        self.c.n_beads, self.c.n_swimmers = len(beads), len(sws)
        self.c.n_nodes, self.c.n_tris = self.nodes.shape[0], self.tris.shape[0]
        self.c.beads = ctypes.cast(self.B, ctypes.POINTER(_lib.Bead))
        self.c.swimmers = ctypes.cast(self.S, ctypes.POINTER(_lib.Swimmer))
        self.c.rest_nodes = self.nodes.ctypes.data_as(ctypes.c_void_p)
        self.c.tris = self.tris.ctypes.data_as(ctypes.c_void_p)


def required_sizes(dims, structure=None, *, tau=1.0, rho0=1.0, storage="f32", forcing="guo", kernel="peskin4",
                   deterministic=False, g=(0.0, 0.0, 0.0), store_scale=0.0):
    L = _lib.load()
    p = _params(dims, tau, rho0, storage, forcing, kernel, deterministic, g, store_scale)
    hs = _HostStructure(structure)
    out = (ctypes.c_size_t * _lib.NBUF)()
    check(L.lbib_required_sizes(ctypes.byref(p), ctypes.byref(hs.c), out))
    return [int(v) for v in out]


class Simulation:
    """A periodic D3Q19 box with immersed three-bead swimmers on one GPU.

    Method names follow the C ABI (lb_step, ib_spread, ib_interpolate,
    swimmer_state, ...).  Work is queued on `stream` (default: torch's current
    stream at construction)."""

    def __init__(self, dims, structure=None, *, tau=1.0, rho0=1.0, storage="f32", forcing="guo",
                 kernel="peskin4", deterministic=False, g=(0.0, 0.0, 0.0), store_scale=0.0, device="cuda",
                 stream=None):
        self.L = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        self.rho0 = float(rho0)
        self.p = _params(dims, tau, rho0, storage, forcing, kernel, deterministic, g, store_scale)
        self.hs = _HostStructure(structure)
        self.n_nodes = self.hs.nodes.shape[0]
        self.n_swimmers = self.hs.c.n_swimmers
        out = (ctypes.c_size_t * _lib.NBUF)()
        check(self.L.lbib_required_sizes(ctypes.byref(self.p), ctypes.byref(self.hs.c), out))
        self.device = torch.device(device)
        # 256-byte aligned torch allocations (the caching allocator aligns to 512 B)
        self.bufs = [torch.empty(int(n), dtype=torch.uint8, device=self.device) for n in out]
        b = _lib.Buffers(*(t.data_ptr() for t in self.bufs))
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = ctypes.c_void_p()
        check(self.L.lb_init(ctypes.byref(self.p), ctypes.byref(self.hs.c), ctypes.byref(b),
                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.ctx)))
        self.c_lat, self.w_lat = lattice()

    # -- the coupled step ---------------------------------------------------
    def lb_step(self, n=1):
        check(self.L.lb_step(self.ctx, int(n)))

    def ib_spread(self):
        check(self.L.ib_spread(self.ctx))

    def ib_interpolate(self, out=None):
        if out is None:
            out = torch.empty((self.n_nodes, 3), dtype=torch.float32, device=self.device)
        check(self.L.ib_interpolate(self.ctx, ctypes.c_void_p(out.data_ptr())))
        return out

    def checkpoint(self):
        """The context's state as a versioned, checksummed blob (numpy uint8)."""
        n = ctypes.c_size_t()
        check(self.L.lb_checkpoint_size(self.ctx, ctypes.byref(n)))
        blob = np.empty(n.value, dtype=np.uint8)
        check(self.L.lb_checkpoint(self.ctx, blob.ctypes.data_as(ctypes.c_void_p), blob.nbytes))
        return blob

    def restore(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        check(self.L.lb_restore(self.ctx, blob.ctypes.data_as(ctypes.c_void_p), blob.nbytes))

    def swimmer_state_async(self, out):
        """Queue every swimmer's observables into `out` (host memory of at least
        n_swimmers records, e.g. a pinned uint8 tensor, or an array of
        _lib.SwimmerState); valid after sync()."""
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else ctypes.addressof(out)
        check(self.L.swimmer_state_async(self.ctx, ctypes.c_void_p(ptr)))

    def track_async(self, n_steps, out):
        """Queue a copy of the trajectory points of the last n_steps steps into
        `out` (host memory of n_steps x n_swimmers records of 176 bytes, e.g. a
        pinned uint8 tensor); valid after sync()."""
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        check(self.L.lb_track(self.ctx, int(n_steps), ctypes.c_void_p(ptr)))

    def track(self, n_steps):
        """The trajectory points of the last n_steps steps as a structured
        numpy array [n_steps, n_swimmers] (fields step, x_cm, R, V)."""
        out = np.zeros((int(n_steps), self.n_swimmers), dtype=_lib.TRACK_DTYPE)
        if self.n_swimmers:
            self.track_async(n_steps, out)
        else:
            check(self.L.lb_track(self.ctx, int(n_steps), None))
        self.sync()
        return out

    def swimmer_state(self, s=0):
        st = _lib.SwimmerState()
        check(self.L.swimmer_state(self.ctx, int(s), ctypes.byref(st)))
        m = lambda a: np.array([[a[i][j] for j in range(3)] for i in range(3)])
        return dict(step=st.step, R=m(st.R), V=m(st.V), F=m(st.F), T=m(st.T), x_cm=np.array(list(st.x_cm)),
                    disp=np.array(list(st.disp)), periods=st.periods, v_period=np.array(list(st.v_period)),
                    re_swim=st.re_swim, re_bead=st.re_bead)

    def sync(self):
        check(self.L.lb_sync(self.ctx))

    # -- state access ---------------------------------------------------------
    def lb_get_macros(self):
        rho = torch.empty(self.N, dtype=torch.float32, device=self.device)
        u = torch.empty((self.N, 3), dtype=torch.float32, device=self.device)
        check(self.L.lb_get_macros(self.ctx, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(u.data_ptr())))
        return rho, u

    def get_populations(self):
        """Raw f as (19, N) float64 in the library's lattice order."""
        f = np.empty((19, self.N))
        check(self.L.lb_get_populations(self.ctx, f.ctypes.data_as(ctypes.c_void_p)))
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(19, self.N)
        check(self.L.lb_set_populations(self.ctx, f.ctypes.data_as(ctypes.c_void_p)))

    def get_nodes(self):
        r = np.empty((self.n_nodes, 3))
        check(self.L.lb_get_nodes(self.ctx, r.ctypes.data_as(ctypes.c_void_p)))
        return r

    def set_nodes(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(self.n_nodes, 3)
        check(self.L.lb_set_nodes(self.ctx, r.ctypes.data_as(ctypes.c_void_p)))

    def get_node_forces(self):
        f = np.empty((self.n_nodes, 3), dtype=np.float32)
        check(self.L.ib_get_node_forces(self.ctx, f.ctypes.data_as(ctypes.c_void_p)))
        return f

    def get_force_field(self):
        F = np.empty((self.N, 3), dtype=np.float32)
        check(self.L.lb_get_force_field(self.ctx, F.ctypes.data_as(ctypes.c_void_p)))
        return F

    def set_velocity(self, u):
        u = np.ascontiguousarray(u, dtype=np.float32).reshape(self.N, 3)
        check(self.L.lb_set_velocity(self.ctx, u.ctypes.data_as(ctypes.c_void_p)))

    def profile(self, on=True):
        """Bracket every main fluid-kernel launch with CUDA events (lb_profile)."""
        check(self.L.lb_profile(self.ctx, 1 if on else 0))

    def profile_read(self):
        """(total milliseconds, launches) of the fluid kernel since profile(True)."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        check(self.L.lb_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def marked_cells(self):
        """Cells in the tiles marked for the next step (updated with the force field)."""
        n = ctypes.c_longlong()
        check(self.L.lb_marked_cells(self.ctx, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.ctx:
            self.L.lb_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent boxes advanced together by one set of launches per step.

    The simulations keep their own buffers and accessors; while batched they
    are stepped only through the batch."""

    def __init__(self, sims):
        self.L = _lib.load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*(s.ctx.value for s in self.sims))
        self.b = ctypes.c_void_p()
        check(self.L.lb_batch_create(arr, len(self.sims), ctypes.byref(self.b)))

    def lb_step(self, n=1):
        check(self.L.lb_batch_step(self.b, int(n)))

    def profile(self, on=True):
        check(self.L.lb_batch_profile(self.b, 1 if on else 0))

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        check(self.L.lb_batch_profile_read(self.b, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def autotune(self, steps_per_trial=4):
        """Time the launch-shape candidates on real steps and keep the fastest
        (lb_batch_autotune); returns the tuning report as a dict."""
        r = _lib.BatchTuning()
        check(self.L.lb_batch_autotune(self.b, int(steps_per_trial), ctypes.byref(r)))
        n = min(r.n_classes, _lib.TUNE_MAX_CLASSES)
        cands = [c for c in r.marked_candidates if c > 0]
        return {
            "classes": [{"dims": list(r.class_dims[k]), "boxes": r.class_boxes[k],
                         "cells_per_thread": r.class_cells_per_thread[k],
                         "us_by_cells_per_thread": {str(c): r.class_us[k][i] for i, c in enumerate((1, 2, 4))
                                                    if r.class_us[k][i] > 0}} for k in range(n)],
            "marked_blocks": r.marked_blocks,
            "marked_step_us": {str(c): r.marked_step_us[i] for i, c in enumerate(cands)},
            "steps_taken": r.steps_taken,
        }

    def close(self):
        if self.b:
            self.L.lb_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
