"""Seeded synthetic workloads: periodic boxes with three-bead swimmers.

Input generators only.  Nothing here evaluates the time step; the oracle and
the CUDA path both consume the plain arrays that `assemble` returns.

Conventions (readings of a paper that leaves them open):
  * lattice nodes sit at integer coordinates 0..N-1 of a periodic box; x is
    the swimming axis (Sec. 2.2 drives the beads along x);
  * a swimmer is three equal icosphere beads on the x axis whose centres are
    `spacing` apart; the middle bead sits at `center` (Sec. 2.2, Fig. 1);
  * the drive on bead b is amp[b] * sin(2 pi t / T + phase[b]) along x; with
    `balance` the middle bead instead carries minus the sum of the outer two,
    which is the paper's protocol f1 = A sin(wt), f3 = B sin(wt + alpha),
    f2 = -f1 - f3 (Sec. 2.2, driving-force equation);
  * "separation of n bead radii" between two swimmers is the surface gap
    between their nearest beads, n * a (in-line: centre-bead distance
    2*spacing + 2a + gap; side by side along y: 2a + gap), placed
    symmetrically about the box centre.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

from .mesh import icosphere


@dataclass(frozen=True)
class SwimmerSpec:
    center: tuple
    radius: float = 4.0
    subdiv: int = 2
    spacing: float = 12.0
    k_spring: float = 0.005
    Gs: float = 0.01
    amp: tuple = (1e-3, 0.0, 1e-3)
    phase: tuple = (0.0, 0.0, math.pi / 2)
    balance: bool = True
    period: float = 500.0
    # membrane law of the beads (Sec. 2.2): "neohooke" (shear modulus Gs) or
    # "skalak" (Gs is then kappa_s, and C the area-dilatation parameter,
    # kappa_a / kappa_s = 1 + 2 C); bending modulus kb of the Helfrich energy
    # and volume-penalty modulus kv (Eq. vol_cons); zero switches a term off
    law: str = "neohooke"
    C: float = 0.0
    kb: float = 0.0
    kv: float = 0.0

    def with_drive(self, A, B, alpha):
        """The paper's protocol: f1 = A sin(wt), f3 = B sin(wt+alpha), f2 = -f1-f3."""
        return replace(self, amp=(A, 0.0, B), phase=(0.0, 0.0, alpha), balance=True)

    def with_paper_membrane(self):
        """The paper's bead membrane (Sec. 3): Skalak law with kappa_s = 5e-2
        and kappa_a = 1 (C = (kappa_a / kappa_s - 1) / 2 = 9.5), bending
        modulus 1.25e-3, volume penalty kappa_v = 1."""
        return replace(self, law="skalak", Gs=5e-2, C=9.5, kb=1.25e-3, kv=1.0)


@dataclass(frozen=True)
class BoxSpec:
    dims: tuple  # (nx, ny, nz), x fastest in memory
    tau: float = 1.0
    rho0: float = 1.0
    swimmers: tuple = field(default_factory=tuple)
    forcing: str = "guo"        # "guo" | "shan_chen"
    kernel: str = "peskin4"     # "peskin4" | "linear2"
    g: tuple = (0.0, 0.0, 0.0)  # uniform body-force density (test flows)
    name: str = ""

    @property
    def n_cells(self):
        nx, ny, nz = self.dims
        return nx * ny * nz


def assemble(box: BoxSpec):
    """Flatten a box into plain arrays.

    Returns a dict:
      nodes   (M,3) float64  initial node positions (= membrane rest shape)
      tris    (T,3) int32    global node ids, outward orientation
      beads   (B,4) int32    node_start, node_count, tri_start, tri_count
      bead_Gs (B,)  float64  neo-Hookean shear modulus (Skalak: kappa_s) per bead
      bead_law (B,) int32    0 neo-Hookean, 1 Skalak
      bead_C, bead_kb, bead_kv (B,) float64  Skalak C, bending and volume moduli
      swimmers list of dicts: beads (3 ids), k, L, amp, phase, balance, period
    """
    nodes, tris, beads, gs, sw = [], [], [], [], []
    law, cc, kb, kv = [], [], [], []
    m0 = 0
    t0 = 0
    cache = {}
    for s in box.swimmers:
        if s.subdiv not in cache:
            cache[s.subdiv] = icosphere(s.subdiv)
        unit, utris = cache[s.subdiv]
        ids = []
        for b in range(3):
            c = np.array(s.center, dtype=np.float64) + np.array([(b - 1) * s.spacing, 0.0, 0.0])
            nodes.append(unit * s.radius + c)
            tris.append(utris + m0)
            beads.append((m0, len(unit), t0, len(utris)))
            gs.append(s.Gs)
            if s.law not in ("neohooke", "skalak"):
                raise ValueError(f"unknown membrane law {s.law}")
            law.append(1 if s.law == "skalak" else 0)
            cc.append(s.C)
            kb.append(s.kb)
            kv.append(s.kv)
            ids.append(len(beads) - 1)
            m0 += len(unit)
            t0 += len(utris)
        sw.append(dict(beads=ids, k=s.k_spring, L=s.spacing, amp=tuple(s.amp),
                       phase=tuple(s.phase), balance=bool(s.balance), period=float(s.period),
                       radius=float(s.radius)))
    if nodes:
        nodes = np.concatenate(nodes)
        tris = np.concatenate(tris).astype(np.int32)
    else:
        nodes = np.zeros((0, 3))
        tris = np.zeros((0, 3), dtype=np.int32)
    return dict(nodes=nodes, tris=tris, beads=np.array(beads, dtype=np.int32).reshape(-1, 4),
                bead_Gs=np.array(gs, dtype=np.float64), bead_law=np.array(law, dtype=np.int32),
                bead_C=np.array(cc, dtype=np.float64), bead_kb=np.array(kb, dtype=np.float64),
                bead_kv=np.array(kv, dtype=np.float64), swimmers=sw)


# ----------------------------------------------------------------------------
# The workloads.  Sizes follow the three-bead swimmer problem of Sec. 3 scaled
# to boxes that one GPU steps thousands of times per second.
# ----------------------------------------------------------------------------

def single_swimmer_48(period=500.0, alpha=math.pi / 2, A=1e-3, B=1e-3, dims=(48, 48, 48)):
    """One swimmer, D3Q19 tau=1 rho0=1, periodic 48^3; beads of radius 4 at
    subdivision 2 (162 nodes, 320 triangles), spacing 12, k=0.005, Gs=0.01,
    drive amplitude 1e-3, period 500 steps, phase shift pi/2."""
    c = tuple(float(d // 2) for d in dims)
    s = SwimmerSpec(center=c, radius=4.0, subdiv=2, spacing=12.0, k_spring=0.005, Gs=0.01,
                    period=period).with_drive(A, B, alpha)
    return BoxSpec(dims=dims, swimmers=(s,), name="single_swimmer_48")


def _pair_swimmer(center, period):
    return SwimmerSpec(center=center, radius=6.0, subdiv=3, spacing=18.0, k_spring=0.005,
                       Gs=0.01, period=period).with_drive(1e-3, 1e-3, math.pi / 2)


def swimmer_pair(arrangement: str, gap_radii: int, dims=(256, 128, 128), period=2000.0):
    """Two swimmers (radius 6, subdivision 3 = 642 nodes, spacing 18, k=0.005,
    drive 1e-3, period 2000) in-line along x or side by side along y, with a
    surface gap of `gap_radii` bead radii, placed symmetrically about the box
    centre."""
    a, L = 6.0, 18.0
    gap = gap_radii * a
    cx, cy, cz = (float(d // 2) for d in dims)
    if arrangement == "inline":
        h = (2 * L + 2 * a + gap) / 2.0
        centers = ((cx - h, cy, cz), (cx + h, cy, cz))
    elif arrangement == "side":
        h = (2 * a + gap) / 2.0
        centers = ((cx, cy - h, cz), (cx, cy + h, cz))
    else:
        raise ValueError(arrangement)
    sw = tuple(_pair_swimmer(c, period) for c in centers)
    return BoxSpec(dims=dims, swimmers=sw, name=f"pair_{arrangement}_{gap_radii}a_{dims[0]}x{dims[1]}x{dims[2]}")


PAIR_CASES = [(arr, n) for arr in ("inline", "side") for n in (3, 5, 8)]


def pair_boxes_256x128x128():
    """The six two-swimmer boxes: in-line and side-by-side at gaps 3, 5, 8 radii."""
    return [swimmer_pair(arr, n) for arr, n in PAIR_CASES]


def pair_side_256cube():
    """Precision workload: 256^3 with two side-by-side swimmers, gap 3 radii."""
    return swimmer_pair("side", 3, dims=(256, 256, 256))


def paper_box_1024x256x256(period=20000.0):
    """The paper's simulation box (Sec. 3): 1024 x 256 x 256 cells, with two
    swimmers of bead radius 5 and spring length 36 (subdivision 3 = 642
    nodes per bead, k = 0.005, drive 1e-3, alpha = pi/2, period 2e4 steps)
    in line along x, their centres two swimmer lengths apart (the paper's
    closest in-line case), placed symmetrically about the box centre."""
    a, L = 5.0, 36.0
    l_swim = 2 * L + 2 * a
    dims = (1024, 256, 256)
    cx, cy, cz = (float(d // 2) for d in dims)
    sw = tuple(SwimmerSpec(center=(cx + s * l_swim, cy, cz), radius=a, subdiv=3, spacing=L, k_spring=0.005, Gs=0.01,
                           period=period).with_drive(1e-3, 1e-3, math.pi / 2) for s in (-1.0, 1.0))
    return BoxSpec(dims=dims, swimmers=sw, name="paper_inline_2L_1024x256x256")


# The paper's own set-up (Sec. 3): bead radius 5, springs of rest length 36 and
# stiffness 2e-2, drive period 2e4 steps, phase shift pi/2, the Skalak /
# bending / volume membrane and Shan-Chen forcing.  The paper's 2-point delta
# kernel (Sec. 2.3) with this membrane (kappa_a = 1) makes the explicit
# coupling unstable here (non-finite within 75 steps, in the oracle as on the
# GPU), so the 4-point kernel is used.  The printed amplitudes (A = 1e-1, B = 5e-3) are read as
# A = B = 5e-3: with A = 1e-1 the fastest bead would reach Re_bead ~ 0.4,
# against the ~1e-2 the paper states (Sec. 3), which A = 5e-3 gives.  The
# swimmer length is taken as 2 L_spring = 72, the approximation of Sec. 3.
PAPER_L_SWIM = 72.0


def _paper_swimmer(center, period=20000.0, A=5e-3):
    return SwimmerSpec(center=center, radius=5.0, subdiv=3, spacing=36.0, k_spring=2e-2, period=period).with_drive(
        A, A, math.pi / 2).with_paper_membrane()


def paper_study_box(case, dims=(1024, 256, 256), period=20000.0, tau=1.0):
    """The paper's 1024 x 256 x 256 box (Sec. 3) with: "lone" one swimmer
    at the centre; "inline_<n>" two swimmers on the x axis whose centres are
    n swimmer lengths apart; "side_<n>" two swimmers side by side along y, n
    swimmer lengths apart; placed symmetrically about the box centre.  tau
    sets the viscosity, mu = rho0 (tau - 1/2) / 3 (1/6 at tau = 1)."""
    cx, cy, cz = (float(d // 2) for d in dims)
    if case == "lone":
        sw = (_paper_swimmer((cx, cy, cz), period),)
    else:
        arr, n = case.split("_")
        h = float(n) * PAPER_L_SWIM / 2.0
        if arr == "inline":
            sw = tuple(_paper_swimmer((cx + s * h, cy, cz), period) for s in (-1.0, 1.0))
        elif arr == "side":
            sw = tuple(_paper_swimmer((cx, cy + s * h, cz), period) for s in (-1.0, 1.0))
        else:
            raise ValueError(case)
    return BoxSpec(dims=dims, swimmers=sw, tau=tau, forcing="shan_chen", kernel="peskin4", name=f"paper_{case}")


def balanced_drive(A=1e-3, B=1e-3, alpha=math.pi / 2):
    """Per-bead drive (A1, A2, A3, phi1, phi2, phi3) whose middle bead carries
    minus the sum of the outer two: f1 + f3 = A sin(wt) + B sin(wt + alpha)
    = C sin(wt + beta) with C = sqrt(A^2 + B^2 + 2AB cos alpha) and
    beta = atan2(B sin alpha, A + B cos alpha), so f2 = C sin(wt + beta + pi).
    For A = B = 1e-3, alpha = pi/2: A2 = sqrt(2) 1e-3, phi2 = 5 pi/4."""
    C = math.sqrt(A * A + B * B + 2.0 * A * B * math.cos(alpha))
    beta = math.atan2(B * math.sin(alpha), A + B * math.cos(alpha))
    return (A, C, B, 0.0, beta + math.pi, alpha)


def free_drive(spec: SwimmerSpec, theta):
    """The swimmer with independent per-bead drives theta = (A1, A2, A3, phi1, phi2, phi3)."""
    return replace(spec, amp=tuple(float(v) for v in theta[:3]), phase=tuple(float(v) for v in theta[3:6]),
                   balance=False)


def adjoint_single_96(period=1000.0):
    """Single swimmer (radius 6, subdivision 3, spacing 18) in 96^3, period
    1000, with independent per-bead drives at the base point that reproduces
    the paper's protocol (A = B = 1e-3, alpha = pi/2, see `balanced_drive`)."""
    s = free_drive(_pair_swimmer((48.0, 48.0, 48.0), period), balanced_drive())
    return BoxSpec(dims=(96, 96, 96), swimmers=(s,), name="adjoint_single_96")


def adjoint_small(dims=(32, 24, 24), period=100.0):
    """Small adjoint test box: one swimmer of radius 3 (subdivision 1, 42
    nodes per bead), spacing 9, period 100, free per-bead drives at the
    balanced base point."""
    c = tuple(float(d // 2) for d in dims)
    s = SwimmerSpec(center=c, radius=3.0, subdiv=1, spacing=9.0, k_spring=0.005, Gs=0.01, period=period)
    return BoxSpec(dims=dims, swimmers=(free_drive(s, balanced_drive()),), name=f"adjoint_small_{dims[0]}x{dims[1]}x{dims[2]}")


def fluid_box(dims, tau=1.0, g=(0.0, 0.0, 0.0), forcing="guo"):
    return BoxSpec(dims=dims, tau=tau, g=tuple(g), forcing=forcing, name=f"fluid_{dims}")


# ----------------------------------------------------------------------------
# Seeded random state for parity tests
# ----------------------------------------------------------------------------

def random_populations(n_cells, weights, seed=0, rho_amp=1e-3, u_amp=1e-3):
    """Raw populations f_i = w_i (rho0 + noise) with small seeded noise, as an
    (n_cells, 19) float64 array in the order of `weights`.  Each side maps
    the columns to its own lattice order by velocity vector."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=np.float64)
    noise = rng.uniform(-1.0, 1.0, size=(n_cells, len(w)))
    return w[None, :] * (1.0 + rho_amp * noise) + u_amp * w[None, :] * rng.uniform(-1, 1, size=(n_cells, 1))


def perturbed_nodes(nodes, seed=0, amp=0.05):
    rng = np.random.default_rng(seed)
    return nodes + amp * rng.uniform(-1.0, 1.0, size=nodes.shape)


ENSEMBLE_SIZES = [(48, 48, 48), (64, 64, 64), (96, 96, 96), (192, 128, 128)]


def ensemble_boxes(n=64, seed=0, period=2000.0):
    """Independent boxes for batched runs, drawn with numpy default_rng(seed):
    sizes uniformly from 48^3, 64^3, 96^3 and 128x128x192 (stored with the
    long side along x); one or two swimmers (radius 6 at subdivision 3,
    spacing 18) with drive amplitude A = B drawn from [5e-4, 2e-3], phase
    shift from [pi/4, 3pi/4], pairs in-line or side by side with a surface
    gap of 2-8 radii.  Fit rules: a 48^3 box holds one smaller swimmer
    (radius 4, subdivision 2, spacing 12); every swimmer keeps a clearance of
    two radii to the periodic images, so an in-line pair that does not fit
    becomes side by side, a side-by-side gap is clamped to fit, and a pair
    that still does not fit keeps one swimmer."""
    rng = np.random.default_rng(seed)
    boxes = []
    for b in range(n):
        dims = ENSEMBLE_SIZES[int(rng.integers(len(ENSEMBLE_SIZES)))]
        n_sw = 1 + int(rng.integers(2))
        arr = "inline" if rng.random() < 0.5 else "side"
        gap_r = float(rng.uniform(2.0, 8.0))
        alpha = float(rng.uniform(math.pi / 4, 3 * math.pi / 4))
        amp = float(rng.uniform(5e-4, 2e-3))
        nx, ny, nz = dims
        cx, cy, cz = (float(d // 2) for d in dims)
        if dims == (48, 48, 48):
            a, L, sub, n_sw = 4.0, 12.0, 2, 1
        else:
            a, L, sub = 6.0, 18.0, 3
        gap = gap_r * a
        ext = 2 * L + 2 * a
        clear = 2 * a
        if n_sw == 2 and arr == "inline" and 2 * ext + gap + clear > nx:
            arr = "side"
        if n_sw == 2 and arr == "side" and 4 * a + gap + clear > ny:
            gap = ny - 4 * a - clear
            if gap < 2 * a:
                n_sw = 1
        spec = dict(radius=a, subdiv=sub, spacing=L, k_spring=0.005, Gs=0.01, period=period)
        if n_sw == 1:
            sw = (SwimmerSpec(center=(cx, cy, cz), **spec).with_drive(amp, amp, alpha),)
        elif arr == "inline":
            h = (ext + gap) / 2.0
            sw = tuple(SwimmerSpec(center=(cx + s * h, cy, cz), **spec).with_drive(amp, amp, alpha) for s in (-1, 1))
        else:
            h = (2 * a + gap) / 2.0
            sw = tuple(SwimmerSpec(center=(cx, cy + s * h, cz), **spec).with_drive(amp, amp, alpha) for s in (-1, 1))
        boxes.append(BoxSpec(dims=dims, swimmers=sw, name=f"ensemble_{b}_{nx}x{ny}x{nz}_{len(sw)}sw"))
    return boxes
