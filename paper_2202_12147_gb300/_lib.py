"""ctypes mirror of include/lbib.h.  Argument marshalling only: every step of
the coupled update runs inside liblbib.so.  There is no fallback; if the
library cannot be loaded the import of a caller fails loudly."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

LBIB_OK, LBIB_EINVAL, LBIB_ECUDA, LBIB_ENONFINITE, LBIB_EUNSTABLE, LBIB_ETIMEOUT, LBIB_ESIZE = 0, -1, -2, -3, -4, -5, -6
F32, F16, BF16, F64 = 0, 1, 2, 3
NEOHOOKE, SKALAK = 0, 1
GUO, SHAN_CHEN = 0, 1
PESKIN4, LINEAR2 = 0, 1
NBUF = 3

EXPORTS = [
    "lbib_version", "lbib_strerror", "lbib_last_error", "lbib_lattice", "lbib_required_sizes", "lb_init", "lb_step",
    "ib_spread", "ib_interpolate", "swimmer_state", "lb_sync", "lb_get_macros", "lb_get_populations",
    "lb_set_populations", "lb_get_nodes", "lb_set_nodes", "ib_get_node_forces", "lb_get_force_field",
    "lb_set_velocity", "lb_profile", "lb_profile_read", "lb_marked_cells", "ib_spread_fixed_noalloc",
    "lb_batch_create", "lb_batch_step", "lb_batch_profile", "lb_batch_profile_read", "lb_batch_destroy",
    "lb_destroy", "lb_adjoint_required_bytes", "lb_adjoint_create", "lb_adjoint_set_drive",
    "lb_adjoint_set_initial", "lb_adjoint_forward", "lb_adjoint_backward", "lb_adjoint_get_final",
    "lb_adjoint_timing", "lb_adjoint_destroy", "lb_batch_autotune", "swimmer_state_async",
    "lb_checkpoint_size", "lb_checkpoint", "lb_restore", "lb_track",
]


class LbParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("storage", ctypes.c_int), ("forcing", ctypes.c_int),
                ("kernel", ctypes.c_int), ("deterministic", ctypes.c_int), ("g", ctypes.c_double * 3),
                ("store_scale", ctypes.c_double)]


class Bead(ctypes.Structure):
    _fields_ = [("node_start", ctypes.c_int), ("node_count", ctypes.c_int), ("tri_start", ctypes.c_int),
                ("tri_count", ctypes.c_int), ("Gs", ctypes.c_double), ("law", ctypes.c_int), ("C", ctypes.c_double),
                ("kb", ctypes.c_double), ("kv", ctypes.c_double)]


class Swimmer(ctypes.Structure):
    _fields_ = [("bead", ctypes.c_int * 3), ("k_spring", ctypes.c_double), ("L_spring", ctypes.c_double),
                ("amp", ctypes.c_double * 3), ("phase", ctypes.c_double * 3), ("balance", ctypes.c_int),
                ("period", ctypes.c_double)]


class Structure(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int), ("n_swimmers", ctypes.c_int), ("n_nodes", ctypes.c_int),
                ("n_tris", ctypes.c_int), ("beads", ctypes.POINTER(Bead)), ("swimmers", ctypes.POINTER(Swimmer)),
                ("rest_nodes", ctypes.c_void_p), ("tris", ctypes.c_void_p)]


class Buffers(ctypes.Structure):
    _fields_ = [("pops", ctypes.c_void_p), ("fields", ctypes.c_void_p), ("aux", ctypes.c_void_p)]


class SwimmerState(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("R", (ctypes.c_double * 3) * 3), ("V", (ctypes.c_double * 3) * 3),
                ("F", (ctypes.c_double * 3) * 3), ("T", (ctypes.c_double * 3) * 3), ("x_cm", ctypes.c_double * 3),
                ("disp", ctypes.c_double * 3), ("periods", ctypes.c_longlong), ("v_period", ctypes.c_double * 3),
                ("re_swim", ctypes.c_double), ("re_bead", ctypes.c_double)]


TRACK_STEPS = 256


class TrackPoint(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("x_cm", ctypes.c_double * 3), ("R", (ctypes.c_double * 3) * 3),
                ("V", (ctypes.c_double * 3) * 3)]


# the same record as a numpy dtype (176 bytes)
TRACK_DTYPE = [("step", "<i8"), ("x_cm", "<f8", (3,)), ("R", "<f8", (3, 3)), ("V", "<f8", (3, 3))]

TUNE_MAX_CLASSES = 32


class BatchTuning(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int), ("class_dims", (ctypes.c_int * 3) * TUNE_MAX_CLASSES),
                ("class_boxes", ctypes.c_int * TUNE_MAX_CLASSES),
                ("class_cells_per_thread", ctypes.c_int * TUNE_MAX_CLASSES),
                ("class_us", (ctypes.c_double * 3) * TUNE_MAX_CLASSES), ("marked_candidates", ctypes.c_int * 4),
                ("marked_step_us", ctypes.c_double * 4), ("marked_blocks", ctypes.c_int),
                ("steps_taken", ctypes.c_longlong)]


class LbibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbib error {code}: {msg}")
        self.code = code


def library_path():
    """liblbib.so in the package directory, or the build named by the
    LBIB_LIBRARY environment variable (used to compare build variants)."""
    return os.environ.get("LBIB_LIBRARY") or _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbib.so (building it in-tree with nvcc when it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing or path != _build.LIB:
                raise OSError(f"{path} missing: run paper_2202_12147_gb300.build.build()")
            _build.build()
        L = ctypes.CDLL(path)
        P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        L.lbib_version.restype = ctypes.c_char_p
        L.lbib_strerror.restype = ctypes.c_char_p
        L.lbib_strerror.argtypes = [I]
        L.lbib_last_error.restype = ctypes.c_char_p
        L.lbib_lattice.argtypes = [P, P]
        L.lbib_required_sizes.argtypes = [ctypes.POINTER(LbParams), ctypes.POINTER(Structure), P]
        L.lb_init.argtypes = [ctypes.POINTER(LbParams), ctypes.POINTER(Structure), ctypes.POINTER(Buffers), P,
                              ctypes.POINTER(P)]
        L.lb_step.argtypes = [P, LL]
        L.ib_spread.argtypes = [P]
        L.ib_interpolate.argtypes = [P, P]
        L.swimmer_state.argtypes = [P, I, ctypes.POINTER(SwimmerState)]
        L.swimmer_state_async.argtypes = [P, P]
        L.lb_track.argtypes = [P, ctypes.c_longlong, P]
        L.lb_checkpoint_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.lb_checkpoint.argtypes = [P, P, ctypes.c_size_t]
        L.lb_restore.argtypes = [P, P, ctypes.c_size_t]
        L.lb_sync.argtypes = [P]
        L.lb_get_macros.argtypes = [P, P, P]
        for n in ("lb_get_populations", "lb_set_populations", "lb_get_nodes", "lb_set_nodes", "ib_get_node_forces",
                  "lb_get_force_field", "lb_set_velocity"):
            getattr(L, n).argtypes = [P, P]
        L.lb_profile.argtypes = [P, I]
        L.lb_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(LL)]
        L.lb_marked_cells.argtypes = [P, ctypes.POINTER(LL)]
        L.ib_spread_fixed_noalloc.argtypes = [P, P, I, I, I, I, I, P, P]
        L.lb_batch_create.argtypes = [P, I, ctypes.POINTER(P)]
        L.lb_batch_step.argtypes = [P, LL]
        L.lb_batch_profile.argtypes = [P, I]
        L.lb_batch_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(LL)]
        L.lb_batch_destroy.argtypes = [P]
        L.lb_batch_autotune.argtypes = [P, I, ctypes.POINTER(BatchTuning)]
        L.lb_destroy.argtypes = [P]
        L.lb_adjoint_required_bytes.argtypes = [ctypes.POINTER(LbParams), ctypes.POINTER(Structure), LL, I, P]
        L.lb_adjoint_create.argtypes = [ctypes.POINTER(LbParams), ctypes.POINTER(Structure), LL, I, P,
                                        ctypes.c_size_t, P, ctypes.POINTER(P)]
        L.lb_adjoint_set_drive.argtypes = [P, P]
        L.lb_adjoint_set_initial.argtypes = [P, P, P]
        L.lb_adjoint_forward.argtypes = [P, P]
        L.lb_adjoint_backward.argtypes = [P, P, P, P, P, P, P]
        L.lb_adjoint_get_final.argtypes = [P, P, P]
        L.lb_adjoint_timing.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(LL), ctypes.POINTER(LL)]
        L.lb_adjoint_destroy.argtypes = [P]
        for n in EXPORTS:
            if n not in ("lbib_version", "lbib_strerror", "lbib_last_error"):
                getattr(L, n).restype = I
        _lib = L
        return L


def check(code):
    if code != LBIB_OK:
        L = load()
        raise LbibError(code, L.lbib_last_error().decode())
    return code
