"""The C-ABI library builds, loads and exports every function the header
declares; argument errors are reported before any launch.  CPU only (no
call here touches a device)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbib.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("LBIB")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lb_init", "lb_step", "ib_interpolate", "ib_spread", "swimmer_state", "lb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2202_12147_gb300 import _lib
    L = _lib.load()
    for n in _declared():
        assert hasattr(L, n), n
    assert set(_lib.EXPORTS) == set(_declared())


def test_lattice_and_sizes_without_gpu():
    from paper_2202_12147_gb300 import lattice, required_sizes
    from workloads import assemble, single_swimmer_48
    c, w = lattice()
    assert w.sum() == pytest.approx(1.0)
    for i in range(1, 19, 2):  # opposite directions adjacent
        assert (c[i] == -c[i + 1]).all()
    s0 = required_sizes((48, 48, 48))
    s1 = required_sizes((48, 48, 48), assemble(single_swimmer_48()))
    assert s0[0] == 19 * 48 ** 3 * 4
    assert s1[2] > s0[2]
    s16 = required_sizes((48, 48, 48), storage="f16")
    assert s16[0] == 19 * 48 ** 3 * 2
    assert all(v % 256 == 0 for v in s1)


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(rho0=0.0), dict(storage="f8"), dict(dims=(0, 4, 4))])
def test_invalid_arguments_rejected(bad):
    from paper_2202_12147_gb300 import _lib, required_sizes
    kw = dict(tau=1.0, rho0=1.0, storage="f32")
    dims = bad.pop("dims", (8, 8, 8))
    kw.update(bad)
    with pytest.raises((_lib.LbibError, KeyError)):
        required_sizes(dims, **kw)


def test_structure_validation():
    import numpy as np
    from paper_2202_12147_gb300 import _lib, required_sizes
    from workloads import assemble, single_swimmer_48
    a = assemble(single_swimmer_48())
    a["tris"] = a["tris"].copy()
    a["tris"][0, 0] = 200  # node of another bead
    with pytest.raises(_lib.LbibError, match="outside its bead"):
        required_sizes((48, 48, 48), a)
    a = assemble(single_swimmer_48())
    a["nodes"] = a["nodes"].copy()
    a["nodes"][3, 1] = np.nan
    with pytest.raises(_lib.LbibError, match="non-finite"):
        required_sizes((48, 48, 48), a)


def _adjoint_bytes(dims, structure, n_steps, K, storage=3, forcing=0, kernel=0):
    from paper_2202_12147_gb300 import _lib
    from paper_2202_12147_gb300.sim import _HostStructure
    L = _lib.load()
    p = _lib.LbParams()
    p.nx, p.ny, p.nz = dims
    p.tau, p.rho0 = 1.0, 1.0
    p.storage, p.forcing, p.kernel = storage, forcing, kernel
    hs = _HostStructure(structure)
    out = ctypes.c_size_t()
    _lib.check(L.lb_adjoint_required_bytes(ctypes.byref(p), ctypes.byref(hs.c), n_steps, K, ctypes.byref(out)))
    return out.value


def test_adjoint_workspace_sizes_without_gpu():
    """Checkpoint-and-recompute memory: two sets of K + 1 step records (the
    reverse sweep of one segment runs beside the recompute of the one before
    it) plus one checkpoint per segment (and the final state), not one record
    per step."""
    from workloads import adjoint_single_96, assemble
    box = adjoint_single_96()
    asm = assemble(box)
    n = 96 ** 3
    b64 = _adjoint_bytes(box.dims, asm, 1000, 100)
    b32 = _adjoint_bytes(box.dims, asm, 1000, 100, storage=0)
    rec64 = 25 * n * 8       # populations, F and u of one step, FP64
    ck64 = 19 * n * 8
    assert 202 * rec64 + 11 * ck64 < b64 < 202 * rec64 + 11 * ck64 + 2 * 19 * n * 8 + 8 * n * 8 + (64 << 20)
    assert b32 < 0.55 * b64
    # ten periods cost ten more checkpoints, not ten times the records
    b10 = _adjoint_bytes(box.dims, asm, 10000, 100)
    assert b10 - b64 == pytest.approx(90 * ck64, rel=0.01)


@pytest.mark.parametrize("bad", [dict(storage=1), dict(storage=0, forcing=1), dict(kernel=1), dict(K=0),
                                 dict(n_steps=0)])
def test_adjoint_invalid_arguments_rejected(bad):
    from paper_2202_12147_gb300 import _lib
    from workloads import adjoint_small, assemble
    box = adjoint_small()
    kw = dict(n_steps=10, K=5)
    kw.update(bad)
    with pytest.raises(_lib.LbibError):
        _adjoint_bytes(box.dims, assemble(box), **kw)


def test_membrane_model_sizes_and_validation():
    """The paper's membrane (Skalak, bending, volume penalty) adds bending
    edges (3/2 per triangle of a closed bead) and volume data to the
    auxiliary buffer; bending on an open surface, an unknown law and
    negative moduli are rejected before anything is allocated."""
    import math
    from paper_2202_12147_gb300 import _lib, required_sizes
    from workloads import BoxSpec, SwimmerSpec, assemble
    sw = SwimmerSpec(center=(16.0, 12.0, 12.0), radius=3.0, subdiv=1, spacing=9.0).with_drive(1e-3, 1e-3, math.pi / 2)
    plain = assemble(BoxSpec(dims=(32, 24, 24), swimmers=(sw,)))
    paper = assemble(BoxSpec(dims=(32, 24, 24), swimmers=(sw.with_paper_membrane(),)))
    assert list(paper["bead_law"]) == [1, 1, 1] and paper["bead_kb"][0] == 1.25e-3 and paper["bead_kv"][0] == 1.0
    s0 = required_sizes((32, 24, 24), plain)
    s1 = required_sizes((32, 24, 24), paper)
    assert s1[2] > s0[2] and s1[:2] == s0[:2]
    bad = dict(paper)
    bad["tris"] = paper["tris"][1:]  # one triangle missing: open surface
    bad["beads"] = paper["beads"].copy()
    bad["beads"][0, 3] -= 1
    bad["beads"][1:, 2] -= 1
    with pytest.raises(_lib.LbibError):
        required_sizes((32, 24, 24), bad)
    for key, val in (("bead_law", np.array([2, 1, 1], np.int32)), ("bead_kb", np.array([-1.0, 0.0, 0.0])),
                     ("bead_kv", np.array([np.nan, 0.0, 0.0]))):
        st = dict(paper)
        st[key] = val
        with pytest.raises(_lib.LbibError):
            required_sizes((32, 24, 24), st)


def test_paper_study_workloads():
    """The paper-scale study boxes (Sec. 3): 1024 x 256 x 256, swimmers of
    radius 5 with springs of length 36 (swimmer length 72), the paper's
    membrane, Shan-Chen forcing; pairs placed symmetrically about the centre
    n swimmer lengths apart, in line along x or side by side along y; the
    viscosity set by tau.  Every structure passes the library's validation."""
    from paper_2202_12147_gb300 import required_sizes
    from workloads import PAPER_L_SWIM, assemble, paper_study_box
    assert PAPER_L_SWIM == 72
    for case, axis, n in (("lone", None, 0), ("inline_2", 0, 2.0), ("side_1.5", 1, 1.5)):
        box = paper_study_box(case, tau=2.0)
        assert box.dims == (1024, 256, 256) and box.tau == 2.0 and box.forcing == "shan_chen"
        sw = box.swimmers
        assert all(s.radius == 5.0 and s.spacing == 36.0 and s.law == "skalak" for s in sw)
        if axis is None:
            assert len(sw) == 1 and sw[0].center == (512.0, 128.0, 128.0)
        else:
            c = np.array([s.center for s in sw])
            assert np.allclose(c.mean(axis=0), (512.0, 128.0, 128.0))
            sep = c[1] - c[0]
            assert sep[axis] == n * PAPER_L_SWIM and np.count_nonzero(sep) == 1
        sizes = required_sizes(box.dims, assemble(box), tau=box.tau, forcing=box.forcing)
        assert sizes[0] == 19 * 1024 * 256 * 256 * 4
