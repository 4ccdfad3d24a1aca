"""Failure detection and recovery, with the failures made on the host (no
device fault, trap or hang): a non-finite population written through
lb_set_populations, and a flow fast enough that the nodes outrun the
stability bound.  The kernels latch the condition in device memory, the next
synchronising call reports it, and restoring the checkpoint taken before the
failure continues the run as if nothing had happened."""
import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_sim, lattice_perm
from workloads import BoxSpec, SwimmerSpec, assemble

pytestmark = pytest.mark.gpu


def _box():
    sw = SwimmerSpec(center=(20.0, 12.0, 12.0), radius=3.0, subdiv=1, spacing=9.0, period=40.0).with_drive(
        1e-3, 1e-3, 1.2)
    return BoxSpec(dims=(40, 24, 24), swimmers=(sw,))


def test_non_finite_population_is_reported_and_restore_recovers(gpu_lib):
    from paper_2202_12147_gb300 import _lib
    from paper_2202_12147_gb300._lib import LbibError
    box = _box()
    asm = assemble(box)
    ref = gpu_sim(box, asm, deterministic=True)
    ref.lb_step(15)
    f_ref = ref.get_populations()
    ref.close()
    sim = gpu_sim(box, asm, deterministic=True)
    sim.lb_step(10)
    blob = sim.checkpoint()
    f = sim.get_populations()
    f[4, 1234] = np.nan
    sim.set_populations(f)
    sim.lb_step(3)
    with pytest.raises(LbibError) as e:
        sim.sync()
    assert e.value.code == _lib.LBIB_ENONFINITE
    with pytest.raises(LbibError):
        sim.checkpoint()  # a failed run is not saved
    sim.restore(blob)
    sim.sync()  # the restored control block carries no error
    sim.lb_step(5)
    assert np.array_equal(sim.get_populations(), f_ref)
    sim.close()


def test_fast_flow_trips_the_stability_bound(gpu_lib):
    """Equilibrium populations of a uniform flow of 0.3 lattice units per step
    carry the nodes faster than the 0.1 bound the interpolation checks."""
    from paper_2202_12147_gb300 import _lib, lattice
    from paper_2202_12147_gb300._lib import LbibError
    box = _box()
    sim = gpu_sim(box, assemble(box))
    c, w = lattice()
    feq = oracle.equilibrium(1.0, [0.3, 0.0, 0.0])
    perm = lattice_perm()
    f = np.repeat(feq[perm][:, None], box.n_cells, axis=1)
    sim.set_populations(f)
    sim.lb_step(2)
    with pytest.raises(LbibError) as e:
        sim.sync()
    assert e.value.code == _lib.LBIB_EUNSTABLE
    sim.close()
