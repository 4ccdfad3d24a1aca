"""Shared helpers of the GPU parity tests: lattice-order mapping between the
oracle and the CUDA library, and construction of both sides from one
workload."""
import numpy as np


def lattice_perm():
    """perm[i_gpu] = index of the same velocity in the oracle's order."""
    import oracle
    from paper_2202_12147_gb300 import lattice
    cg, wg = lattice()
    co, wo = oracle.lattice()
    perm = np.array([next(k for k in range(19) if (co[k] == cg[i]).all()) for i in range(19)])
    assert np.allclose(wo[perm], wg)
    return perm


def gpu_sim(box, asm=None, **kw):
    from paper_2202_12147_gb300 import Simulation
    from workloads import assemble
    asm = assemble(box) if asm is None else asm
    return Simulation(box.dims, asm, tau=box.tau, rho0=box.rho0, forcing=box.forcing, kernel=box.kernel, g=box.g, **kw)


def gpu_f_to_oracle(f_gpu, perm):
    """(19, N) library order -> (N, 19) oracle order."""
    out = np.empty((f_gpu.shape[1], 19))
    out[:, perm] = f_gpu.T
    return out


def oracle_f_to_gpu(f_orc, perm):
    return np.ascontiguousarray(f_orc[:, perm].T)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
