"""GB300-native coupled lattice-Boltzmann / immersed-boundary step for
three-bead microswimmers (Geyer et al., arXiv 2202.12147).

The compute path is liblbib.so (hand-written CUDA for sm_103a behind the C ABI
in include/lbib.h); this package only marshals arguments to it.
"""
from . import _lib  # noqa: F401
from .build import build  # noqa: F401


def __getattr__(name):
    # the simulation wrapper needs torch; import it lazily
    if name in ("Simulation", "Batch", "lattice", "required_sizes"):
        from . import sim
        return getattr(sim, name)
    if name in ("Adjoint", "DisplacementFn", "displacement"):
        from . import adjoint
        return getattr(adjoint, name)
    raise AttributeError(name)
