"""FP64 CPU oracle of the coupled LB/IB step (test infrastructure only: used
by the tests, the smoke check and the benchmark's CPU baseline; the product
library never imports it)."""
from .oracle import *  # noqa: F401,F403
from .oracle import OracleSim, build, lattice  # noqa: F401
