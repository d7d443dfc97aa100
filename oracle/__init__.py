"""Plain FP64 CPU oracle of the liquid-gas-solid lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package.  It never imports the GPU
package, and the GPU package never imports it.
"""
from .oracle import GAS, INTERFACE, LIQUID, OBSTACLE, OracleSim, build_oracle, feq, force_term, lattice, set_mutation  # noqa: F401
