"""CPU FP64 oracle of the reactive-mixture lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the independent, slow, obviously
correct restatement of the method that the CUDA library is checked against.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import it; the library and its Python binding never do, and the two share no
code (only the seeded input generators in lbm_workloads serve both).

Modules and the parts of the paper they follow:
  lattice    Sec. 2.2 (velocity set, product form, equilibria), Sec. 3.3-3.4
  thermo     Sec. 2.1 (mixture relations), Sec. 3.1 (energies, temperature)
  chemistry  Sec. 2.4 (reaction term, sub-steps), Sec. 3.6 (rates)
  transport  Sec. 2.3 (relaxation times), Sec. 3.5 (viscosity, conductivity)
  lbm        the whole step (Sec. 2.3, Sec. 3, Sec. 4.1 streaming)
  boundary   Sec. 4 (bounce-back, Tamm-Mott-Smith wall, inlet, outlet)

Parity status per function is listed in the test files that pin them.
"""
from .lbm import OracleLBM, Units, default_reference_speed  # noqa: F401
