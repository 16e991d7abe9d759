"""GB300 (sm_103a) CUDA implementation of the reactive-mixture lattice
Boltzmann step of Sawant, Dorschner & Karlin (arXiv 2108.07605).

The C ABI is include/lbm.h; `paper_2108_07605_gb300.lbm` is its Python
binding (same function names) and `lbm.Solver` a convenience wrapper.  The
library is built in-tree by `paper_2108_07605_gb300.build.build()`.
"""
