"""GB300 (sm_103a) relativistic lattice Boltzmann model with improved dissipation (arXiv:1301.3423).

The compute path is the C-ABI library librlb (include/rlb.h) built from csrc/ for sm_103a; ``rlb``
is its thin Python binding.  ``build()`` compiles the library in-tree."""
from .builder import build
from .rlb import RLB, Batch, RLBError, load, quadrature, read_quadrature_file

__all__ = ["RLB", "Batch", "RLBError", "build", "load", "quadrature", "read_quadrature_file"]
